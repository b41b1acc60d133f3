"""The warm-start U-Net on the GPU (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 NumPy reference, and its use in a time step."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from oracle import unet_ref as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1109_3524_gb300 as P
    from paper_1109_3524_gb300.build import ensure_built
    ensure_built()
    P.load()
    return P


def _small(pkg, base=4, levels=3, seed=2):
    specs = U.conv_specs(base, levels)
    theta = W.he_normal([(k, ci, co) for ci, co, k in specs], seed=seed)
    net = pkg.Unet(base, levels, max_pixels=4 * 32 * 32)
    net.set_params(theta)
    return net, specs, theta


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def test_params_roundtrip(pkg):
    net, specs, theta = _small(pkg)
    assert net.n_params == U.n_params(specs)
    back = net.get_params()
    assert np.abs(back - theta).max() <= 1e-6 * np.abs(theta).max()   # FP32 master copy


@pytest.mark.parametrize("levels,base", [(3, 4), (4, 8)])
def test_forward_matches_reference(pkg, levels, base):
    import torch
    net, specs, theta = _small(pkg, base, levels)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 16, 24, 3))
    y = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    yr = U.forward(theta, x, specs, levels)[..., 0]
    # BF16 weights and activations (8-bit mantissa), FP32 accumulation
    assert _rel(y, yr) < 3e-2, _rel(y, yr)


def test_tensor_core_forward_matches_mma_sync(pkg, monkeypatch):
    """The benchmark network (base 16, 4 levels): every 3x3 convolution of the
    forward pass on tcgen05 (accumulator in tensor memory, weights staged by
    bulk copies) against the same network with every convolution on the
    mma.sync implicit GEMM (IBM_CNN_NO_TC=1), on a batch of 3 non-square
    images whose sizes leave ragged 8 x 16 tiles on every level.  Both take
    the same BF16 operands and accumulate in FP32 in different orders, so the
    outputs agree to about the BF16 rounding of the activations (1e-2); both
    follow the FP64 reference to 3e-2."""
    import torch
    specs = U.conv_specs(16, 4)
    theta = W.he_normal([(k, ci, co) for ci, co, k in specs], seed=7)
    shape = (3, 48, 80)
    net_tc = pkg.Unet(16, 4, max_pixels=int(np.prod(shape)))
    monkeypatch.setenv("IBM_CNN_NO_TC", "1")
    net_ms = pkg.Unet(16, 4, max_pixels=int(np.prod(shape)))
    monkeypatch.delenv("IBM_CNN_NO_TC")
    net_tc.set_params(theta)
    net_ms.set_params(theta)
    x = np.random.default_rng(8).standard_normal(shape + (3,))
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    y_tc = net_tc.forward(xt).cpu().numpy()
    y_ms = net_ms.forward(xt).cpu().numpy()
    yr = U.forward(theta, x, specs, 4)[..., 0]
    print(f"tcgen05 vs mma.sync {_rel(y_tc, y_ms):.3e}, vs FP64 {_rel(y_tc, yr):.3e} (mma.sync {_rel(y_ms, yr):.3e})")
    assert _rel(y_tc, y_ms) < 1e-2
    assert _rel(y_tc, yr) < 3e-2


def test_gradients_match_reference(pkg):
    """Toy network (3 levels, base 4): the whole gradient against the FP64
    reference.  BF16 activations and pre-activation gradients (unit roundoff
    2^-8) flip ReLU masks near zero and compound through the backward chain,
    so FP64 is checked on the whole gradient (8%) and its direction (cosine
    0.99); the per-layer check is on the full-size network below."""
    import torch
    net, specs, theta = _small(pkg, 4, 3)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((3, 16, 16, 3))
    t = rng.standard_normal((3, 16, 16))
    loss, g = net.loss_grad(torch.tensor(x, dtype=torch.float32, device="cuda"),
                            torch.tensor(t, dtype=torch.float32, device="cuda"), want_grad=True)
    lr, gr = U.loss_and_grad(theta, x, t[..., None], specs, 3)
    assert abs(loss - lr) < 3e-2 * lr
    assert _rel(g, gr) < 8e-2, _rel(g, gr)
    assert g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr)) > 0.99


def test_gradients_per_layer_on_the_benchmark_network(pkg):
    """The benchmark's network (4 levels, 16-32-64-128 channels) on a
    non-square batch of 4 x 64 x 96 pixels: the weight and the bias gradient
    of every convolution separately against the reference that rounds the
    convolution operands to BF16 where the kernels store them (network input,
    weights, post-ReLU and pooled activations, pre-activation gradients), to
    2% relative.  The two sides round the same quantities; they differ by
    FP32 against FP64 accumulation ahead of each rounding, which moves
    individual rounded values by one BF16 unit and leaves a noise of about
    1% per layer at this size (the FP64 reference is as far from the rounding
    one).  A wrong tap, transposed weight or dropped bias term is off by
    order one."""
    import torch
    base, levels = 16, 4
    specs = U.conv_specs(base, levels)
    theta = W.he_normal([(k, ci, co) for ci, co, k in specs], seed=2)
    B, H, Wd = 4, 64, 96
    net = pkg.Unet(base, levels, max_pixels=B * H * Wd)
    net.set_params(theta)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((B, H, Wd, 3))
    t = rng.standard_normal((B, H, Wd))
    loss, g = net.loss_grad(torch.tensor(x, dtype=torch.float32, device="cuda"),
                            torch.tensor(t, dtype=torch.float32, device="cuda"), want_grad=True)
    U.ROUND = U.bf16_round
    try:
        lb, gb = U.loss_and_grad(theta, x, t[..., None], specs, levels)
    finally:
        U.ROUND = None
    assert abs(loss - lb) < 1e-3 * lb
    o = 0
    ew, eb = [], []
    for ci, co, k in specs:
        nw = k * k * ci * co
        ew.append(_rel(g[o:o + nw], gb[o:o + nw]))
        eb.append(_rel(g[o + nw:o + nw + co], gb[o + nw:o + nw + co]))
        o += nw + co
    print("per-layer relative error, weights:", np.round(ew, 4).tolist())
    print("per-layer relative error, biases: ", np.round(eb, 4).tolist())
    assert max(ew) < 2e-2 and max(eb) < 2e-2, (ew, eb)
    net.close()


def test_adam_reduces_the_loss(pkg):
    import torch
    net, specs, theta = _small(pkg, 4, 3)
    rng = np.random.default_rng(8)
    x = torch.tensor(rng.standard_normal((4, 16, 16, 3)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.standard_normal((4, 16, 16)) * 0.1, dtype=torch.float32, device="cuda")
    first, _ = net.loss_grad(x, t)
    for _ in range(60):
        loss, _ = net.loss_grad(x, t)
        net.adam_step(3e-3)
    assert loss < 0.5 * first, (first, loss)


@pytest.mark.parametrize("window", [None, (32, 48, 64, 32)])
def test_learned_warm_start_keeps_the_solution(pkg, window):
    """With the network attached (on the whole grid, or on a window of cells
    around the body) the converged step still equals the oracle's direct
    solve (the warm start only changes the initial guess)."""
    case = W.cylinder_re40_128()
    sim = pkg.Sim.from_case(case, tol1=1e-12, tol2=1e-12, warm=pkg.IBM_WARM_CNN,
                            poisson_precond=pkg.IBM_PRECOND_SCHUR)
    U0, V0 = case.initial_velocity()
    sim.set_state(u=U0, v=V0, v_right=np.zeros(case.ny + 1))
    net = pkg.Unet(8, 4, max_pixels=case.nx * case.ny, stream=sim.stream)
    specs = U.conv_specs(8, 4)
    net.set_params(W.he_normal([(k, ci, co) for ci, co, k in specs], seed=3) * 0.1)
    if window:
        net.set_window(*window)
    sim.attach_cnn(net)
    o = Oracle(case)
    for _ in range(4):
        xb, yb, ub, vb = case.body_state(o.t + case.dt)
        sim.set_body(xb, yb, ub, vb)
        st = sim.step(1)[0]
        o.step()
        assert st["solve2"]["status"] == 0
    s = sim.get_state()
    Uo, Vo = o.face_arrays()
    assert np.abs(s["u"] - Uo).max() < 1e-8 * np.abs(Uo).max()
    assert _rel(s["lambda"], o.lam) < 1e-8


def test_trained_warm_start_gain_is_measured(pkg):
    """Trains the network on the solver's own snapshots (128^2 workload,
    90/10 split by time) with the library's kernels and measures what it
    gains on the held-out steps: the training loss falls by two orders of
    magnitude, the network reduces the error of the extrapolated guess on
    training samples, and on the held-out steps the Poisson iteration count is
    at least half an iteration per step below the extrapolated warm start
    (both below the plain lambda^n warm start)."""
    from paper_1109_3524_gb300 import warmstart as WS
    case = W.cylinder_re40_128()
    phi, r0, state, t_end = WS.generate_snapshots(case, 240)
    net = pkg.Unet(16, 4, max_pixels=max(case.nx * case.ny, 8 * 64 * 64))
    specs = U.conv_specs(16, 4)
    net.set_params(W.he_normal([(k, ci, co) for ci, co, k in specs], seed=0))
    hist = WS.train(net, phi[:216], r0[:216], case.nx, case.ny, steps=800, batch=8, crop=64, lr=1e-3)
    assert np.mean(hist[-20:]) < 0.05 * hist[0]
    assert WS.prediction_error(net, phi, r0, case.nx, case.ny, list(range(2, 20))) < 1.0
    res = WS.compare_iterations(case, net, state, t_end, 12)
    print("warm-start comparison:", res)
    assert res["extrap"]["k2_mean"] < res["prev"]["k2_mean"]
    # the held-out gain: at least half a Poisson iteration per step below the
    # extrapolated warm start (training is deterministic: the weight-gradient
    # slices are summed in a fixed order; measured on GB300: 10.5 against 13.0)
    assert res["cnn"]["k2_mean"] <= res["extrap"]["k2_mean"] - 0.5, res
