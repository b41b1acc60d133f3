"""Pins of the NumPy U-Net reference: convolution against an independent
scipy.signal correlation, pooling/upsampling adjoints, and the full backward
pass against central finite differences."""
import numpy as np
import scipy.signal

import workloads as W
from oracle import unet_ref as U


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    Wt = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    y = U.conv(x, Wt, b)
    for n in range(2):
        for co in range(4):
            ref = sum(scipy.signal.correlate2d(x[n, :, :, ci], Wt[:, :, ci, co], mode="same")
                      for ci in range(3)) + b[co]
            assert np.allclose(y[n, :, :, co], ref, rtol=0, atol=1e-12)


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 8, 6, 3))
    c = rng.standard_normal((2, 4, 3, 3))
    assert abs(np.sum(U.pool(a) * c) - np.sum(a * U.pool_backward(c))) < 1e-12
    assert abs(np.sum(U.up(c) * a) - np.sum(c * U.up_backward(a))) < 1e-12


def test_backward_matches_finite_differences():
    specs = U.conv_specs(base=2, levels=3)
    theta = W.he_normal([(k, ci, co) for ci, co, k in specs], seed=1)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 8, 8, 3))
    t = rng.standard_normal((2, 8, 8, 1))
    _, g = U.loss_and_grad(theta, x, t, specs, levels=3)
    eps = 1e-6
    for i in rng.choice(theta.size, 30, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (U.loss_and_grad(tp, x, t, specs, 3)[0] - U.loss_and_grad(tm, x, t, specs, 3)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(1e-6, abs(fd) + abs(g[i])), (i, fd, g[i])


def test_he_normal_statistics():
    th = W.he_normal([(3, 16, 32)], seed=5)
    w = th[:3 * 3 * 16 * 32]
    assert abs(w.mean()) < 0.02 and abs(w.std() - np.sqrt(2.0 / 144)) < 0.01
    assert np.all(th[-32:] == 0.0)


def test_library_network_shapes_match_reference():
    """The binding's layer list (used for initialisation) is the network the
    reference defines."""
    from paper_1109_3524_gb300.sim import Unet

    class Shape:
        pass

    for base, levels in ((16, 4), (4, 3), (8, 2)):
        f = Shape()
        f.base, f.levels = base, levels
        assert Unet.conv_shapes(f) == [(k, ci, co) for ci, co, k in U.conv_specs(base, levels)]
