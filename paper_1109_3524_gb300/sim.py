"""Python binding of the C ABI: torch owns the device workspace and the
stream; every step of the method runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import _abi as A


class IbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{A.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(A.DP)


def _f64(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclasses.dataclass
class Config:
    """Mirror of ibm_config (include/ibm.h)."""
    nx: int
    ny: int
    nu: float
    dt: float
    uinf: float = 1.0
    vinf: float = 0.0
    bc: int = A.IBM_BC_FREESTREAM
    bn_order: int = 1
    h: float = 0.0
    tol1: float = 1e-8
    tol2: float = 1e-8
    max_iter1: int = 1000
    max_iter2: int = 1000
    poisson_precond: int = A.IBM_PRECOND_AMG
    precision: int = A.IBM_PREC_FP64
    warm: int = A.IBM_WARM_PREV
    pin_i: int = 0
    pin_j: int = 0
    amg_theta: float = 0.08
    amg_omega: float = 2.0 / 3.0
    amg_pre: int = 2
    amg_post: int = 2
    amg_max_coarse: int = 256
    amg_max_levels: int = 12
    amg_rebuild_every: int = 2
    moving: int = 0
    amg_trunc: float = 0.1
    amg_tail_rows: int = 16384
    amg_sweeps0: int = 0
    schur_cache: int = -1

    def to_c(self) -> A.ibm_config:
        c = A.ibm_config()
        for f in dataclasses.fields(self):
            setattr(c, f.name, getattr(self, f.name))
        return c

    @classmethod
    def for_case(cls, case, **kw) -> "Config":
        bc = A.IBM_BC_FREESTREAM if case.bc == "freestream" else A.IBM_BC_WALLS
        c = cls(nx=case.nx, ny=case.ny, nu=case.nu, dt=case.dt, uinf=case.uinf, vinf=case.vinf,
                bc=bc, h=case.h, moving=int(case.moving))
        for k, v in kw.items():
            setattr(c, k, v)
        return c


def _stats_dict(s: A.ibm_solve_stats) -> dict:
    return {"iters": s.iters, "status": s.status, "rel_res": s.rel_res, "rel_res0": s.rel_res0}


class Sim:
    """One simulation context bound to a CUDA device."""

    def __init__(self, cfg: Config, xf, yf, xb=None, yb=None, device="cuda:0", stream=None):
        import torch
        self._torch = torch
        self.lib = A.load()
        self.cfg = cfg
        xf, yf = _f64(xf), _f64(yf)
        xb = _f64(xb) if xb is not None else np.zeros(0)
        yb = _f64(yb) if yb is not None else np.zeros(0)
        self.n_b = len(xb)
        ctx = A.CTX()
        cc = cfg.to_c()
        rc = self.lib.ibm_create(C.byref(cc), _dp(xf), _dp(yf), self.n_b, _dp(xb), _dp(yb), C.byref(ctx))
        self.ctx = ctx
        if rc:
            msg = self.lib.ibm_last_error(ctx).decode() if ctx else ""
            self.close()
            raise IbmError(rc, msg)
        nbytes = C.c_size_t()
        self._check(self.lib.ibm_workspace_bytes(ctx, C.byref(nbytes)))
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        if self.workspace.data_ptr() % 256:
            raise IbmError(A.IBM_ERR_ARG, "torch workspace is not 256-byte aligned")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.lib.ibm_bind_workspace(ctx, C.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                                C.c_void_p(self.stream.cuda_stream)))
        nq, nl, nb = C.c_int64(), C.c_int64(), C.c_int32()
        self._check(self.lib.ibm_sizes(ctx, C.byref(nq), C.byref(nl), C.byref(nb)))
        self.n_q, self.n_lambda = nq.value, nl.value
        npad = C.c_int64()
        self._check(self.lib.ibm_layout(ctx, C.byref(npad)))
        self.nq_padded = npad.value

    @classmethod
    def from_case(cls, case, device="cuda:0", **cfg_kw) -> "Sim":
        cfg = Config.for_case(case, **cfg_kw)
        xb, yb, _, _ = case.body_state(0.0)
        s = cls(cfg, case.xf, case.yf, xb, yb, device=device)
        if case.n_b:
            xb, yb, ub, vb = case.body_state(case.dt)
            s.set_body(xb, yb, ub, vb)
        return s

    # ------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != A.IBM_OK:
            raise IbmError(rc, self.lib.ibm_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ibm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def set_body(self, xb, yb, ub=None, vb=None):
        xb, yb, ub, vb = _f64(xb), _f64(yb), _f64(ub), _f64(vb)
        self._check(self.lib.ibm_set_body(self.ctx, _dp(xb), _dp(yb), _dp(ub), _dp(vb)))

    def step(self, n: int = 1, check: bool = True):
        st = (A.ibm_step_stats * max(n, 1))()
        rc = self.lib.ibm_step(self.ctx, n, st)
        if check and rc not in (A.IBM_OK,):
            self._check(rc)
        out = []
        for k in range(n):
            s = st[k]
            out.append({"t": s.t, "solve1": _stats_dict(s.solve1), "solve2": _stats_dict(s.solve2),
                        "fx": s.fx, "fy": s.fy, "cd": s.cd, "cl": s.cl, "div_max": s.div_max,
                        "slip_max": s.slip_max, "poisson_ms": s.poisson_ms,
                        "poisson_bytes": s.poisson_bytes, "amg_rebuilt": s.amg_rebuilt})
        return out

    def solve_poisson(self, rhs, lam0=None):
        """rhs, lam0: CUDA float64 tensors of n_lambda; returns (lambda, stats)."""
        torch = self._torch
        lam = torch.empty(self.n_lambda, dtype=torch.float64, device=self.device)
        s = A.ibm_solve_stats()
        rc = self.lib.ibm_solve_poisson(self.ctx, C.c_void_p(rhs.data_ptr()), C.c_void_p(lam.data_ptr()),
                                        C.c_void_p(lam0.data_ptr()) if lam0 is not None else None, C.byref(s))
        if rc not in (A.IBM_OK, A.IBM_ERR_NOT_CONVERGED):
            self._check(rc)
        return lam, _stats_dict(s)

    def apply_poisson(self, x):
        torch = self._torch
        y = torch.empty_like(x)
        self._check(self.lib.ibm_apply_poisson(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def residual_norms_noalloc(self, lam, rhs):
        """(||rhs||^2, ||rhs - S lam||^2) through the allocation-free entry
        point (no device memory is allocated by the call)."""
        out = np.zeros(2)
        self._check(self.lib.ibm_poisson_residual_norms_noalloc(
            self.ctx, C.c_void_p(lam.data_ptr()), C.c_void_p(rhs.data_ptr()), _dp(out)))
        return float(out[0]), float(out[1])

    def vcycle(self, r):
        torch = self._torch
        z = torch.empty_like(r)
        self._check(self.lib.ibm_vcycle(self.ctx, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr())))
        return z

    def forces(self):
        fx = np.zeros(self.n_b)
        fy = np.zeros(self.n_b)
        cd, cl = C.c_double(), C.c_double()
        self._check(self.lib.ibm_forces(self.ctx, _dp(fx), _dp(fy), C.byref(cd), C.byref(cl)))
        return fx, fy, cd.value, cl.value

    def get_state(self):
        nx, ny = self.cfg.nx, self.cfg.ny
        u = np.zeros((ny, nx + 1))
        v = np.zeros((ny + 1, nx))
        vr = np.zeros(ny + 1)
        npv = np.zeros(self.nq_padded)
        lam = np.zeros(self.n_lambda)
        t = C.c_double()
        step = C.c_int64()
        self._check(self.lib.ibm_get_state(self.ctx, _dp(u), _dp(v), _dp(vr), _dp(npv), _dp(lam),
                                           C.byref(t), C.byref(step)))
        return {"u": u, "v": v, "v_right": vr, "nprev": npv, "lambda": lam, "t": t.value, "step": step.value}

    def set_state(self, u=None, v=None, v_right=None, nprev=None, lam=None, t=0.0, step=0):
        u, v, v_right, nprev, lam = (_f64(a) for a in (u, v, v_right, nprev, lam))
        self._check(self.lib.ibm_set_state(self.ctx, _dp(u), _dp(v), _dp(v_right), _dp(nprev), _dp(lam),
                                           float(t), int(step)))

    # ------------------------------------------------------------------
    def amg_levels(self) -> int:
        n = C.c_int32()
        self._check(self.lib.ibm_amg_levels(self.ctx, C.byref(n)))
        return n.value

    def amg_level_info(self, level: int):
        n, w = C.c_int64(), C.c_double()
        self._check(self.lib.ibm_amg_level_info(self.ctx, level, C.byref(n), C.byref(w)))
        return n.value, w.value

    def amg_matrix(self, level: int, which: int = 0):
        """(n, m, rowptr, col, val) of the level operator (which=0), its
        prolongator (1), or its fused transfers Rt (2) and Q (3)."""
        n, m, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.ibm_amg_matrix(self.ctx, level, which, C.byref(n), C.byref(m), C.byref(nnz),
                                            None, None, None))
        rp = np.zeros(n.value + 1, dtype=np.int64)
        ci = np.zeros(nnz.value, dtype=np.int32)
        va = np.zeros(nnz.value)
        self._check(self.lib.ibm_amg_matrix(self.ctx, level, which, None, None, None,
                                            rp.ctypes.data_as(A.I64P), ci.ctypes.data_as(A.I32P), _dp(va)))
        return n.value, m.value, rp, ci, va

    def profile(self, on: bool = True):
        self._check(self.lib.ibm_profile_enable(self.ctx, 1 if on else 0))

    def profile_reset(self):
        self._check(self.lib.ibm_profile_reset(self.ctx))

    def profile_read(self) -> dict:
        n = C.c_int32()
        self._check(self.lib.ibm_profile_count(self.ctx, C.byref(n)))
        out = {}
        for k in range(n.value):
            name = C.c_char_p()
            la = C.c_int64()
            ms = C.c_double()
            by = C.c_double()
            self._check(self.lib.ibm_profile_get(self.ctx, k, C.byref(name), C.byref(la), C.byref(ms),
                                                 C.byref(by)))
            out[name.value.decode()] = {"launches": la.value, "ms": ms.value, "bytes": by.value}
        return out

    def profile_graph_class(self, name: str, reps: int = 20) -> dict:
        """Graph-mode time per launch of one kernel class (runs one more step;
        the context's state is not usable afterwards)."""
        n = C.c_int32()
        self._check(self.lib.ibm_profile_count(self.ctx, C.byref(n)))
        names = []
        for k in range(n.value):
            nm = C.c_char_p()
            self._check(self.lib.ibm_profile_get(self.ctx, k, C.byref(nm), None, None, None))
            names.append(nm.value.decode())
        k = names.index(name)
        la, ms, by = C.c_int64(), C.c_double(), C.c_double()
        self._check(self.lib.ibm_profile_graph_class(self.ctx, k, reps, C.byref(la), C.byref(ms), C.byref(by)))
        return {"launches": la.value, "ms_per_launch": ms.value, "bytes_per_launch": by.value}

    def transfer_bytes(self):
        h, d = C.c_int64(), C.c_int64()
        self._check(self.lib.ibm_transfer_bytes(self.ctx, C.byref(h), C.byref(d)))
        return h.value, d.value

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.ibm_launch_count(self.ctx, C.byref(n)))
        return n.value


def create_host_only(cfg: Config, xf, yf, xb=None, yb=None):
    """Host-side set-up without a GPU (ibm_create only): returns a handle
    whose AMG hierarchy and sizes can be inspected."""
    return HostCtx(cfg, xf, yf, xb, yb)


class HostCtx:
    def __init__(self, cfg, xf, yf, xb=None, yb=None):
        self.lib = A.load()
        xf, yf = _f64(xf), _f64(yf)
        xb = _f64(xb) if xb is not None else np.zeros(0)
        yb = _f64(yb) if yb is not None else np.zeros(0)
        self.ctx = A.CTX()
        cc = cfg.to_c()
        rc = self.lib.ibm_create(C.byref(cc), _dp(xf), _dp(yf), len(xb), _dp(xb), _dp(yb), C.byref(self.ctx))
        if rc:
            msg = self.lib.ibm_last_error(self.ctx).decode() if self.ctx else ""
            raise IbmError(rc, msg)

    amg_levels = Sim.amg_levels
    amg_matrix = Sim.amg_matrix
    amg_level_info = Sim.amg_level_info
    _check = Sim._check

    def workspace_bytes(self) -> int:
        n = C.c_size_t()
        self._check(self.lib.ibm_workspace_bytes(self.ctx, C.byref(n)))
        return n.value

    def close(self):
        if self.ctx:
            self.lib.ibm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Unet:
    """The warm-start U-Net (ibm_cnn_* in include/ibm.h): parameters, Adam
    state and activations live in one torch-owned device workspace."""

    def __init__(self, base=16, levels=4, max_pixels=1 << 20, device="cuda:0", stream=None):
        import torch
        self._torch = torch
        self.lib = A.load()
        self.base, self.levels = base, levels
        self.net = A.CTX()
        rc = self.lib.ibm_cnn_create(base, levels, int(max_pixels), C.byref(self.net))
        if rc:
            raise IbmError(rc, "ibm_cnn_create")
        nb = C.c_size_t()
        self._check(self.lib.ibm_cnn_workspace_bytes(self.net, C.byref(nb)))
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.lib.ibm_cnn_bind(self.net, C.c_void_p(self.workspace.data_ptr()), nb.value,
                                          C.c_void_p(self.stream.cuda_stream)))
        n = C.c_int64()
        self._check(self.lib.ibm_cnn_param_count(self.net, C.byref(n)))
        self.n_params = n.value

    def _check(self, rc):
        if rc != A.IBM_OK:
            raise IbmError(rc, self.lib.ibm_cnn_last_error(self.net).decode())

    def conv_shapes(self, cin=3, cout=1):
        """(k, cin, cout) of every convolution in parameter order: two 3x3
        convolutions per encoder level (base * 2^l channels), two per decoder
        level after the skip concatenation, and the final 1x1 convolution."""
        ch = [self.base * (2 ** l) for l in range(self.levels)]
        out, c = [], cin
        for l in range(self.levels):
            out += [(3, c, ch[l]), (3, ch[l], ch[l])]
            c = ch[l]
        for l in range(self.levels - 2, -1, -1):
            out += [(3, c + ch[l], ch[l]), (3, ch[l], ch[l])]
            c = ch[l]
        out.append((1, c, cout))
        return out

    def init_params(self, seed=0):
        """He-normal initial weights from the seeded generator of `workloads`."""
        import workloads
        self.set_params(workloads.he_normal(self.conv_shapes(), seed=seed))

    def close(self):
        if getattr(self, "net", None):
            self.lib.ibm_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        theta = _f64(theta)
        self._check(self.lib.ibm_cnn_set_params(self.net, _dp(theta), theta.size))

    def get_params(self):
        out = np.zeros(self.n_params)
        self._check(self.lib.ibm_cnn_get_params(self.net, _dp(out), out.size))
        return out

    def forward(self, x):
        """x: float32 CUDA tensor (B, H, W, 3) -> (B, H, W)."""
        B, H, W, _ = x.shape
        y = self._torch.empty((B, H, W), dtype=self._torch.float32, device=self.device)
        self._check(self.lib.ibm_cnn_forward(self.net, B, H, W, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, x, t, want_grad=False):
        B, H, W, _ = x.shape
        loss = C.c_double()
        g = np.zeros(self.n_params) if want_grad else None
        self._check(self.lib.ibm_cnn_loss_grad(self.net, B, H, W, C.c_void_p(x.data_ptr()),
                                               C.c_void_p(t.data_ptr()), C.byref(loss), _dp(g)))
        return loss.value, g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.ibm_cnn_adam_step(self.net, lr, beta1, beta2, eps))

    def layers(self):
        """Per convolution: dict(cin, cout, ks, level, tcgen05)."""
        out = []
        n = 2 * self.levels + 2 * (self.levels - 1) + 1
        for i in range(n):
            v = [C.c_int32() for _ in range(5)]
            self._check(self.lib.ibm_cnn_layer_info(self.net, i, *[C.byref(x) for x in v]))
            out.append(dict(zip(("cin", "cout", "ks", "level", "tcgen05"), (x.value for x in v))))
        return out

    def time_forward(self, batch, h, w, reps=20):
        """Mean milliseconds of each convolution of the forward pass (CUDA
        events on the network's stream) on the input in the workspace."""
        n = 2 * self.levels + 2 * (self.levels - 1) + 1
        ms = np.zeros(n)
        self._check(self.lib.ibm_cnn_time_forward(self.net, batch, h, w, reps, _dp(ms), n))
        return ms

    def set_window(self, x0=0, y0=0, w=0, h=0):
        """Inference window of the warm start (cells [x0, x0+w) x [y0, y0+h));
        w = h = 0: the whole grid."""
        self._check(self.lib.ibm_cnn_set_window(self.net, int(x0), int(y0), int(w), int(h)))

    def prepare(self, nx, ny, phi_n, phi_nm1, b_phi, phi_np1, crops, crop_h, crop_w):
        """Standardised inputs (ncrop, crop_h, crop_w, 3) and targets from
        device pressure fields (nx*ny float64 each); crops: (ncrop, 2) int
        array of (x0, y0)."""
        torch = self._torch
        xy = np.ascontiguousarray(np.asarray(crops, dtype=np.int32).reshape(-1))
        n = xy.size // 2
        x = torch.empty((n, crop_h, crop_w, 3), dtype=torch.float32, device=self.device)
        t = torch.empty((n, crop_h, crop_w), dtype=torch.float32, device=self.device) if phi_np1 is not None else None
        self._check(self.lib.ibm_cnn_prepare(
            self.net, nx, ny, C.c_void_p(phi_n.data_ptr()), C.c_void_p(phi_nm1.data_ptr()),
            C.c_void_p(b_phi.data_ptr()), C.c_void_p(phi_np1.data_ptr()) if phi_np1 is not None else None,
            n, xy.ctypes.data_as(A.I32P), crop_h, crop_w, C.c_void_p(x.data_ptr()),
            C.c_void_p(t.data_ptr()) if t is not None else None))
        return x, t


def _sim_attach(self, net):
    self._check(self.lib.ibm_attach_cnn(self.ctx, net.net if net is not None else None))
    self._net = net


def _sim_snapshot(self):
    torch = self._torch
    lam = torch.empty(self.n_lambda, dtype=torch.float64, device=self.device)
    prev = torch.empty_like(lam)
    rhs = torch.empty_like(lam)
    r0 = torch.empty_like(lam)
    self._check(self.lib.ibm_snapshot(self.ctx, C.c_void_p(lam.data_ptr()), C.c_void_p(prev.data_ptr()),
                                      C.c_void_p(rhs.data_ptr()), C.c_void_p(r0.data_ptr())))
    return lam, prev, rhs, r0


Sim.attach_cnn = _sim_attach
Sim.snapshot = _sim_snapshot
