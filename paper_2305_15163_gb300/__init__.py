"""Python binding of libddnm.so, the GB300 (sm_103a) library for the online solve of the
DD NM-ROM with hyper-reduction (arXiv 2305.15163, Sec. 3.1 / 4.1 / 7.1).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
The functions keep the C names of ``include/ddnm.h``; ``Solver`` bundles them.
Arrays may be numpy (host memory) or torch CUDA tensors (device memory, queued on
the current torch stream).  There is no CPU path: if the library cannot be loaded,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddnm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2305_15163_gb300/build.py` "
                      "(or __graft_entry__.build()); there is no fallback implementation")
_lib = C.CDLL(LIB_PATH)

DDNM_OK, DDNM_E_INVALID, DDNM_E_STATE, DDNM_E_CUDA, DDNM_E_NOMEM, DDNM_E_UNSUPPORTED = 0, -1, -2, -3, -4, -5
DDNM_FP64, DDNM_MIXED = 0, 1
DDNM_ACT = {"swish": 0, "sigmoid": 1, "identity": 2}
DDNM_MEM_HOST, DDNM_MEM_DEVICE = 0, 1
DDNM_DECODER_INTERIOR, DDNM_DECODER_INTERFACE = 0, 1
DDNM_CONVERGED, DDNM_MAX_ITER, DDNM_NONFINITE, DDNM_KKT_FAIL = 0, 1, 2, 3
DDNM_FLAG_LS_FAIL, DDNM_FLAG_WS_FALLBACK, DDNM_FLAG_STEP = 1, 2, 4

_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class ddnm_problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nu", C.c_double), ("box", C.c_double * 4),
                ("kx", C.c_int), ("ky", C.c_int), ("xb", _ip), ("yb", _ip), ("n_omega", _ip),
                ("n_gamma", _ip), ("hr_count", _ip), ("hr_rows", _ip), ("n_c", C.c_int),
                ("precision", C.c_int), ("device", C.c_int)]


class ddnm_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("armijo_c1", C.c_double),
                ("beta", C.c_double), ("max_backtracks", C.c_int), ("step_tol", C.c_double)]


class ddnm_decoder(C.Structure):
    _fields_ = [("N", C.c_int), ("w", C.c_int), ("n", C.c_int), ("act", C.c_int), ("K", C.c_int),
                ("W1", _dp), ("b1", _dp), ("cols", _ip), ("vals", _dp), ("scale", _dp), ("offset", _dp)]


class ddnm_encoder(C.Structure):
    _fields_ = [("N", C.c_int), ("w", C.c_int), ("n", C.c_int), ("Kt", C.c_int), ("cols", _ip), ("vals", _dp),
                ("b1", _dp), ("W2", _dp)]


class ddnm_sizes(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("N_x", C.c_int), ("n_D", C.c_int), ("n_C", C.c_int),
                ("N_A", C.c_int), ("sum_hr", C.c_int), ("sum_gamma", C.c_int)]


class ddnm_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("flags", C.c_int), ("n_evals", C.c_int),
                ("merit", C.c_double), ("alpha_last", C.c_double)]


class ddnm_timing(C.Structure):
    _fields_ = [("eval_ms", C.c_double), ("constraint_ms", C.c_double), ("step_ms", C.c_double),
                ("eval_launches", C.c_longlong), ("constraint_launches", C.c_longlong),
                ("step_launches", C.c_longlong), ("other_launches", C.c_longlong)]


class ddnm_work(C.Structure):
    _fields_ = [("eval_flops", C.c_double), ("eval_fp64_flops", C.c_double), ("eval_bytes", C.c_double),
                ("constraint_fp64_flops", C.c_double), ("step_fp64_flops", C.c_double),
                ("table_bytes", C.c_double), ("instance_bytes", C.c_double)]


class ddnm_tune(C.Structure):
    _fields_ = [("graph", C.c_int), ("chains", C.c_int), ("con_split", C.c_int), ("eval_persist", C.c_int),
                ("d_gemm", C.c_int), ("eval_groups", C.c_int), ("atil", C.c_int)]


FOM_STATS_DTYPE = np.dtype([("newton_iters", np.int32), ("krylov_iters", np.int32), ("status", np.int32),
                            ("pad", np.int32), ("res0", np.float64), ("res", np.float64)])

STATS_DTYPE = np.dtype([("iters", np.int32), ("status", np.int32), ("flags", np.int32),
                        ("n_evals", np.int32), ("merit", np.float64), ("alpha_last", np.float64)])

_vp = C.c_void_p
_sig = {
    "ddnm_setup": (C.c_int, [C.POINTER(ddnm_problem), C.POINTER(_vp)]),
    "ddnm_destroy": (None, [_vp]),
    "ddnm_last_error": (C.c_char_p, [_vp]),
    "ddnm_get_sizes": (C.c_int, [_vp, C.POINTER(ddnm_sizes)]),
    "ddnm_get_subdomain": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "ddnm_get_constraints": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ddnm_set_test_matrix": (C.c_int, [_vp, _vp]),
    "ddnm_load_decoders": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(ddnm_decoder)]),
    "ddnm_set_options": (C.c_int, [_vp, C.POINTER(ddnm_options)]),
    "ddnm_solve_batch": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "ddnm_residual": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "ddnm_linearize": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "ddnm_reconstruct": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "ddnm_residual_noalloc": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "ddnm_ws_init": (C.c_int, [_vp, C.c_int, _vp]),
    "ddnm_ws_set_norm": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ddnm_ws_loss_grad": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "ddnm_ws_train": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_double, _vp, _vp]),
    "ddnm_ws_predict": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "ddnm_ws_get_params": (C.c_int, [_vp, _vp, _vp]),
    "ddnm_ws_enable": (C.c_int, [_vp, C.c_int]),
    "ddnm_ws_save": (C.c_int, [_vp, C.c_char_p]),
    "ddnm_ws_load": (C.c_int, [_vp, C.c_char_p]),
    "ddnm_load_encoder": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(ddnm_encoder)]),
    "ddnm_ae_train": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_int, C.c_double, _vp, _vp, C.c_int, _vp]),
    "ddnm_ae_loss_grad": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]),
    "ddnm_ae_layout": (C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    "ddnm_get_decoder": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "ddnm_fom_solve": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "ddnm_measure_peaks": (C.c_int, [_vp, _dp, _dp]),
    "ddnm_fom_residual": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int, _vp]),
    "ddnm_set_hr_projection": (C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    "ddnm_hr_select": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "ddnm_get_ports": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "ddnm_set_srpc": (C.c_int, [_vp, C.c_int]),
    "ddnm_load_port_decoder": (C.c_int, [_vp, C.c_int, C.POINTER(ddnm_decoder)]),
    "ddnm_get_port_matrix": (C.c_int, [_vp, C.c_int, _vp]),
    "ddnm_timing_enable": (C.c_int, [_vp, C.c_int]),
    "ddnm_get_timing": (C.c_int, [_vp, C.POINTER(ddnm_timing)]),
    "ddnm_get_work": (C.c_int, [_vp, C.POINTER(ddnm_work)]),
    "ddnm_set_tune": (C.c_int, [_vp, C.POINTER(ddnm_tune)]),
    "ddnm_get_tune": (C.c_int, [_vp, C.POINTER(ddnm_tune)]),
    "ddnm_autotune": (C.c_int, [_vp, C.c_int, _vp, C.c_int, _vp, C.c_int, C.c_int, C.POINTER(ddnm_tune),
                                C.POINTER(C.c_float)]),
}
for _n, (_res, _args) in _sig.items():
    _f = getattr(_lib, _n)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class DDNMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ddnm error {code}: {msg}")
        self.code = code


def ddnm_last_error(ctx) -> str:
    return (_lib.ddnm_last_error(ctx) or b"").decode()


def _check(ctx, rc):
    if rc != DDNM_OK:
        raise DDNMError(rc, ddnm_last_error(ctx))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()   # torch tensor


# ------------------------------------------------------------------ C entry points

def ddnm_setup(nx, ny, xb, yb, n_omega, n_gamma, hr_count, hr_rows, n_c, precision=DDNM_MIXED,
               nu=0.1, box=(-1.0, 1.0, -1.0, 1.0), device=0):
    keep = [_i32(xb), _i32(yb), _i32(n_omega), _i32(n_gamma), _i32(hr_count), _i32(hr_rows)]
    p = ddnm_problem(nx, ny, nu, (C.c_double * 4)(*box), len(keep[0]) - 1, len(keep[1]) - 1,
                     *[k.ctypes.data_as(_ip) for k in keep], n_c, precision, device)
    ctx = _vp()
    _check(None, _lib.ddnm_setup(C.byref(p), C.byref(ctx)))
    return ctx


def ddnm_destroy(ctx):
    _lib.ddnm_destroy(ctx)


def ddnm_get_sizes(ctx) -> ddnm_sizes:
    s = ddnm_sizes()
    _check(ctx, _lib.ddnm_get_sizes(ctx, C.byref(s)))
    return s


def ddnm_get_subdomain(ctx, sub):
    info = np.zeros(6, dtype=np.int32)
    _check(ctx, _lib.ddnm_get_subdomain(ctx, sub, info.ctypes.data, None, None))
    inter = np.zeros(info[1], dtype=np.int32)
    face = np.zeros(info[2], dtype=np.int32)
    _check(ctx, _lib.ddnm_get_subdomain(ctx, sub, info.ctypes.data, inter.ctypes.data, face.ctypes.data))
    return dict(N_r=int(info[0]), N_omega=int(info[1]), N_gamma=int(info[2]), n_omega=int(info[3]),
                n_gamma=int(info[4]), N_B=int(info[5]), interior=inter, interface=face)


def ddnm_get_constraints(ctx):
    n = ddnm_get_sizes(ctx).N_A
    var, lo, hi = (np.zeros(n, dtype=np.int32) for _ in range(3))
    _check(ctx, _lib.ddnm_get_constraints(ctx, var.ctypes.data, lo.ctypes.data, hi.ctypes.data))
    return var, lo, hi


def ddnm_set_test_matrix(ctx, Cmat):
    Cm = _f64(Cmat)
    _check(ctx, _lib.ddnm_set_test_matrix(ctx, Cm.ctypes.data))


def ddnm_set_options(ctx, tol=1e-4, max_iter=15, armijo_c1=1e-4, beta=0.5, max_backtracks=20, step_tol=0.0):
    o = ddnm_options(tol, max_iter, armijo_c1, beta, max_backtracks, float(step_tol))
    _check(ctx, _lib.ddnm_set_options(ctx, C.byref(o)))


def ddnm_load_decoders(ctx, sub, kind, spec: dict):
    """spec: the decoder dict of ``inputs.decoder`` (N, w, n, act, W1, b1, cols, vals, scale, offset)."""
    W1, b1, vals = _f64(spec["W1"]), _f64(spec["b1"]), _f64(spec["vals"])
    cols = _i32(spec["cols"])
    sc, off = _f64(spec["scale"]), _f64(spec["offset"])
    d = ddnm_decoder(spec["N"], spec["w"], spec["n"], DDNM_ACT[spec.get("act", "swish")], cols.shape[1],
                     W1.ctypes.data_as(_dp), b1.ctypes.data_as(_dp), cols.ctypes.data_as(_ip),
                     vals.ctypes.data_as(_dp), sc.ctypes.data_as(_dp), off.ctypes.data_as(_dp))
    _check(ctx, _lib.ddnm_load_decoders(ctx, sub, kind, C.byref(d)))


def _mem_kind(*arrays):
    kinds = {isinstance(a, np.ndarray) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise TypeError("mix of host (numpy) and device (torch) arrays")
    return DDNM_MEM_HOST if (not kinds or kinds == {True}) else DDNM_MEM_DEVICE


def _stream(kind):
    if kind != DDNM_MEM_DEVICE:
        return None
    import torch
    return torch.cuda.current_stream().cuda_stream


def ddnm_solve_batch(ctx, B, mu, x0, lam0, x_out, lam_out, state_out, stats):
    """Raw call: arrays are numpy (host) or torch CUDA tensors (device); stats is a numpy
    STATS_DTYPE array (host) or a torch uint8 tensor of B*32 bytes (device)."""
    kind = _mem_kind(mu, x0, lam0, x_out, lam_out, state_out, stats)
    _check(ctx, _lib.ddnm_solve_batch(ctx, B, _ptr(mu), _ptr(x0), _ptr(lam0), _ptr(x_out), _ptr(lam_out),
                                      _ptr(state_out), _ptr(stats), kind, _stream(kind)))


def ddnm_residual(ctx, B, mu, x, lam, F_out, r_hr_out, r_full_out):
    kind = _mem_kind(mu, x, lam, F_out, r_hr_out, r_full_out)
    _check(ctx, _lib.ddnm_residual(ctx, B, _ptr(mu), _ptr(x), _ptr(lam), _ptr(F_out), _ptr(r_hr_out),
                                   _ptr(r_full_out), kind, _stream(kind)))


def ddnm_reconstruct(ctx, B, x, state_out):
    """g(xh) of B latent vectors into state_out (B x N_x): numpy host arrays or torch CUDA tensors."""
    kind = _mem_kind(x, state_out)
    _check(ctx, _lib.ddnm_reconstruct(ctx, int(B), _ptr(x), _ptr(state_out), kind, _stream(kind)))


def ddnm_linearize(ctx, B, mu, x, lam, H_out, D_out, Atil_out):
    kind = _mem_kind(mu, x, lam, H_out, D_out, Atil_out)
    _check(ctx, _lib.ddnm_linearize(ctx, B, _ptr(mu), _ptr(x), _ptr(lam), _ptr(H_out), _ptr(D_out),
                                    _ptr(Atil_out), kind, _stream(kind)))


def ddnm_residual_noalloc(ctx, B, mu, x, lam, F_out):
    """F at (x, lam) with no device allocation; all arrays are torch CUDA tensors (device memory),
    queued on the current torch stream.  For callers that cannot allocate device memory; the
    tables must already be on the device (one allocating call on ctx first).  Calls that overlap
    on the GPU race on the library's shared static scratch.

    The C call dereferences raw pointers whose sizes it cannot see, so the tensors are checked here:
    float64, contiguous, on one CUDA device, with shapes (B, 2), (B, n_D), (B, n_C) and (B, n_D + n_C)."""
    sz = ddnm_get_sizes(ctx)
    want = {"mu": (mu, (B, 2)), "x": (x, (B, sz.n_D)), "F_out": (F_out, (B, sz.n_D + sz.n_C))}
    if lam is not None:
        want["lam"] = (lam, (B, sz.n_C))
    devs = set()
    for name, (t, shape) in want.items():
        if isinstance(t, np.ndarray) or not hasattr(t, "is_cuda") or not t.is_cuda:
            raise TypeError(f"ddnm_residual_noalloc: {name} must be a torch CUDA tensor (device memory)")
        import torch
        if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != shape:
            raise ValueError(f"ddnm_residual_noalloc: {name} must be a contiguous float64 tensor of shape {shape}, "
                             f"got {t.dtype} {tuple(t.shape)}{'' if t.is_contiguous() else ' (strided)'}")
        devs.add(t.device)
    if len(devs) != 1:
        raise ValueError(f"ddnm_residual_noalloc: tensors on several devices {sorted(map(str, devs))}")
    _check(ctx, _lib.ddnm_residual_noalloc(ctx, B, _ptr(mu), _ptr(x), _ptr(lam), _ptr(F_out),
                                           _stream(DDNM_MEM_DEVICE)))


def ddnm_load_encoder(ctx, sub, kind, spec: dict):
    """spec: the encoder dict of ``inputs.encoder`` (N, w, n, cols (w x Kt), vals, b1, W2)."""
    cols, vals = _i32(spec["cols"]), _f64(spec["vals"])
    b1, W2 = _f64(spec["b1"]), _f64(spec["W2"])
    e = ddnm_encoder(spec["N"], spec["w"], spec["n"], cols.shape[1], cols.ctypes.data_as(_ip), vals.ctypes.data_as(_dp),
                     b1.ctypes.data_as(_dp), W2.ctypes.data_as(_dp))
    _check(ctx, _lib.ddnm_load_encoder(ctx, sub, kind, C.byref(e)))


def ddnm_ae_train(ctx, X, epochs, batch, lr, order=None):
    """Train every subdomain's autoencoders on the snapshots X (n_snap x N_x; numpy host or torch CUDA
    tensor); returns the epoch losses (epochs x 2 n_sub)."""
    kind = _mem_kind(X)
    if kind == DDNM_MEM_HOST:
        X = _f64(X)
    n_snap = int(X.shape[0])
    o = None if order is None else _i32(order)
    losses = np.zeros((max(epochs, 1), 2 * ddnm_get_sizes(ctx).n_sub))
    _check(ctx, _lib.ddnm_ae_train(ctx, n_snap, _ptr(X), int(epochs), int(batch), float(lr),
                                   None if o is None else o.ctypes.data, losses.ctypes.data, kind, _stream(kind)))
    return losses[:epochs]


def ddnm_ae_layout(ctx, sub, kind):
    off = np.zeros(7, dtype=np.int64)
    _check(ctx, _lib.ddnm_ae_layout(ctx, sub, kind, off.ctypes.data))
    return off


def ddnm_ae_loss_grad(ctx, sub, kind, Xt):
    """(loss, flat FP32 gradient, layout offsets) of one batch of normalised inputs Xt (nb x N)."""
    Xt = np.ascontiguousarray(np.asarray(Xt, dtype=np.float32))
    loss = C.c_double()
    _check(ctx, _lib.ddnm_ae_loss_grad(ctx, sub, kind, Xt.shape[0], Xt.ctypes.data, None, C.byref(loss)))
    off = ddnm_ae_layout(ctx, sub, kind)
    g = np.zeros(int(off[6]), dtype=np.float32)
    _check(ctx, _lib.ddnm_ae_loss_grad(ctx, sub, kind, Xt.shape[0], Xt.ctypes.data, g.ctypes.data, C.byref(loss)))
    return loss.value, g, off


def ddnm_get_decoder(ctx, sub, kind, like: dict):
    """The context's current decoder (sub, kind) as a decoder dict shaped like ``like`` (same N, w, n, mask)."""
    W1, b1 = np.zeros_like(_f64(like["W1"])), np.zeros(like["w"])
    vals = np.zeros(np.asarray(like["cols"]).shape)
    sc, off = np.zeros(like["N"]), np.zeros(like["N"])
    _check(ctx, _lib.ddnm_get_decoder(ctx, sub, kind, W1.ctypes.data, b1.ctypes.data, vals.ctypes.data, sc.ctypes.data,
                                      off.ctypes.data))
    return dict(like, W1=W1, b1=b1, vals=vals, scale=sc, offset=off)


def ddnm_fom_solve(ctx, mu, x0=None, x_out=None, max_newton=20, max_krylov=400):
    """Batched FOM solve (Newton, preconditioned BiCGSTAB) on ctx's grid.  mu (B x 2) numpy -> returns
    (x (B x N_x), stats) in host memory; or torch CUDA tensors mu, x0, x_out (device memory, current
    stream), returning (x_out, stats)."""
    kind = _mem_kind(mu, x0, x_out)
    B = int(mu.shape[0])
    Nx = ddnm_get_sizes(ctx).N_x
    if kind == DDNM_MEM_HOST:
        mu = _f64(mu).reshape(B, 2)
        x0 = None if x0 is None else _f64(x0).reshape(B, Nx)
        x_out = np.zeros((B, Nx)) if x_out is None else x_out
    st = np.zeros(B, dtype=FOM_STATS_DTYPE)
    _check(ctx, _lib.ddnm_fom_solve(ctx, B, _ptr(mu), _ptr(x0), _ptr(x_out), st.ctypes.data, int(max_newton),
                                    int(max_krylov), kind, _stream(kind)))
    return x_out, st


def ddnm_fom_residual(ctx, mu, x, r_out=None):
    """FOM residual r(x; mu) of B full states: numpy (returns r) or torch CUDA tensors (fills r_out)."""
    kind = _mem_kind(mu, x, r_out)
    B = int(mu.shape[0])
    if kind == DDNM_MEM_HOST:
        mu, x = _f64(mu).reshape(B, 2), _f64(x).reshape(B, -1)
        r_out = np.zeros_like(x) if r_out is None else r_out
    _check(ctx, _lib.ddnm_fom_residual(ctx, B, _ptr(mu), _ptr(x), _ptr(r_out), kind, _stream(kind)))
    return r_out


def ddnm_set_hr_projection(ctx, sub, proj):
    """Gappy-POD projector (Z_i Phi_i^r)^+ (nr x N_B numpy array) of subdomain sub; None returns to collocation."""
    if proj is None:
        _check(ctx, _lib.ddnm_set_hr_projection(ctx, int(sub), 0, None))
        return
    p = _f64(proj)
    _check(ctx, _lib.ddnm_set_hr_projection(ctx, int(sub), int(p.shape[0]), p.ctypes.data))


def ddnm_hr_select(ctx, snaps, nr, n_samples):
    """Gappy-POD rows and projectors from residual snapshots (n_snap x N_x numpy): returns (rows per subdomain,
    projectors per subdomain (nr_i x n_samples_i))."""
    S = _f64(snaps)
    nr, ns = _i32(nr), _i32(n_samples)
    rows = np.zeros(int(ns.sum()), dtype=np.int32)
    proj = np.zeros(int((nr.astype(np.int64) * ns).sum()))
    _check(ctx, _lib.ddnm_hr_select(ctx, S.shape[0], S.ctypes.data, nr.ctypes.data, ns.ctypes.data, rows.ctypes.data,
                                    proj.ctypes.data))
    out_r, out_p, r0, p0 = [], [], 0, 0
    for a, b in zip(nr, ns):
        out_r.append(rows[r0:r0 + b].copy())
        out_p.append(proj[p0:p0 + a * b].reshape(a, b).copy())
        r0 += b
        p0 += a * b
    return out_r, out_p


def ddnm_get_ports(ctx, n_tilde):
    """Ports under n~: (list of (subdomains, N_j^p, n_j^p), n_gamma per subdomain)."""
    n = C.c_int()
    n_sub = ddnm_get_sizes(ctx).n_sub
    ng = np.zeros(n_sub, dtype=np.int32)
    _check(ctx, _lib.ddnm_get_ports(ctx, int(n_tilde), 0, C.byref(n), None, None, None, ng.ctypes.data))
    m = n.value
    subs = np.zeros(4 * m, dtype=np.int32)
    pN, pn = np.zeros(m, dtype=np.int32), np.zeros(m, dtype=np.int32)
    _check(ctx, _lib.ddnm_get_ports(ctx, int(n_tilde), m, C.byref(n), subs.ctypes.data, pN.ctypes.data,
                                    pn.ctypes.data, ng.ctypes.data))
    return [(tuple(int(v) for v in subs[4 * j:4 * j + 4] if v >= 0), int(pN[j]), int(pn[j])) for j in range(m)], ng


def ddnm_set_srpc(ctx, n_tilde):
    _check(ctx, _lib.ddnm_set_srpc(ctx, int(n_tilde)))


def ddnm_load_port_decoder(ctx, port, spec: dict):
    """spec: a decoder dict (N = N_j^p rows in the port's variable order, n = n_j^p)."""
    W1, b1 = _f64(spec["W1"]), _f64(spec["b1"])
    cols, vals = _i32(spec["cols"]), _f64(spec["vals"])
    sc, off = _f64(spec["scale"]), _f64(spec["offset"])
    d = ddnm_decoder(spec["N"], spec["w"], spec["n"], DDNM_ACT[spec.get("act", "swish")], cols.shape[1],
                     W1.ctypes.data_as(_dp), b1.ctypes.data_as(_dp), cols.ctypes.data_as(_ip),
                     vals.ctypes.data_as(_dp), sc.ctypes.data_as(_dp), off.ctypes.data_as(_dp))
    _check(ctx, _lib.ddnm_load_port_decoder(ctx, int(port), C.byref(d)))


def ddnm_get_port_matrix(ctx, sub, n_gamma):
    out = np.zeros((ddnm_get_sizes(ctx).n_C, int(n_gamma)))
    _check(ctx, _lib.ddnm_get_port_matrix(ctx, int(sub), out.ctypes.data))
    return out


def mlp_param_count(n_in, H, n_out):
    return H * n_in + H + H * H + H + n_out * H + n_out


def ddnm_ws_init(ctx, hidden, params):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    _check(ctx, _lib.ddnm_ws_init(ctx, hidden, p.ctypes.data))


def ddnm_ws_set_norm(ctx, mu_c, mu_s, out_mean, out_std):
    a = [_f64(v) for v in (mu_c, mu_s, out_mean, out_std)]
    _check(ctx, _lib.ddnm_ws_set_norm(ctx, *[v.ctypes.data for v in a]))


def ddnm_ws_loss_grad(ctx, z, t, n_params):
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
    g = np.zeros(n_params, dtype=np.float32)
    loss = C.c_double()
    _check(ctx, _lib.ddnm_ws_loss_grad(ctx, z.shape[0], z.ctypes.data, t.ctypes.data, g.ctypes.data, C.byref(loss)))
    return loss.value, g


def ddnm_ws_train(ctx, mu, x_star, epochs, batch, lr, order=None):
    mu, x_star = _f64(mu), _f64(x_star)
    o = None if order is None else _i32(order)
    losses = np.zeros(max(epochs, 1))
    _check(ctx, _lib.ddnm_ws_train(ctx, mu.shape[0], mu.ctypes.data, x_star.ctypes.data, epochs, batch, lr,
                                   None if o is None else o.ctypes.data, losses.ctypes.data))
    return losses[:epochs]


def ddnm_ws_predict(ctx, mu, n_out):
    mu = _f64(mu).reshape(-1, 2)
    x0 = np.zeros((mu.shape[0], n_out))
    _check(ctx, _lib.ddnm_ws_predict(ctx, mu.shape[0], mu.ctypes.data, x0.ctypes.data, DDNM_MEM_HOST, None))
    return x0


def ddnm_ws_get_params(ctx, n_params, n_out):
    p = np.zeros(n_params, dtype=np.float32)
    nrm = np.zeros(4 + 2 * n_out)
    _check(ctx, _lib.ddnm_ws_get_params(ctx, p.ctypes.data, nrm.ctypes.data))
    return p, nrm


def ddnm_ws_enable(ctx, on=True):
    _check(ctx, _lib.ddnm_ws_enable(ctx, int(bool(on))))


def ddnm_ws_save(ctx, path):
    _check(ctx, _lib.ddnm_ws_save(ctx, os.fsencode(path)))


def ddnm_ws_load(ctx, path):
    _check(ctx, _lib.ddnm_ws_load(ctx, os.fsencode(path)))


def ddnm_measure_peaks(ctx):
    """(FP32, FP64) FMA throughput of ctx's device in TFLOP/s, measured."""
    a, b = C.c_double(), C.c_double()
    _check(ctx, _lib.ddnm_measure_peaks(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def ddnm_timing_enable(ctx, on=True):
    _check(ctx, _lib.ddnm_timing_enable(ctx, int(bool(on))))


def ddnm_get_timing(ctx) -> dict:
    t = ddnm_timing()
    _check(ctx, _lib.ddnm_get_timing(ctx, C.byref(t)))
    return {k: getattr(t, k) for k, _ in ddnm_timing._fields_}


def ddnm_get_work(ctx) -> dict:
    w = ddnm_work()
    _check(ctx, _lib.ddnm_get_work(ctx, C.byref(w)))
    return {k: getattr(w, k) for k, _ in ddnm_work._fields_}


def ddnm_set_tune(ctx, graph=1, chains=1, con_split=512, eval_persist=0, d_gemm=-1, eval_groups=1, atil=-1):
    t = ddnm_tune(int(graph), int(chains), int(con_split), int(eval_persist), int(d_gemm), int(eval_groups),
                  int(atil))
    _check(ctx, _lib.ddnm_set_tune(ctx, C.byref(t)))


def ddnm_get_tune(ctx) -> dict:
    t = ddnm_tune()
    _check(ctx, _lib.ddnm_get_tune(ctx, C.byref(t)))
    return {k: getattr(t, k) for k, _ in ddnm_tune._fields_}


def ddnm_autotune(ctx, mu, max_iter=0, reps=3, stream=None):
    """Autotune the launch plan on host mu (B x 2); returns (plan dict, median ms per solve)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    t = ddnm_tune()
    ms = C.c_float()
    _check(ctx, _lib.ddnm_autotune(ctx, int(mu.shape[0]), mu.ctypes.data, DDNM_MEM_HOST, stream, int(max_iter),
                                   int(reps), C.byref(t), C.byref(ms)))
    return {k: getattr(t, k) for k, _ in ddnm_tune._fields_}, float(ms.value)


# ------------------------------------------------------------------ convenience wrapper

class Solver:
    """One library context for a workload (``inputs.Workload``-like object)."""

    def __init__(self, wl, precision=None, device=0, n_gamma=None, n_c=None):
        """n_gamma / n_c override the workload's interface latent sizes and constraint count (the SRPC
        formulation takes them from the ports: ddnm_get_ports)."""
        prec = precision if precision is not None else (DDNM_MIXED if wl.mixed else DDNM_FP64)
        self.wl = wl
        hr = getattr(wl, "hr_override", None)
        if hr is None:
            import inputs   # seeded generator (not method code)
            hr = inputs.hr_sets(wl)
        self.hr = hr
        self.ctx = ddnm_setup(wl.nx, wl.ny, wl.xb, wl.yb, wl.n_omega, wl.n_gamma if n_gamma is None else n_gamma,
                              [len(h) for h in hr], np.concatenate(hr), wl.n_c() if n_c is None else n_c, prec,
                              wl.nu, device=device)
        self.sizes = ddnm_get_sizes(self.ctx)
        self.subs = [ddnm_get_subdomain(self.ctx, i) for i in range(self.sizes.n_sub)]

    def close(self):
        if self.ctx:
            ddnm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, dec_o, dec_g, Cmat):
        for i, (a, b) in enumerate(zip(dec_o, dec_g)):
            ddnm_load_decoders(self.ctx, i, DDNM_DECODER_INTERIOR, a)
            ddnm_load_decoders(self.ctx, i, DDNM_DECODER_INTERFACE, b)
        ddnm_set_test_matrix(self.ctx, Cmat)

    def load_srpc(self, n_tilde, dec_o, port_decs):
        """SRPC formulation: interior decoders per subdomain and one decoder per port (ddnm_get_ports order)."""
        ddnm_set_srpc(self.ctx, n_tilde)
        for i, a in enumerate(dec_o):
            ddnm_load_decoders(self.ctx, i, DDNM_DECODER_INTERIOR, a)
        for j, d in enumerate(port_decs):
            ddnm_load_port_decoder(self.ctx, j, d)

    def options(self, **kw):
        ddnm_set_options(self.ctx, **kw)

    def solve(self, mu, x0=None, lam0=None, state=False):
        """Host (numpy) solve: returns (x, lam, stats[, state])."""
        mu = _f64(mu).reshape(-1, 2)
        B = mu.shape[0]
        s = self.sizes
        x = np.zeros((B, s.n_D))
        lam = np.zeros((B, s.n_C))
        st = np.zeros(B, dtype=STATS_DTYPE)
        stt = np.zeros((B, s.N_x)) if state else None
        ddnm_solve_batch(self.ctx, B, mu, None if x0 is None else _f64(x0), None if lam0 is None else _f64(lam0),
                         x, lam, stt, st)
        return (x, lam, st, stt) if state else (x, lam, st)

    def residual(self, mu, x, lam=None, full=False):
        mu = _f64(mu).reshape(-1, 2)
        B = mu.shape[0]
        s = self.sizes
        F = np.zeros((B, s.n_D + s.n_C))
        r = np.zeros((B, s.sum_hr))
        rf = np.zeros((B, s.N_x)) if full else None
        ddnm_residual(self.ctx, B, mu, _f64(x).reshape(B, -1), None if lam is None else _f64(lam).reshape(B, -1),
                      F, r, rf)
        return (F, r, rf) if full else (F, r)

    def linearize(self, mu, x, lam=None):
        mu = _f64(mu).reshape(-1, 2)
        B = mu.shape[0]
        s = self.sizes
        hs = sum((d["n_omega"] + d["n_gamma"]) ** 2 for d in self.subs)
        ds = sum(s.n_C * d["n_gamma"] for d in self.subs)
        H = np.zeros((B, hs))
        D = np.zeros((B, ds))
        A = np.zeros((B, s.n_C))
        ddnm_linearize(self.ctx, B, mu, _f64(x).reshape(B, -1), None if lam is None else _f64(lam).reshape(B, -1),
                       H, D, A)
        return H, D, A
