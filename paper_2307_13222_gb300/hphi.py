"""Thin ctypes binding of libhphi (include/hphi.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
computation happens in the CUDA library.  Device vectors are torch CUDA
tensors, [D] or [D][nvec] with unit column stride; the library works on the
caller's current torch stream.  There is no CPU path: without the built
library or without a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhphi.so")

HPHI_OK = 0
ERRORS = {-1: "INVAL", -2: "NOMEM", -3: "CUDA", -4: "NOTCONV", -5: "NUMERIC", -6: "DEVICE_CHECK", -7: "TIMEOUT"}
MODELS = {"SPIN_HALF": 0, "SPIN_HALF_GC": 1, "HUBBARD": 2}
KINDS = {"EXCHANGE": 0, "XXZ": 1, "HOP": 2, "HUBBARD_U": 3, "DENS_DENS": 4}
F64, F32, C128, C64 = 0, 1, 2, 3


class HphiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hphi error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Term(C.Structure):
    _fields_ = [("kind", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("spin", C.c_int32),
                ("v0", C.c_double), ("v1", C.c_double)]


class _LanczosOpts(C.Structure):
    _fields_ = [("max_steps", C.c_int), ("tol", C.c_double), ("dtype", C.c_int), ("check_every", C.c_int),
                ("reorth", C.c_int)]


class _LanczosResult(C.Structure):
    _fields_ = [("e0", C.c_double), ("resid_est", C.c_double), ("resid", C.c_double), ("steps", C.c_int),
                ("breakdown", C.c_int), ("e0_rq", C.c_double)]


class _KrylovOpts(C.Structure):
    _fields_ = [("max_steps", C.c_int), ("tol", C.c_double), ("dtype", C.c_int), ("check_every", C.c_int)]


class _KrylovResult(C.Structure):
    _fields_ = [("steps", C.c_int), ("converged", C.c_int), ("max_resid", C.c_double)]


class _ServerOpts(C.Structure):
    _fields_ = [("mem_budget", C.c_double), ("max_active", C.c_int), ("chunk", C.c_int),
                ("small_max_dim", C.c_int64), ("grid_workers", C.c_int), ("grid_dtype", C.c_int)]


class _Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("ham", C.c_void_p), ("seed", C.c_uint64), ("max_steps", C.c_int),
                ("tol", C.c_double), ("q", C.c_double), ("eta", C.c_double), ("nz", C.c_int),
                ("omega", C.c_void_p)]


class _Reply(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("steps", C.c_int), ("krylov_steps", C.c_int),
                ("lane", C.c_int), ("e0", C.c_double), ("max_resid", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double)]


class _ServerStats(C.Structure):
    _fields_ = [("block_launches", C.c_int64), ("block_done", C.c_int64), ("grid_done", C.c_int64),
                ("block_running", C.c_int), ("grid_running", C.c_int), ("queued", C.c_int),
                ("arena_used", C.c_double), ("arena_peak", C.c_double)]


_lib = None
vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
_SIGS = {
    "hphi_ctx_create": (i32, [i32, vp, C.POINTER(vp)]),
    "hphi_ctx_set_stream": (i32, [vp, vp]),
    "hphi_ctx_destroy": (None, [vp]),
    "hphi_last_error": (C.c_char_p, [vp]),
    "hphi_last_kernel": (C.c_char_p, [vp]),
    "hphi_ctx_sm_count": (i32, [vp]),
    "hphi_ctx_profile": (i32, [vp, i32]),
    "hphi_ctx_profile_read": (i32, [vp, i32, C.POINTER(i64), C.POINTER(dbl)]),
    "hphi_build_basis": (i32, [vp, i32, i32, i32, i32, C.POINTER(vp)]),
    "hphi_basis_destroy": (None, [vp]),
    "hphi_basis_dim": (i64, [vp]),
    "hphi_basis_table_sizes": (i32, [vp, i32, C.POINTER(i64), C.POINTER(i64)]),
    "hphi_basis_export": (i32, [vp, vp, i32, vp, vp]),
    "hphi_basis_states": (i32, [vp, vp, i64, i64, vp, vp]),
    "hphi_basis_rank": (i32, [vp, vp, vp, vp, i64, vp]),
    "hphi_build_hamiltonian": (i32, [vp, vp, vp, i32, C.POINTER(vp)]),
    "hphi_ham_destroy": (None, [vp]),
    "hphi_ham_dim": (i64, [vp]),
    "hphi_ham_set_tuning": (i32, [vp, i32, i32]),
    "hphi_ham_get_tuning": (i32, [vp, i32, C.POINTER(i32)]),
    "hphi_ham_autotune": (i32, [vp, vp, i32, i32, i32, C.POINTER(dbl), C.POINTER(i32)]),
    "hphi_apply_H": (i32, [vp, vp, i32, i32, vp, i64, vp, i64, dbl, dbl]),
    "hphi_apply_H_host": (i32, [vp, vp, i32, i32, i64, vp, vp, dbl]),
    "hphi_dump_pattern": (i32, [vp, vp, i64, i64, vp, vp, vp, vp, C.POINTER(i64)]),
    "hphi_dump_pattern_merged": (i32, [vp, vp, i64, i64, vp, vp, vp, C.POINTER(i64)]),
    "hphi_dot": (i32, [vp, i32, i64, i32, vp, i64, vp, i64, vp]),
    "hphi_nrm2": (i32, [vp, i32, i64, i32, vp, i64, vp]),
    "hphi_axpy": (i32, [vp, i32, i64, i32, vp, vp, i64, vp, i64]),
    "hphi_scal": (i32, [vp, i32, i64, i32, vp, vp, i64]),
    "hphi_random_vector": (i32, [vp, i32, i64, i32, C.c_uint64, vp, i64]),
    "hphi_lanczos": (i32, [vp, vp, C.POINTER(_LanczosOpts), vp, vp, vp, vp, C.POINTER(_LanczosResult)]),
    "hphi_tpq_step": (i32, [vp, vp, i32, i32, vp, i64, dbl, i32, vp, vp, vp, vp]),
    "hphi_mtpq_step": (i32, [vp, vp, i32, i32, vp, i64, dbl, i32, i32, vp, vp, vp, vp, vp]),
    "hphi_tpq_bootstrap": (i32, [i32, i32, vp, vp, vp, vp, i32, i32, vp, C.c_uint64, vp, vp, vp, vp]),
    "hphi_lobpcg": (i32, [vp, vp, i32, vp, i32, dbl, vp, vp, C.POINTER(i32)]),
    "hphi_tridiag_eigen": (i32, [i32, vp, vp, vp, vp]),
    "hphi_dot_static": (i32, [i32, vp, i32, i64, i32, vp, i64, vp, i64, vp]),
    "hphi_apply_sz_sum": (i32, [vp, vp, i32, vp, i64, vp, i64, vp]),
    "hphi_time_step": (i32, [vp, vp, i32, i32, vp, i64, dbl, i32, vp, vp, vp, vp]),
    "hphi_lanczos_batch": (i32, [vp, i32, vp, vp, vp, C.POINTER(_LanczosOpts), vp, vp]),
    "hphi_server_create": (i32, [vp, C.POINTER(_ServerOpts), C.POINTER(vp)]),
    "hphi_server_destroy": (None, [vp]),
    "hphi_server_clock": (dbl, [vp]),
    "hphi_server_submit": (i32, [vp, C.POINTER(_Request), C.POINTER(i64)]),
    "hphi_server_step": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
    "hphi_server_result": (i32, [vp, i64, C.POINTER(_Reply), vp]),
    "hphi_server_get_stats": (i32, [vp, C.POINTER(_ServerStats)]),
    "hphi_shifted_krylov": (i32, [vp, vp, C.POINTER(_KrylovOpts), i32, vp, i64, i32, vp, vp, vp, vp, vp,
                                  C.POINTER(_KrylovResult)]),
    "hphi_szz_spectrum": (i32, [vp, vp, C.POINTER(_KrylovOpts), vp, i32, vp, i32, vp, vp, vp, vp,
                                C.POINTER(_KrylovResult)]),
}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libhphi.so (built by paper_2307_13222_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libhphi not built ({path} missing): run paper_2307_13222_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _np(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dtype_code(t) -> int:
    import torch
    m = {torch.float64: F64, torch.float32: F32, torch.complex128: C128, torch.complex64: C64}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _vec(t):
    """(pointer, nvec, ld) of a [D] or [D][nvec] CUDA tensor with unit column stride."""
    if not t.is_cuda:
        raise ValueError("libhphi takes CUDA tensors only (no CPU path)")
    if t.dim() == 1:
        if t.stride(0) != 1:
            raise ValueError("vector must be contiguous")
        return C.c_void_p(t.data_ptr()), 1, 1
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected [D] or [D][nvec] with unit column stride")
    return C.c_void_p(t.data_ptr()), t.shape[1], max(t.stride(0), t.shape[1])


class Context:
    """A library context on one CUDA device, following torch's current stream."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: libhphi has no CPU fallback")
        self.lib = load_library()
        self.device = device
        h = vp()
        torch.cuda.set_device(device)
        torch.cuda.init()
        st = self.lib.hphi_ctx_create(device, C.c_void_p(torch.cuda.current_stream(device).cuda_stream), C.byref(h))
        if st != HPHI_OK:
            raise HphiError(st, "hphi_ctx_create failed")
        self.h = h

    def _sync_stream(self):
        import torch
        self.lib.hphi_ctx_set_stream(self.h, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def check(self, st: int):
        if st != HPHI_OK:
            raise HphiError(st, (self.lib.hphi_last_error(self.h) or b"").decode())

    @property
    def sm_count(self) -> int:
        return int(self.lib.hphi_ctx_sm_count(self.h))

    def last_kernel(self) -> str:
        """Name and selecting template arguments of the last H*x kernel launched."""
        return (self.lib.hphi_last_kernel(self.h) or b"").decode()

    def profile(self, enable: bool = True):
        """Record CUDA-event times around every kernel launch of this context."""
        self.check(self.lib.hphi_ctx_profile(self.h, 1 if enable else 0))

    def profile_read(self, kind: int = 0):
        """(launches, total_ms) of kernel class kind (0: H*x, 1: vector kernels) since the last read."""
        n, t = i64(0), dbl(0.0)
        self.check(self.lib.hphi_ctx_profile_read(self.h, kind, C.byref(n), C.byref(t)))
        return int(n.value), float(t.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.hphi_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Basis:
    def __init__(self, ctx: Context, model: str, n_sites: int, n_up: int = 0, n_dn: int = 0):
        self.ctx = ctx
        ctx._sync_stream()
        h = vp()
        ctx.check(ctx.lib.hphi_build_basis(ctx.h, MODELS[model], n_sites, n_up, n_dn, C.byref(h)))
        self.h = h
        self.model, self.n_sites, self.n_up, self.n_dn = model, n_sites, n_up, n_dn
        self.dim = int(ctx.lib.hphi_basis_dim(h))

    def export_tables(self, species: int = 0):
        na, nb = i64(0), i64(0)
        self.ctx.check(self.ctx.lib.hphi_basis_table_sizes(self.h, species, C.byref(na), C.byref(nb)))
        ja = np.zeros(na.value, np.uint32)
        jb = np.zeros(nb.value, np.uint64)
        self.ctx._sync_stream()
        self.ctx.check(self.ctx.lib.hphi_basis_export(self.ctx.h, self.h, species, _np(ja), _np(jb)))
        return ja, jb

    def states(self, row0: int, n: int):
        import torch
        su = torch.empty(n, dtype=torch.int64, device=f"cuda:{self.ctx.device}")
        sd = torch.empty(n, dtype=torch.int64, device=f"cuda:{self.ctx.device}")
        self.ctx._sync_stream()
        self.ctx.check(self.ctx.lib.hphi_basis_states(self.ctx.h, self.h, row0, n, C.c_void_p(su.data_ptr()),
                                                      C.c_void_p(sd.data_ptr())))
        return su, sd

    def rank(self, su, sd=None):
        import torch
        n = su.numel()
        out = torch.empty(n, dtype=torch.int64, device=su.device)
        self.ctx._sync_stream()
        self.ctx.check(self.ctx.lib.hphi_basis_rank(self.ctx.h, self.h, C.c_void_p(su.data_ptr()),
                                                    C.c_void_p(sd.data_ptr()) if sd is not None else None, n,
                                                    C.c_void_p(out.data_ptr())))
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hphi_basis_destroy(self.h)
            self.h = None


class Hamiltonian:
    def __init__(self, ctx: Context, basis: Basis, terms):
        self.ctx, self.basis = ctx, basis
        arr = (_Term * max(len(terms), 1))()
        for k, (kind, i, j, spin, v0, v1) in enumerate(terms):
            arr[k] = _Term(KINDS[kind], i, j, spin, v0, v1)
        ctx._sync_stream()
        h = vp()
        ctx.check(ctx.lib.hphi_build_hamiltonian(ctx.h, basis.h, C.cast(arr, vp), len(terms), C.byref(h)))
        self.h = h
        self.dim = int(ctx.lib.hphi_ham_dim(h))

    TUNE = {"inner_bits": 0, "split": 1, "l2_hints": 2, "variant": 3, "coop": 4, "staged_lists": 5}

    def set_tuning(self, **knobs):
        """Launch knobs of the H*x kernel: inner_bits, split, l2_hints, variant, coop, staged_lists."""
        for k, v in knobs.items():
            self.ctx.check(self.ctx.lib.hphi_ham_set_tuning(self.h, self.TUNE[k], int(v)))

    def autotune(self, dtype, nvec: int = 1, reps: int = 3):
        """Time every valid launch setting for nvec columns of dtype (a torch
        dtype) and keep the fastest.  Returns (ms per launch, settings tried)."""
        import torch
        code = {torch.float64: F64, torch.float32: F32, torch.complex128: C128, torch.complex64: C64}[dtype]
        ms, n = dbl(0.0), i32(0)
        self.ctx._sync_stream()
        self.ctx.check(self.ctx.lib.hphi_ham_autotune(self.ctx.h, self.h, code, int(nvec), int(reps), C.byref(ms),
                                                      C.byref(n)))
        return ms.value, n.value

    def get_tuning(self):
        out = {}
        for k, code in self.TUNE.items():
            v = C.c_int(0)
            self.ctx.check(self.ctx.lib.hphi_ham_get_tuning(self.h, code, C.byref(v)))
            out[k] = v.value
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hphi_ham_destroy(self.h)
            self.h = None


# ---- entry points with the C names -------------------------------------------------

def hphi_apply_H(ham: Hamiltonian, x, y, alpha: float = 1.0, beta: float = 0.0):
    """y <- alpha H x + beta y (asynchronous on the current stream)."""
    ctx = ham.ctx
    if x.dtype != y.dtype or x.shape != y.shape:
        raise ValueError("x and y must have the same dtype and shape")
    px, nv, ldx = _vec(x)
    py, _, ldy = _vec(y)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_apply_H(ctx.h, ham.h, _dtype_code(x), nv, px, ldx, py, ldy, float(alpha), float(beta)))
    return y


def hphi_apply_H_host(ham: Hamiltonian, x_host, y_host, alpha: float = 1.0):
    """y_b <- alpha H x_b for a batch of HOST vectors: x_host, y_host are CPU
    tensors of shape [nbatch, D] or [nbatch, D, nvec], contiguous, same dtype
    (pinned memory gives full copy speed).  Copies and products overlap inside
    the library; returns when y_host is complete."""
    import torch
    ctx = ham.ctx
    if x_host.device.type != "cpu" or y_host.device.type != "cpu":
        raise ValueError("x_host and y_host must be host (CPU) tensors")
    if x_host.dtype != y_host.dtype or x_host.shape != y_host.shape:
        raise ValueError("x_host and y_host must have the same dtype and shape")
    if x_host.dim() not in (2, 3) or x_host.shape[1] != ham.basis.dim:
        raise ValueError("expected shape [nbatch, D] or [nbatch, D, nvec] with D = %d" % ham.basis.dim)
    if not (x_host.is_contiguous() and y_host.is_contiguous()):
        raise ValueError("x_host and y_host must be contiguous")
    nv = 1 if x_host.dim() == 2 else int(x_host.shape[2])
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_apply_H_host(ctx.h, ham.h, _dtype_code(x_host), nv, int(x_host.shape[0]),
                                        C.c_void_p(x_host.data_ptr()), C.c_void_p(y_host.data_ptr()), float(alpha)))
    return y_host


def hphi_dot(ctx: Context, x, y) -> np.ndarray:
    px, nv, ldx = _vec(x)
    py, _, ldy = _vec(y)
    dc = _dtype_code(x)
    out = np.zeros(2 * nv if dc in (C128, C64) else nv)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_dot(ctx.h, dc, x.shape[0], nv, px, ldx, py, ldy, _np(out)))
    if dc in (C128, C64):
        return out[0::2] + 1j * out[1::2]
    return out


def hphi_dot_static(device: int, x, y) -> np.ndarray:
    """<x_q|y_q> like hphi_dot, through the entry point that allocates no device
    memory (no context needed); runs on torch's current stream of `device`."""
    import torch
    lib = load_library()
    if x.device != y.device or not x.is_cuda or x.device.index != device:
        raise ValueError(f"x and y must both be on cuda:{device}")
    if x.dtype != y.dtype or x.shape != y.shape:
        raise ValueError("x and y must have the same dtype and shape")
    px, nv, ldx = _vec(x)
    py, _, ldy = _vec(y)
    dc = _dtype_code(x)
    out = np.zeros(2 * nv if dc in (C128, C64) else nv)
    st = lib.hphi_dot_static(device, C.c_void_p(torch.cuda.current_stream(device).cuda_stream), dc, x.shape[0], nv,
                             px, ldx, py, ldy, _np(out))
    if st != HPHI_OK:
        raise HphiError(st, "hphi_dot_static failed")
    if dc in (C128, C64):
        return out[0::2] + 1j * out[1::2]
    return out


def hphi_nrm2(ctx: Context, x) -> np.ndarray:
    px, nv, ldx = _vec(x)
    out = np.zeros(nv)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_nrm2(ctx.h, _dtype_code(x), x.shape[0], nv, px, ldx, _np(out)))
    return out


def _coefs(a, nv, cplx):
    a = np.atleast_1d(np.asarray(a, dtype=np.complex128 if cplx else np.float64))
    if a.size == 1:
        a = np.repeat(a, nv)
    return np.ascontiguousarray(a.view(np.float64) if cplx else a)


def hphi_axpy(ctx: Context, a, x, y):
    px, nv, ldx = _vec(x)
    py, _, ldy = _vec(y)
    dc = _dtype_code(x)
    av = _coefs(a, nv, dc in (C128, C64))
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_axpy(ctx.h, dc, x.shape[0], nv, _np(av), px, ldx, py, ldy))
    return y


def hphi_scal(ctx: Context, a, x):
    px, nv, ldx = _vec(x)
    dc = _dtype_code(x)
    av = _coefs(a, nv, dc in (C128, C64))
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_scal(ctx.h, dc, x.shape[0], nv, _np(av), px, ldx))
    return x


def hphi_random_vector(ctx: Context, x, seed: int):
    px, nv, ldx = _vec(x)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_random_vector(ctx.h, _dtype_code(x), x.shape[0], nv, C.c_uint64(seed), px, ldx))
    return x


def hphi_lanczos(ham: Hamiltonian, v0, max_steps: int, tol: float, check_every: int = 1, gs_out=None,
                 reorth: bool = False):
    """Lanczos from v0 (F64 or F32 CUDA vector). Returns a dict; NOTCONV is reported, not raised."""
    ctx = ham.ctx
    dc = _dtype_code(v0)
    opts = _LanczosOpts(max_steps, tol, dc, check_every, 1 if reorth else 0)
    res = _LanczosResult()
    alpha = np.zeros(max_steps)
    beta = np.zeros(max_steps + 1)
    ctx._sync_stream()
    st = ctx.lib.hphi_lanczos(ctx.h, ham.h, C.byref(opts), C.c_void_p(v0.data_ptr()),
                              C.c_void_p(gs_out.data_ptr()) if gs_out is not None else None, _np(alpha), _np(beta),
                              C.byref(res))
    if st not in (HPHI_OK, -4):
        ctx.check(st)
    m = res.steps
    return dict(converged=st == HPHI_OK, status=st, e0=res.e0, resid_est=res.resid_est, resid=res.resid, steps=m,
                breakdown=bool(res.breakdown), alpha=alpha[:m], beta=beta[1:m + 1], e0_rq=res.e0_rq)


def hphi_lanczos_batch(hams, v0s, max_steps: int, tol: float, check_every: int = 8, gs_outs=None):
    """Ground states of many small problems at once (FP64 CUDA start vectors).
    Returns one dict per problem (as hphi_lanczos, plus its status)."""
    n = len(hams)
    if n == 0:
        return []
    ctx = hams[0].ctx
    if len(v0s) != n or (gs_outs is not None and len(gs_outs) != n):
        raise ValueError("one start vector (and ground-state buffer) per problem")
    for h, v in zip(hams, v0s):
        if not v.is_cuda or v.dtype.itemsize != 8 or v.is_complex() or v.dim() != 1 or v.stride(0) != 1:
            raise ValueError("start vectors must be contiguous FP64 CUDA vectors")
        if v.numel() != int(ctx.lib.hphi_ham_dim(h.h)):
            raise ValueError("start vector length differs from the problem's dimension")
    for h, g in zip(hams, gs_outs or []):
        if g is not None and (not g.is_cuda or g.dtype.itemsize != 8 or g.is_complex() or not g.is_contiguous()
                              or g.numel() != int(ctx.lib.hphi_ham_dim(h.h))):
            raise ValueError("ground-state buffers must be contiguous FP64 CUDA vectors of the problem's length")
    hs = (vp * n)(*[h.h for h in hams])
    vs = (vp * n)(*[C.c_void_p(v.data_ptr()) for v in v0s])
    gs = (vp * n)(*[C.c_void_p(g.data_ptr()) if g is not None else None for g in gs_outs]) if gs_outs else None
    opts = _LanczosOpts(max_steps, tol, F64, check_every, 0)
    res = (_LanczosResult * n)()
    stat = (C.c_int * n)()
    ctx._sync_stream()
    st = ctx.lib.hphi_lanczos_batch(ctx.h, n, hs, vs, gs, C.byref(opts), res, stat)
    if st != HPHI_OK and st not in list(stat):  # a call-level error, not a per-problem status
        ctx.check(st)
    return [dict(status=stat[p], converged=stat[p] == HPHI_OK, e0=res[p].e0, resid_est=res[p].resid_est,
                 resid=res[p].resid, steps=res[p].steps, breakdown=bool(res[p].breakdown)) for p in range(n)]


class Server:
    """Continuous-batching server of ground-state and spectrum requests
    (hphi_server_*).  Hamiltonians passed to submit() must outlive their
    requests; the server keeps a reference to them."""

    GROUND, SPECTRUM = 0, 1

    def __init__(self, ctx: Context, mem_budget: float, max_active: int = 0, chunk: int = 0, small_max_dim: int = 0,
                 grid_workers: int = 0, grid_dtype: str = "f64"):
        self.ctx = ctx
        if grid_dtype not in ("f64", "f32"):
            raise ValueError("grid_dtype is 'f64' or 'f32'")
        o = _ServerOpts(float(mem_budget), max_active, chunk, small_max_dim, grid_workers,
                        F32 if grid_dtype == "f32" else F64)
        h = vp()
        ctx._sync_stream()
        ctx.check(ctx.lib.hphi_server_create(ctx.h, C.byref(o), C.byref(h)))
        self.h = h
        self._keep = {}

    def clock(self) -> float:
        return float(self.ctx.lib.hphi_server_clock(self.h))

    def submit(self, ham: Hamiltonian, kind: int = 0, seed: int = 1, max_steps: int = 500, tol: float = 1e-10,
               q: float = 0.0, eta: float = 0.05, omega=None) -> int:
        om = np.ascontiguousarray(np.asarray(omega if omega is not None else [], dtype=np.float64))
        r = _Request(kind, ham.h, seed, max_steps, tol, q, eta, om.size, _np(om) if om.size else None)
        rid = i64(0)
        self.ctx._sync_stream()
        self.ctx.check(self.ctx.lib.hphi_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (ham, om.size)
        return rid.value

    def step(self):
        """One scheduling step; returns (running, queued)."""
        a, b = i32(0), i32(0)
        self.ctx.check(self.ctx.lib.hphi_server_step(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def result(self, rid: int):
        rep = _Reply()
        nz = self._keep[rid][1]
        d = np.zeros(2 * max(nz, 1))
        self.ctx.check(self.ctx.lib.hphi_server_result(self.h, rid, C.byref(rep), _np(d)))
        out = {k: getattr(rep, k) for k, _ in _Reply._fields_}
        out["done"] = bool(out["done"])
        out["D"] = (d[0::2] + 1j * d[1::2])[:nz] if nz else None
        return out

    def stats(self) -> dict:
        st = _ServerStats()
        self.ctx.check(self.ctx.lib.hphi_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def run_until_done(self, ids, max_steps: int = 1000000):
        for _ in range(max_steps):
            if all(self.result(i)["done"] for i in ids):
                return
            self.step()
            st = self.stats()
            if st["block_running"] == 0 and st["queued"] == 0:
                import time
                time.sleep(0.0005)  # only the grid lane's workers run
        raise RuntimeError("server did not finish")

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.hphi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hphi_tpq_step(ham: Hamiltonian, V, dtau: float, nmax: int, norm2: np.ndarray):
    """One cTPQ step in place on V; norm2 (float64[nvec]) is updated in place.
    Returns (e, h2, logd) per column."""
    ctx = ham.ctx
    pv, nv, ld = _vec(V)
    assert norm2.dtype == np.float64 and norm2.size == nv and norm2.flags.c_contiguous
    e, h2, logd = np.zeros(nv), np.zeros(nv), np.zeros(nv)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_tpq_step(ctx.h, ham.h, _dtype_code(V), nv, pv, ld, float(dtau), int(nmax), _np(norm2),
                                    _np(e), _np(h2), _np(logd)))
    return e, h2, logd


def hphi_time_step(ham: Hamiltonian, V, dt: float, nmax: int):
    """One real-time step in place on complex V ([D] or [D][nvec], C128/C64).
    Returns (norm2, e, h2) of the state before the step and norm2 after it."""
    ctx = ham.ctx
    pv, nv, ld = _vec(V)
    dc = _dtype_code(V)
    if dc not in (C128, C64):
        raise ValueError("real-time evolution needs complex vectors")
    n2, e, h2, n2n = np.zeros(nv), np.zeros(nv), np.zeros(nv), np.zeros(nv)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_time_step(ctx.h, ham.h, dc, nv, pv, ld, float(dt), int(nmax), _np(n2), _np(e), _np(h2),
                                     _np(n2n)))
    return n2, e, h2, n2n


def hphi_apply_sz_sum(basis: Basis, x, y, A):
    """y = sum_l A_l S^z_l x (Sec. 3.2 excitation operator).  x: real CUDA
    vector [D] (any element stride); y: complex CUDA vector [D] or real
    [D][>=2] (Re in column 0, Im in column 1) of x's precision; A: N complex
    weights (e^{i q l} for S^z(q))."""
    import torch
    ctx = basis.ctx
    if not (x.is_cuda and y.is_cuda):
        raise ValueError("libhphi takes CUDA tensors only (no CPU path)")
    if x.dim() != 1 or x.dtype not in (torch.float64, torch.float32):
        raise ValueError("x must be a real [D] vector")
    if y.is_complex():
        if y.dim() != 1 or y.stride(0) != 1:
            raise ValueError("complex y must be a contiguous [D] vector")
        yr = torch.view_as_real(y)
        ldy = 2
    else:
        if y.dim() != 2 or y.stride(1) != 1 or y.shape[1] < 2:
            raise ValueError("real y must be [D][>=2] with unit column stride")
        yr, ldy = y, y.stride(0)
    if yr.dtype != x.dtype:
        raise ValueError("x and y must have the same precision")
    a = np.asarray(A, dtype=np.complex128).reshape(-1)
    if a.size != basis.n_sites:
        raise ValueError(f"need {basis.n_sites} weights")
    ah = np.ascontiguousarray(np.stack([a.real, a.imag], axis=1).reshape(-1))
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_apply_sz_sum(ctx.h, basis.h, _dtype_code(x), C.c_void_p(x.data_ptr()), x.stride(0),
                                        C.c_void_p(yr.data_ptr()), ldy, _np(ah)))
    return y


def hphi_shifted_krylov(ham: Hamiltonian, B, z, max_steps: int, tol: float, check_every: int = 1):
    """D_c(z_j) = <b_c|(z_j - H)^{-1}|b_c> for the real CUDA columns of B ([D]
    or [D][ncol], F64 or F32) and complex shifts z.  Returns a dict with G
    [ncol][nz] complex, resid [ncol][nz], steps, converged, status, max_resid,
    alpha / beta per column (beta[0] = |b_c|).  NOTCONV is reported, not raised."""
    ctx = ham.ctx
    pv, nc, ld = _vec(B)
    dc = _dtype_code(B)
    if dc not in (F64, F32):
        raise ValueError("right-hand sides must be real (split a complex vector into its two parts)")
    zz = np.asarray(z, dtype=np.complex128).reshape(-1)
    zh = np.ascontiguousarray(np.stack([zz.real, zz.imag], axis=1).reshape(-1))
    nz = zz.size
    g = np.zeros(2 * nc * nz)
    resid = np.zeros(nc * nz)
    alpha = np.zeros(nc * max_steps)
    beta = np.zeros(nc * (max_steps + 1))
    opts = _KrylovOpts(max_steps, tol, dc, check_every)
    res = _KrylovResult()
    ctx._sync_stream()
    st = ctx.lib.hphi_shifted_krylov(ctx.h, ham.h, C.byref(opts), nc, pv, ld, nz, _np(zh), _np(g), _np(resid),
                                     _np(alpha), _np(beta), C.byref(res))
    if st not in (HPHI_OK, -4):
        ctx.check(st)
    G = (g[0::2] + 1j * g[1::2]).reshape(nc, nz)
    return dict(G=G, resid=resid.reshape(nc, nz), steps=res.steps, converged=bool(res.converged), status=st,
                max_resid=res.max_resid, alpha=alpha.reshape(nc, max_steps), beta=beta.reshape(nc, max_steps + 1))


def hphi_szz_spectrum(ham: Hamiltonian, gs, qs, z, max_steps: int, tol: float, check_every: int = 4):
    """S^zz(q, z) = -Im <Phi_q|(z - H)^{-1}|Phi_q>, Phi_q = sum_l e^{i q l} S^z_l gs,
    for every wave number in qs at once (one shifted-Krylov run of all
    excitation columns inside the library).  gs: real contiguous CUDA vector
    (F64/F32).  Returns (S [nq][nz], D [nq][nz] complex, dict with resid
    [nq][nz], steps, converged, status, max_resid); NOTCONV is reported."""
    ctx = ham.ctx
    if not gs.is_cuda or gs.dim() != 1 or gs.stride(0) != 1 or gs.numel() != ham.dim:
        raise ValueError("gs must be a contiguous CUDA vector of the Hamiltonian's dimension")
    dc = _dtype_code(gs)
    if dc not in (F64, F32):
        raise ValueError("gs must be real (F64 or F32)")
    q = np.ascontiguousarray(np.atleast_1d(np.asarray(qs, dtype=np.float64)))
    zz = np.asarray(z, dtype=np.complex128).reshape(-1)
    zh = np.ascontiguousarray(np.stack([zz.real, zz.imag], axis=1).reshape(-1))
    nq, nz = q.size, zz.size
    S = np.zeros(nq * nz)
    Dh = np.zeros(2 * nq * nz)
    rs = np.zeros(nq * nz)
    opts = _KrylovOpts(max_steps, tol, dc, check_every)
    res = _KrylovResult()
    ctx._sync_stream()
    st = ctx.lib.hphi_szz_spectrum(ctx.h, ham.h, C.byref(opts), C.c_void_p(gs.data_ptr()), nq, _np(q), nz, _np(zh),
                                   _np(S), _np(Dh), _np(rs), C.byref(res))
    if st not in (HPHI_OK, -4):
        ctx.check(st)
    Dq = (Dh[0::2] + 1j * Dh[1::2]).reshape(nq, nz)
    return S.reshape(nq, nz), Dq, dict(resid=rs.reshape(nq, nz), steps=res.steps, converged=bool(res.converged),
                                       status=st, max_resid=res.max_resid)


def hphi_lobpcg(ham: Hamiltonian, X, max_iter: int, tol: float):
    """The m lowest eigenpairs (m = X.shape[1] <= 32) by LOBPCG; X (FP64 CUDA,
    [D][m] contiguous) holds the start block and receives the Ritz vectors.
    Returns a dict (evals, resid, iters, converged); NOTCONV is reported."""
    ctx = ham.ctx
    if not X.is_cuda or X.dtype.itemsize != 8 or X.is_complex() or X.dim() != 2 or not X.is_contiguous():
        raise ValueError("X must be a contiguous FP64 CUDA block [D][m]")
    m = X.shape[1]
    ev, rs, it = np.zeros(m), np.zeros(m), i32(0)
    ctx._sync_stream()
    st = ctx.lib.hphi_lobpcg(ctx.h, ham.h, m, C.c_void_p(X.data_ptr()), int(max_iter), float(tol), _np(ev), _np(rs),
                             C.byref(it))
    if st not in (HPHI_OK, -4):
        ctx.check(st)
    return dict(evals=ev, resid=rs, iters=it.value, converged=st == HPHI_OK, status=st)


def hphi_mtpq_step(ham: Hamiltonian, V, l: float, n_sites: int, k: int, norm2: np.ndarray):
    """One microcanonical TPQ step in place on V (U_m = 1 - H / (l N_s)) from
    the state of step index k; norm2 is updated in place.  Returns (e, h2,
    logd, beta) of the state before the step, beta_k from the library."""
    ctx = ham.ctx
    pv, nv, ld = _vec(V)
    assert norm2.dtype == np.float64 and norm2.size == nv and norm2.flags.c_contiguous
    e, h2, logd, beta = np.zeros(nv), np.zeros(nv), np.zeros(nv), np.zeros(nv)
    ctx._sync_stream()
    ctx.check(ctx.lib.hphi_mtpq_step(ctx.h, ham.h, _dtype_code(V), nv, pv, ld, float(l), int(n_sites), int(k),
                                     _np(norm2), _np(e), _np(h2), _np(logd), _np(beta)))
    return e, h2, logd, beta


def hphi_tpq_bootstrap(e, h2, log_norm, P: int, M: int, beta=None, picks=None, seed: int = 1):
    """E(beta_k), C(beta_k) with standard deviations from TPQ samples by the
    paper's bootstrap (computed in the library).  e, h2, log_norm:
    [n_samples][n_temps]; beta: [n_temps] or None (then C is returned without
    beta^2); picks: [M][P] sample indices or None (Philox draws of seed).
    Returns dict(e_mean, e_sd, c_mean, c_sd)."""
    lib = load_library()
    e, h2, ln = (np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (e, h2, log_norm))
    if e.ndim != 2 or h2.shape != e.shape or ln.shape != e.shape:
        raise ValueError("e, h2 and log_norm must share one [n_samples][n_temps] shape")
    ns, nk = e.shape
    b = None if beta is None else np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1))
    if b is not None and b.size != nk:
        raise ValueError("one beta per temperature")
    pk = None if picks is None else np.ascontiguousarray(np.asarray(picks, dtype=np.int32).reshape(M, P))
    out = {k: np.zeros(nk) for k in ("e_mean", "e_sd", "c_mean", "c_sd")}
    st = lib.hphi_tpq_bootstrap(ns, nk, _np(e), _np(h2), _np(ln), _np(b) if b is not None else None, int(P), int(M),
                                _np(pk) if pk is not None else None, C.c_uint64(seed), _np(out["e_mean"]),
                                _np(out["e_sd"]), _np(out["c_mean"]), _np(out["c_sd"]))
    if st != HPHI_OK:
        raise HphiError(st, "hphi_tpq_bootstrap failed")
    return out


def hphi_dump_pattern(ham: Hamiltonian, row0: int, row1: int):
    """Unmerged off-diagonal pattern of rows [row0, row1) in (row, term) order:
    host arrays rows, cols, signs (int8), term_ids (int32)."""
    ctx = ham.ctx
    cnt = i64(0)
    ctx._sync_stream()
    st = ctx.lib.hphi_dump_pattern(ctx.h, ham.h, row0, row1, None, None, None, None, C.byref(cnt))
    if st not in (HPHI_OK, -1) or cnt.value < 0:
        ctx.check(st)
    n = cnt.value
    rows = np.zeros(max(n, 1), np.int64)
    cols = np.zeros(max(n, 1), np.int64)
    signs = np.zeros(max(n, 1), np.int8)
    tids = np.zeros(max(n, 1), np.int32)
    cnt = i64(max(n, 1))
    ctx.check(ctx.lib.hphi_dump_pattern(ctx.h, ham.h, row0, row1, _np(rows), _np(cols), _np(signs), _np(tids),
                                        C.byref(cnt)))
    n = cnt.value
    return rows[:n], cols[:n], signs[:n], tids[:n]


def hphi_dump_pattern_merged(ham: Hamiltonian, row0: int, row1: int):
    """Merged, column-sorted pattern of rows [row0, row1) as host CSR arrays."""
    ctx = ham.ctx
    n = row1 - row0
    rowptr = np.zeros(n + 1, np.int64)
    cap = i64(0)
    ctx._sync_stream()
    st = ctx.lib.hphi_dump_pattern_merged(ctx.h, ham.h, row0, row1, _np(rowptr), None, None, C.byref(cap))
    if st not in (HPHI_OK, -1) or cap.value <= 0:
        ctx.check(st)
    cols = np.zeros(cap.value, np.int64)
    vals = np.zeros(cap.value, np.float64)
    ctx.check(ctx.lib.hphi_dump_pattern_merged(ctx.h, ham.h, row0, row1, _np(rowptr), _np(cols), _np(vals),
                                               C.byref(cap)))
    return rowptr, cols[:cap.value], vals[:cap.value]


def hphi_tridiag_eigen(a, b):
    """Eigenvalues (ascending) and eigenvectors (columns) of the tridiagonal
    with diagonal a and off-diagonal b[1:]; host-only, no GPU needed."""
    lib = load_library()
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    n = a.size
    ev = np.zeros(n)
    Z = np.zeros((n, n))
    st = lib.hphi_tridiag_eigen(n, _np(a), _np(b), _np(ev), _np(Z))
    if st != HPHI_OK:
        raise HphiError(st, "tridiagonal eigensolver failed")
    return ev, Z


def write_matrix_market(f, n: int, rowptr, cols, vals, row0: int = 0, comment: str = "hphi"):
    """Write rows of a pattern in the Matrix Market layout the paper prints
    (Sec. 3.1.2): a '%' comment line, 'rows cols nnz', then 1-based
    'l m re im' lines."""
    nnz = int(rowptr[-1] - rowptr[0])
    f.write(f"% {comment}\n{n} {n} {nnz} \n")
    for r in range(len(rowptr) - 1):
        for k in range(rowptr[r], rowptr[r + 1]):
            v = complex(vals[k])
            re, im = v.real + 0.0, v.imag + 0.0  # no negative zeros
            f.write(f"{row0 + r + 1} {int(cols[k]) + 1} {re!r}  {im!r}\n")
