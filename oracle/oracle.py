"""ctypes binding of the plain-C oracle plus numpy post-processing.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg, never by the GPU library.

Numpy parts:
  dense_matrix     H assembled from the oracle's own pattern (small D only)
  canonical_thermo exact canonical E(T), C(T) from a full spectrum
  bootstrap_tpq    the paper's bootstrap over TPQ samples (Sec. 3.5.1)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hphi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhphi_oracle.so")

MODELS = {"SPIN_HALF": 0, "SPIN_HALF_GC": 1, "HUBBARD": 2}
KINDS = {"EXCHANGE": 0, "XXZ": 1, "HOP": 2, "HUBBARD_U": 3, "DENS_DENS": 4}


class _Term(C.Structure):
    _fields_ = [("kind", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("spin", C.c_int32),
                ("v0", C.c_double), ("v1", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP row loop) into oracle/_build."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        i64, i32, dbl, vp = C.c_int64, C.c_int, C.c_double, C.c_void_p
        sig = {
            "orc_num_threads": (i32, []),
            "orc_binom": (i64, [i32, i32]),
            "orc_dim": (i64, [i32, i32, i32, i32]),
            "orc_enumerate": (i64, [i32, i32, vp, i64]),
            "orc_rank_search": (i64, [vp, i64, C.c_uint64]),
            "orc_rank_colex": (i64, [C.c_uint64]),
            "orc_unrank_colex": (C.c_uint64, [i64, i32]),
            "orc_lin_tables": (i32, [i32, i32, vp, vp]),
            "orc_model_create": (vp, [i32, i32, i32, i32, vp, i32, i32, C.POINTER(C.c_int)]),
            "orc_model_free": (None, [vp]),
            "orc_model_dim": (i64, [vp]),
            "orc_row_state": (None, [vp, i64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
            "orc_state_row": (i64, [vp, C.c_uint64, C.c_uint64]),
            "orc_row_entries": (i32, [vp, i64, vp, vp, vp, vp, i32]),
            "orc_max_row_entries": (i32, [vp]),
            "orc_pattern": (i64, [vp, i64, i64, vp, vp, vp, i64]),
            "orc_apply": (i32, [vp, i32, vp, i64, vp, i64, dbl, dbl, i64, i64]),
            "orc_sturm_count": (i32, [i32, vp, vp, dbl]),
            "orc_tridiag_eig": (dbl, [i32, vp, vp, i32]),
            "orc_tridiag_vec": (i32, [i32, vp, vp, dbl, vp]),
            "orc_lanczos": (i32, [vp, vp, i32, dbl, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), vp]),
            "orc_tpq_step": (i32, [vp, i32, i32, vp, dbl, i32, vp, vp, vp]),
            "orc_apply_sz_sum": (i32, [vp, vp, vp, vp, vp, vp, i64, i64]),
            "orc_time_step": (i32, [vp, i32, vp, dbl, i32, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    """Threads of the oracle's OpenMP row loop."""
    return int(_L().orc_num_threads())


def binom(n: int, k: int) -> int:
    return int(_L().orc_binom(n, k))


def enumerate_states(N: int, n: int) -> np.ndarray:
    cnt = binom(N, n)
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    got = _L().orc_enumerate(N, n, _ptr(out), cnt)
    assert got == cnt
    return out[:cnt]


def rank_colex(s: int) -> int:
    return int(_L().orc_rank_colex(int(s)))


def unrank_colex(r: int, n: int) -> int:
    return int(_L().orc_unrank_colex(int(r), int(n)))


def lin_tables(N: int, n: int):
    nlo, nhi = N - N // 2, N // 2
    ja = np.zeros(1 << nlo, dtype=np.uint32)
    jb = np.zeros(1 << nhi, dtype=np.uint64)
    st = _L().orc_lin_tables(N, n, _ptr(ja), _ptr(jb))
    if st != 0:
        raise ValueError("orc_lin_tables failed")
    return ja, jb


def sturm_count(a, b, x) -> int:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return int(_L().orc_sturm_count(len(a), _ptr(a), _ptr(b), float(x)))


def tridiag_eig(a, b, k: int = 0) -> float:
    """k-th smallest eigenvalue of the tridiagonal with diagonal a, off-diagonal b[1:]."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(_L().orc_tridiag_eig(len(a), _ptr(a), _ptr(b), k))


def tridiag_vec(a, b, theta) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    y = np.zeros(len(a))
    _L().orc_tridiag_vec(len(a), _ptr(a), _ptr(b), float(theta), _ptr(y))
    return y


class Model:
    """A sector plus an interaction list, held by the oracle."""

    def __init__(self, model: str, n_sites: int, n_up: int, n_dn: int, terms, use_lists: bool = False):
        arr = (_Term * max(len(terms), 1))()
        for k, (kind, i, j, spin, v0, v1) in enumerate(terms):
            arr[k] = _Term(KINDS[kind], i, j, spin, v0, v1)
        st = C.c_int(0)
        self._h = _L().orc_model_create(MODELS[model], n_sites, n_up, n_dn, C.cast(arr, C.c_void_p),
                                        len(terms), 1 if use_lists else 0, C.byref(st))
        if not self._h:
            raise ValueError(f"oracle rejected the model (status {st.value})")
        self.model, self.n_sites, self.n_up, self.n_dn = model, n_sites, n_up, n_dn
        self.terms = list(terms)
        self.dim = int(_L().orc_model_dim(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_model_free(h)
            self._h = None

    def row_state(self, r: int):
        su, sd = C.c_uint64(0), C.c_uint64(0)
        _L().orc_row_state(self._h, int(r), C.byref(su), C.byref(sd))
        return su.value, sd.value

    def state_row(self, su: int, sd: int = 0) -> int:
        return int(_L().orc_state_row(self._h, int(su), int(sd)))

    def row_entries(self, r: int, with_signs: bool = False):
        """Row r's entries in term order (diagonal first, term id -1): columns,
        values, term ids and, with with_signs, the fermion sign of each."""
        mx = _L().orc_max_row_entries(self._h)
        cols = np.zeros(mx, np.int64)
        vals = np.zeros(mx, np.float64)
        tids = np.zeros(mx, np.int32)
        signs = np.zeros(mx, np.int8)
        n = _L().orc_row_entries(self._h, int(r), _ptr(cols), _ptr(vals), _ptr(tids), _ptr(signs), mx)
        if n < 0:
            raise ValueError("row entries failed")
        if with_signs:
            return cols[:n], vals[:n], tids[:n], signs[:n]
        return cols[:n], vals[:n], tids[:n]

    def pattern_terms(self, r0: int, r1: int):
        """The unmerged off-diagonal pattern of rows [r0, r1) ordered by (row,
        term order): arrays rows, cols, signs, term_ids (Sec. 3.1.2 lists H
        entry by entry; here every term's entry is kept separately)."""
        rows, cols, signs, tids = [], [], [], []
        for r in range(r0, r1):
            c, _, t, sg = self.row_entries(r, with_signs=True)
            rows.append(np.full(len(c) - 1, r, np.int64))
            cols.append(c[1:])
            signs.append(sg[1:])
            tids.append(t[1:])
        cat = (lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
        return cat(rows, np.int64), cat(cols, np.int64), cat(signs, np.int8), cat(tids, np.int32)

    def pattern(self, r0: int = 0, r1: int | None = None):
        """Merged, column-sorted CSR pattern of rows [r0, r1)."""
        r1 = self.dim if r1 is None else r1
        mx = _L().orc_max_row_entries(self._h)
        cap = (r1 - r0) * mx
        rowptr = np.zeros(r1 - r0 + 1, np.int64)
        cols = np.zeros(max(cap, 1), np.int64)
        vals = np.zeros(max(cap, 1), np.float64)
        n = _L().orc_pattern(self._h, r0, r1, _ptr(rowptr), _ptr(cols), _ptr(vals), cap)
        if n < 0:
            raise ValueError("pattern failed")
        return rowptr, cols[:n].copy(), vals[:n].copy()

    def apply(self, x: np.ndarray, alpha: float = 1.0, beta: float = 0.0, y: np.ndarray | None = None,
              rows: tuple[int, int] | None = None) -> np.ndarray:
        """y = alpha H x + beta y for real [D] or [D][nvec] float64 x (rows r0..r1 only if given)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        squeeze = x.ndim == 1
        x2 = x.reshape(self.dim, -1)
        nvec = x2.shape[1]
        if y is None:
            y = np.zeros_like(x2)
        y2 = y.reshape(self.dim, -1)
        assert y2.flags.c_contiguous and y2.dtype == np.float64
        r0, r1 = rows if rows is not None else (0, self.dim)
        st = _L().orc_apply(self._h, nvec, _ptr(x2), nvec, _ptr(y2), nvec, float(alpha), float(beta), r0, r1)
        if st != 0:
            raise ValueError("apply failed")
        return y2.reshape(-1) if squeeze else y2

    def lanczos(self, v0: np.ndarray, max_steps: int, tol: float, want_gs: bool = False):
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        alpha = np.zeros(max_steps)
        beta = np.zeros(max_steps + 1)
        steps, e0, res = C.c_int(0), C.c_double(0), C.c_double(0)
        gs = np.zeros(self.dim) if want_gs else None
        st = _L().orc_lanczos(self._h, _ptr(v0), max_steps, tol, _ptr(alpha), _ptr(beta), C.byref(steps),
                              C.byref(e0), C.byref(res), _ptr(gs) if want_gs else None)
        if st < 0:
            raise ValueError("lanczos failed")
        k = steps.value
        return dict(status=st, steps=k, e0=e0.value, resid=res.value, alpha=alpha[:k], beta=beta[:k + 1], gs=gs)

    def sz_sum(self, x: np.ndarray, A, rows: tuple[int, int] | None = None) -> np.ndarray:
        """sum_l A_l S^z_l x for one real vector x and complex weights A[N];
        with rows=(r0, r1), x and the result cover those rows only."""
        r0, r1 = rows if rows is not None else (0, self.dim)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        assert x.size == r1 - r0
        A = np.asarray(A, dtype=np.complex128).reshape(-1)
        assert A.size == self.n_sites
        are, aim = np.ascontiguousarray(A.real), np.ascontiguousarray(A.imag)
        yr, yi = np.zeros(r1 - r0), np.zeros(r1 - r0)
        st = _L().orc_apply_sz_sum(self._h, _ptr(are), _ptr(aim), _ptr(x), _ptr(yr), _ptr(yi), r0, r1)
        if st != 0:
            raise ValueError("sz_sum failed")
        return yr + 1j * yi

    def time_step(self, V: np.ndarray, dt: float, nmax: int):
        """One real-time step in place on complex V ([D] or [D][nvec]).
        Returns (norm2, e) before the step and norm2 after it, per column."""
        assert np.iscomplexobj(V) and V.dtype == np.complex128 and V.flags.c_contiguous
        nvec = 1 if V.ndim == 1 else V.shape[1]
        n2, e, n2n = np.zeros(nvec), np.zeros(nvec), np.zeros(nvec)
        st = _L().orc_time_step(self._h, nvec, _ptr(V.view(np.float64)), float(dt), int(nmax), _ptr(n2), _ptr(e),
                                _ptr(n2n))
        if st != 0:
            raise ValueError("time_step failed")
        return n2, e, n2n

    def tpq_step(self, V: np.ndarray, dtau: float, nmax: int):
        """One cTPQ step in place on V ([D][nvec] real or complex). Returns e, h2, d."""
        cplx = np.iscomplexobj(V)
        assert V.flags.c_contiguous
        nvec = V.shape[1]
        Vr = V.view(np.float64)
        e, h2, d = np.zeros(nvec), np.zeros(nvec), np.zeros(nvec)
        st = _L().orc_tpq_step(self._h, nvec, 2 if cplx else 1, _ptr(Vr), float(dtau), int(nmax), _ptr(e),
                               _ptr(h2), _ptr(d))
        if st != 0:
            raise ValueError("tpq_step failed")
        return e, h2, d


def dense_matrix(m: Model) -> np.ndarray:
    """H as a dense array, assembled from the oracle's pattern (small D only)."""
    rowptr, cols, vals = m.pattern()
    H = np.zeros((m.dim, m.dim))
    for r in range(m.dim):
        a, b = rowptr[r], rowptr[r + 1]
        H[r, cols[a:b]] += vals[a:b]
    return H


def canonical_thermo(evals: np.ndarray, temps: np.ndarray):
    """Exact canonical averages from a full spectrum (k_B = 1):
    E(T) = <H>, C(T) = (<H^2> - <H>^2) / T^2 (the definition in Sec. 3.5.2)."""
    evals = np.asarray(evals, dtype=np.float64)
    E, Cv = [], []
    for T in np.atleast_1d(temps):
        w = np.exp(-(evals - evals.min()) / T)
        Z = w.sum()
        e1 = (w * evals).sum() / Z
        e2 = (w * evals ** 2).sum() / Z
        E.append(e1)
        Cv.append((e2 - e1 ** 2) / T ** 2)
    return np.array(E), np.array(Cv)


def bootstrap_tpq(num_h: np.ndarray, num_h2: np.ndarray, log_norm: np.ndarray, P: int, M: int,
                  seed: int | None = None, picks: np.ndarray | None = None):
    """The paper's bootstrap over N TPQ samples (Sec. 3.5.1).

    Inputs per sample n and temperature index k: the unnormalised expectation
    pieces are num_h[n,k] = <Phi|H|Phi>/<Phi|Phi>, num_h2 likewise for H^2, and
    log_norm[n,k] = log <Phi^n(beta_k)|Phi^n(beta_k)>.  For m = 0..M-1 the
    resampling R_m is a list of P sample indices drawn with replacement
    (picks[m][p]; the random draw is an input: picks, or the seeded Philox
    stream of workloads.rng.bootstrap_picks when only seed is given);
        A_m = sum_p <Phi^R|A|Phi^R>,  Z_m = sum_p <Phi^R|Phi^R>,  <A>_m = A_m / Z_m,
    with all norms divided by W(beta_k) = <Phi^0|Phi^0> (the paper's
    normalisation by sample 0).  Returns mean and standard deviation over m of
    <H>_m, of <H^2>_m and of C_m = beta^2 (<H^2>_m - <H>_m^2) (the latter is
    returned without the beta^2 factor: the caller multiplies).  The variance
    uses the reading sigma^2 = 1/(M-1) sum_m (<A>_m - mean)^2.
    """
    num_h = np.asarray(num_h)
    Nn, K = num_h.shape
    if picks is None:
        from workloads.rng import bootstrap_picks
        picks = bootstrap_picks(M, P, Nn, seed)
    picks = np.asarray(picks, dtype=np.int64)
    assert picks.shape == (M, P) and picks.min() >= 0 and picks.max() < Nn
    w = np.exp(log_norm - log_norm[0:1, :])  # tilde norms relative to sample 0
    eh, eh2 = np.zeros((M, K)), np.zeros((M, K))
    for m in range(M):
        sel = picks[m]
        Z = w[sel].sum(axis=0)
        eh[m] = (w[sel] * num_h[sel]).sum(axis=0) / Z
        eh2[m] = (w[sel] * num_h2[sel]).sum(axis=0) / Z
    fl = eh2 - eh ** 2
    out = {}
    for name, a in (("H", eh), ("H2", eh2), ("fluct", fl)):
        mean = a.mean(axis=0)
        sd = np.sqrt(((a - mean) ** 2).sum(axis=0) / (M - 1)) if M > 1 else np.zeros(K)
        out[name] = (mean, sd)
    return out
