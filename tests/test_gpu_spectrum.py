"""GPU dynamical correlation functions (Sec. 3.2) against the oracle.

Tolerances.  The excitation is one product per row: FP64 1e-14, FP32 2^-23
relative per element.  The Krylov scalars follow the oracle's FP64 Lanczos to
1e-10 over the first steps (rounding in a different summation order, grown by
the recurrence).  Converged D(z) (every residual <= 1e-10) lies within
|r|^2 |b|^2 / eta of the exact resolvent, so the comparison with the dense
resolvent uses 1e-8 relative to max |D|; FP32 vectors (rounding 6e-8 per
element, amplified by the Krylov recurrence) use 1e-4."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import spectrum as S
from gpu_util import ctx, pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_regular_graph, uniform_couplings, \
    random_vectors

pytestmark = pytest.mark.gpu


def _phase(L, q):
    return np.exp(1j * q * np.arange(L))


CASES = {
    "sector": ("SPIN_HALF", 14, 7, 0, lambda: heisenberg_terms(chain(14), 1.0)),
    "sector_odd": ("SPIN_HALF", 13, 4, 0, lambda: heisenberg_terms(chain(13), 1.0)),
    "full": ("SPIN_HALF_GC", 12, 0, 0, lambda: heisenberg_terms(random_regular_graph(12, 3, 2),
                                                               uniform_couplings(18, 0.5, 1.5, 7))),
    "hubbard": ("HUBBARD", 6, 3, 2, lambda: hubbard_terms(6, chain(6), t=1.0, U=4.0)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sz_sum_matches_oracle(case, dtype):
    model, N, nu, nd, terms = CASES[case]
    m, b, h = pair(model, N, nu, nd, terms())
    rng = np.random.default_rng(N)
    A = rng.normal(size=N) + 1j * rng.normal(size=N)
    x = torch.from_numpy(random_vectors(m.dim, 1, 5).reshape(-1)).to(dtype).cuda()
    y = torch.zeros(m.dim, dtype=torch.complex128 if dtype == torch.float64 else torch.complex64, device="cuda")
    hphi.hphi_apply_sz_sum(b, x, y, A)
    want = m.sz_sum(x.cpu().double().numpy(), A)
    tol = 1e-14 if dtype == torch.float64 else 2e-7
    assert np.abs(y.cpu().numpy() - want).max() <= tol * np.abs(want).max()


def test_sz_sum_strided_operands():
    """x a column of a block, y two columns inside a wider block."""
    m, b, h = pair("SPIN_HALF", 12, 6, 0, heisenberg_terms(chain(12), 1.0))
    X = torch.from_numpy(random_vectors(m.dim, 3, 6)).cuda()
    Y = torch.zeros((m.dim, 5), dtype=torch.float64, device="cuda")
    A = _phase(12, 2 * np.pi * 5 / 12)
    hphi.hphi_apply_sz_sum(b, X[:, 1], Y[:, 2:4], A)
    want = m.sz_sum(X[:, 1].cpu().numpy(), A)
    Yh = Y.cpu().numpy()
    assert np.abs(Yh[:, 2] + 1j * Yh[:, 3] - want).max() < 1e-14 * np.abs(want).max()
    assert (Yh[:, [0, 1, 4]] == 0).all()


def test_sz_sum_rejects_overlap_and_cpu_tensors():
    m, b, h = pair("SPIN_HALF", 8, 4, 0, heisenberg_terms(chain(8), 1.0))
    Y = torch.zeros((m.dim, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(hphi.HphiError):
        hphi.hphi_apply_sz_sum(b, Y[:, 0], Y[:, 1:3], np.ones(8))
    with pytest.raises(ValueError):
        hphi.hphi_apply_sz_sum(b, torch.zeros(m.dim, dtype=torch.float64), Y[:, 1:3], np.ones(8))


def test_sz_sum_full_size_sampled():
    """The 4x8 S^z=0 sector (601,080,390 rows), FP32, sampled row windows."""
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    x = torch.empty(m.dim, dtype=torch.float32, device="cuda")
    hphi.hphi_random_vector(b.ctx, x, 7)
    y = torch.empty(m.dim, dtype=torch.complex64, device="cuda")
    A = _phase(32, 2 * np.pi * 3 / 8)
    hphi.hphi_apply_sz_sum(b, x, y, A)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    for r0 in [0, m.dim - 300] + list(rng.integers(0, m.dim - 300, 6)):
        r0 = int(r0)
        xs = x[r0:r0 + 300].cpu().double().numpy()
        want = m.sz_sum(xs, A, rows=(r0, r0 + 300))
        got = y[r0:r0 + 300].cpu().numpy()
        assert np.abs(got - want).max() <= 2e-7 * max(np.abs(want).max(), 1e-30)
    del x, y
    torch.cuda.empty_cache()


def _rhs(m, ncol, seed, dtype):
    return torch.from_numpy(random_vectors(m.dim, ncol, seed)).to(dtype).cuda().contiguous()


@pytest.mark.parametrize("case", ["sector", "full", "hubbard"])
def test_krylov_scalars_match_oracle_lanczos(case):
    model, N, nu, nd, terms = CASES[case]
    m, b, h = pair(model, N, nu, nd, terms())
    B = _rhs(m, 3, 21, torch.float64)
    z = np.array([0.3 + 0.1j, -1.0 + 0.5j])
    k = 25
    r = hphi.hphi_shifted_krylov(h, B, z, k, 0.0)
    assert r["steps"] == k
    Bh = B.cpu().numpy()
    for c in range(3):
        o = m.lanczos(Bh[:, c], k, 0.0)
        assert o["steps"] == k
        assert np.allclose(r["alpha"][c], o["alpha"], rtol=1e-10, atol=1e-12)
        assert np.allclose(r["beta"][c, 1:], o["beta"][1:], rtol=1e-10, atol=1e-12)
        assert r["beta"][c, 0] == pytest.approx(np.linalg.norm(Bh[:, c]), rel=1e-14)
        n2 = Bh[:, c] @ Bh[:, c]
        G, res = S.lanczos_galerkin(o["alpha"], o["beta"], n2, z)
        assert np.allclose(r["G"][c], G, rtol=1e-9)
        assert np.allclose(r["resid"][c], res, rtol=1e-8)


@pytest.mark.parametrize("case", ["sector", "hubbard", "full"])
def test_converged_d_matches_dense_resolvent(case):
    model, N, nu, nd, terms = CASES[case]
    if case == "sector":
        N, nu, terms = 12, 6, (lambda: heisenberg_terms(chain(12), 1.0))
    if case == "full":
        N, terms = 10, (lambda: heisenberg_terms(chain(10), 1.0))
    m, b, h = pair(model, N, nu, nd, terms())
    H = O.dense_matrix(m)
    E = np.linalg.eigvalsh(H)
    z = E[0] + np.linspace(-0.5, 6.0, 33) + 0.1j
    B = _rhs(m, 2, 31, torch.float64)
    r = hphi.hphi_shifted_krylov(h, B, z, 3000, 1e-10, check_every=10)
    assert r["converged"] and r["max_resid"] <= 1e-10
    Bh = B.cpu().numpy()
    for c in range(2):
        want = S.resolvent_dense(H, Bh[:, c], z)
        assert np.abs(r["G"][c] - want).max() < 1e-8 * np.abs(want).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_szz_pipeline_against_dense(dtype):
    """GPU ground state -> S^z(q) excitations of every q at once -> shifted
    Krylov, against the oracle's dense spectrum and eigenvectors."""
    L = 12
    m, b, h = pair("SPIN_HALF", L, L // 2, 0, heisenberg_terms(chain(L), 1.0))
    H = O.dense_matrix(m)
    E, U = np.linalg.eigh(H)
    v0 = torch.empty(m.dim, dtype=dtype, device="cuda")
    hphi.hphi_random_vector(b.ctx, v0, 1)
    gs = torch.empty_like(v0)
    lz = hphi.hphi_lanczos(h, v0, 200, 1e-12 if dtype == torch.float64 else 1e-6, gs_out=gs)
    assert abs(lz["e0"] - E[0]) < (1e-10 if dtype == torch.float64 else 1e-5)
    qs = 2 * np.pi * np.arange(L // 2 + 1) / L
    eta = 0.1
    z = lz["e0"] + np.linspace(0.0, 5.0, 51) + 1j * eta
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    Sq, Dq, r = hphi.hphi_szz_spectrum(h, gs, qs, z, 300, tol)
    assert r["converged"]
    assert np.array_equal(Sq, -Dq.imag)
    for k, q in enumerate(qs):
        phi = m.sz_sum(U[:, 0], _phase(L, q))
        want = S.resolvent_dense(H, phi, E[0] + np.linspace(0.0, 5.0, 51) + 1j * eta)
        bound = (1e-7 if dtype == torch.float64 else 2e-3) * np.abs(want).max() + 1e-12
        assert np.abs(Dq[k] - want).max() < bound, (k, np.abs(Dq[k] - want).max())
    # q = 0: S^z_total Phi_0 = 0 in the S^z = 0 sector (one real column, zero)
    assert np.abs(Dq[0]).max() == 0.0 and r["resid"][0].max() == 0.0


def test_edge_cases():
    m, b, h = pair("SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0))
    H = O.dense_matrix(m)
    E, U = np.linalg.eigh(H)
    B = torch.zeros((m.dim, 3), dtype=torch.float64, device="cuda")
    B[:, 1] = torch.from_numpy(U[:, 0])                  # an eigenvector: invariant after one step
    B[:, 2] = torch.from_numpy(random_vectors(m.dim, 1, 3).reshape(-1))
    z = np.array([E[0] - 1.0 + 0j, 0.5 + 0.2j])         # a real shift below the spectrum, a complex one
    r = hphi.hphi_shifted_krylov(h, B, z, 300, 1e-11)
    assert r["converged"]
    assert (r["G"][0] == 0).all() and (r["resid"][0] == 0).all()   # zero column
    assert np.allclose(r["G"][1], 1.0 / (z - E[0]), rtol=1e-10)
    assert r["beta"][1, 2] == 0.0 and r["alpha"][1, 1] == 0.0        # stopped after one step
    want = S.resolvent_dense(H, B[:, 2].cpu().numpy(), z)
    assert np.allclose(r["G"][2], want, rtol=1e-8)
    assert abs(r["G"][2][0].imag) < 1e-12                           # real z below the spectrum: D real
    # too few steps: NOTCONV with the partial result filled in
    r2 = hphi.hphi_shifted_krylov(h, B[:, 2:3].contiguous(), z, 3, 1e-12)
    assert not r2["converged"] and r2["status"] == -4 and r2["steps"] == 3 and r2["max_resid"] > 1e-12
    G, res = S.lanczos_galerkin(r2["alpha"][0], r2["beta"][0], float(B[:, 2] @ B[:, 2]), z)
    assert np.allclose(r2["G"][0], G, rtol=1e-12) and np.allclose(r2["resid"][0], res, rtol=1e-10)
    with pytest.raises(hphi.HphiError):
        hphi.hphi_shifted_krylov(h, B, np.array([], dtype=complex), 10, 0.0)


def test_full_size_moments():
    """4x8 sector, two FP32 right-hand sides, 3 steps: alpha_0 = <b|H|b>/|b|^2
    (through the H*x entry point) and z D(z) -> |b|^2 at large |z|."""
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    B = torch.empty((m.dim, 2), dtype=torch.float32, device="cuda")
    hphi.hphi_random_vector(b.ctx, B, 9)
    z = np.array([1e6j, -1e6 + 1e6j])
    r = hphi.hphi_shifted_krylov(h, B, z, 3, 0.0)
    HB = torch.empty_like(B)
    hphi.hphi_apply_H(h, B, HB)
    for c in range(2):
        n2 = float((B[:, c].double() ** 2).sum())
        a0 = float((B[:, c].double() * HB[:, c].double()).sum()) / n2
        assert r["alpha"][c, 0] == pytest.approx(a0, rel=1e-5, abs=1e-5)
        assert r["beta"][c, 0] ** 2 == pytest.approx(n2, rel=1e-9)
        assert np.allclose(z * r["G"][c], n2, rtol=1e-4)
    del B, HB
    torch.cuda.empty_cache()
