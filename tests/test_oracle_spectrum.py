"""Pins of the spectrum oracle (Sec. 3.2: D(z) = <Phi_ex|(z - H)^{-1}|Phi_ex>).

The excitation operator is pinned against Kronecker-product S^z matrices and
the sum rule sum_q |S^z(q) Phi|^2 = L^2/4; the dense resolvent against the
two-site closed form and the moment expansion; the continued fraction and
the shifted COCG against the dense resolvent, against each other (the same
Galerkin iterate for real H and a real right-hand side) and against the
explicit residual."""
import numpy as np
import pytest

import oracle as O
from oracle import spectrum as S
import kron_ref as K
from workloads import chain, heisenberg_terms, hubbard_terms, random_vectors


def _gs(m):
    H = O.dense_matrix(m)
    E, U = np.linalg.eigh(H)
    return H, E[0], U[:, 0]


def _phase(L, q):
    return np.exp(1j * q * np.arange(L))


@pytest.mark.parametrize("model,N,nup,ndn", [("SPIN_HALF", 8, 4, 0), ("SPIN_HALF", 7, 2, 0), ("SPIN_HALF_GC", 6, 0, 0),
                                             ("HUBBARD", 4, 2, 1)])
def test_sz_sum_matches_kronecker_operators(model, N, nup, ndn):
    terms = hubbard_terms(N, chain(N), t=1.0, U=2.0) if model == "HUBBARD" else heisenberg_terms(chain(N), 1.0)
    m = O.Model(model, N, nup, ndn, terms)
    rng = np.random.default_rng(N + nup)
    A = rng.normal(size=N) + 1j * rng.normal(size=N)
    x = rng.normal(size=m.dim)
    if model == "HUBBARD":
        M = 2 * N
        cd = [K.fermion_cdag(k, M) for k in range(M)]
        num = [cd[k] @ cd[k].T for k in range(M)]
        op = sum(A[l] * 0.5 * (num[l] - num[N + l]) for l in range(N))
        idx = K.hubbard_sector_indices(N, nup, ndn)
    else:
        op = sum(A[l] * K.site_op(K.SZ, l, N) for l in range(N))
        idx = K.spin_sector_indices(N, nup) if model == "SPIN_HALF" else np.arange(1 << N)
    want = K.project(op.tocsr(), idx) @ x
    assert np.abs(m.sz_sum(x, A) - want).max() < 1e-13


def test_sz_total_is_the_sector_constant():
    m = O.Model("SPIN_HALF", 10, 3, 0, heisenberg_terms(chain(10), 1.0))
    x = np.random.default_rng(1).normal(size=m.dim)
    assert np.allclose(m.sz_sum(x, np.ones(10)), (3 - 5) * x, atol=1e-13, rtol=0)
    h = O.Model("HUBBARD", 5, 3, 1, hubbard_terms(5, chain(5), t=1.0, U=3.0))
    x = np.random.default_rng(2).normal(size=h.dim)
    assert np.allclose(h.sz_sum(x, np.ones(5)), 0.5 * (3 - 1) * x, atol=1e-13, rtol=0)


def test_structure_factor_sum_rule():
    """sum_{m<L} |S^z(q_m) Phi|^2 = L sum_l <(S^z_l)^2> = L^2 / 4 for a normalised Phi."""
    L = 10
    m = O.Model("SPIN_HALF", L, 5, 0, heisenberg_terms(chain(L), 1.0))
    phi = random_vectors(m.dim, 1, 5).reshape(-1)
    phi /= np.linalg.norm(phi)
    tot = sum(np.linalg.norm(m.sz_sum(phi, _phase(L, 2 * np.pi * k / L))) ** 2 for k in range(L))
    assert tot == pytest.approx(L * L / 4, rel=1e-13)


def test_dimer_closed_form():
    """Two sites: (S^z_0 - S^z_1) maps the singlet (E = -3J/4) to the m=0
    triplet (E = J/4) with unit norm, so D(z) = 1 / (z - J/4)."""
    J = 1.3
    m = O.Model("SPIN_HALF", 2, 1, 0, [("EXCHANGE", 0, 1, 0, J, 0.0)])
    H, e0, gs = _gs(m)
    assert e0 == pytest.approx(-0.75 * J, abs=1e-14)
    phi = m.sz_sum(gs, np.array([1.0, -1.0]))
    z = np.array([0.1 + 0.05j, -2.0 + 1.0j, 3.0 + 0.01j])
    want = 1.0 / (z - J / 4)
    assert np.allclose(S.resolvent_dense(H, phi, z), want, rtol=1e-13)
    r = m.lanczos(phi.real, 4, 0.0)
    assert r["steps"] == 1  # an eigenvector: the Krylov space is invariant after one step
    assert np.allclose(S.continued_fraction(r["alpha"], r["beta"], 1.0, z), want, rtol=1e-13)
    G, res = S.lanczos_galerkin(r["alpha"], r["beta"], 1.0, z)
    assert np.allclose(G, want, rtol=1e-13) and res.max() < 1e-14
    G2, res2, it = S.shifted_cocg(m, phi, z, 10, 1e-14)
    assert np.allclose(G2, want, rtol=1e-12) and res2.max() < 1e-13


def _chain_case(L=10, q_index=3):
    m = O.Model("SPIN_HALF", L, L // 2, 0, heisenberg_terms(chain(L), 1.0))
    H, e0, gs = _gs(m)
    phi = m.sz_sum(gs, _phase(L, 2 * np.pi * q_index / L))
    z = e0 + np.linspace(0.0, 5.0, 41) + 0.1j
    return m, H, e0, phi, z


def test_moments_of_the_resolvent():
    """Large |z|: D(z) = |Phi|^2/z + <Phi|H|Phi>/z^2 + <Phi|H^2|Phi>/z^3 + O(z^-4)."""
    m, H, e0, phi, _ = _chain_case()
    n2 = np.vdot(phi, phi).real
    h1 = np.vdot(phi, H @ phi).real
    h2 = np.vdot(H @ phi, H @ phi).real
    for z in (2e3j, 1e3 + 1e3j):
        D = S.resolvent_dense(H, phi, z)[0]
        third = z ** 3 * (D - n2 / z - h1 / z ** 2)
        assert abs(third - h2) < 50 * np.linalg.norm(H, 2) ** 3 * n2 / abs(z)


def test_complex_rhs_splits_into_real_parts():
    """For real symmetric H, G(z) is complex symmetric, so
    <a + ib|G|a + ib> = <a|G|a> + <b|G|b> (the cross terms cancel)."""
    m, H, e0, phi, z = _chain_case()
    full = S.resolvent_dense(H, phi, z)
    parts = S.resolvent_dense(H, phi.real, z) + S.resolvent_dense(H, phi.imag, z)
    assert np.abs(full - parts).max() < 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("q_index", [1, 3, 5])
def test_galerkin_and_cocg_converge_to_the_resolvent(q_index):
    m, H, e0, phi, z = _chain_case(q_index=q_index)
    want = S.resolvent_dense(H, phi, z)
    got = np.zeros_like(want)
    for part in (phi.real, phi.imag):
        n2 = part @ part
        if n2 == 0.0:
            continue
        r = m.lanczos(part, 120, 0.0)
        G, res = S.lanczos_galerkin(r["alpha"], r["beta"], n2, z)
        assert res.max() < 1e-9 or r["status"] == 2
        assert np.allclose(S.continued_fraction(r["alpha"], r["beta"], n2, z), G, rtol=1e-10)
        got += G
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    # shifted COCG on each real part (the complex excitation itself has
    # Phi^T Phi ~ 0, the breakdown case of the bilinear form)
    G2 = np.zeros_like(want)
    for part in (phi.real, phi.imag):
        if part @ part == 0.0:
            continue
        g, res2, it = S.shifted_cocg(m, part + 0j, z, 400, 1e-11)
        assert res2.max() < 1e-9
        G2 += g
    assert np.abs(G2 - want).max() < 1e-9 * np.abs(want).max()


def test_cocg_complex_rhs_and_its_breakdown_case():
    """A generic complex right-hand side converges to the resolvent; the
    excitation S^z(q) Phi_0 has r^T r = 0 up to rounding at the start."""
    m, H, e0, phi, z = _chain_case(q_index=1)
    assert abs(phi @ phi) < 1e-12 * np.vdot(phi, phi).real
    rng = np.random.default_rng(4)
    b = rng.normal(size=m.dim) + 1j * rng.normal(size=m.dim)
    want = S.resolvent_dense(H, b, z)
    G, res, it = S.shifted_cocg(m, b, z, 400, 1e-11)
    assert res.max() < 1e-9
    assert np.abs(G - want).max() < 1e-9 * np.abs(want).max()


def test_cocg_iterate_equals_lanczos_galerkin_iterate():
    """Real H, real b: the k-th shifted-COCG iterate is the Galerkin solution
    on K_k(H, b), so its D and explicit residual equal the Lanczos ones."""
    m, H, e0, phi, z = _chain_case()
    b = random_vectors(m.dim, 1, 9).reshape(-1)
    n2 = b @ b
    # k stays below the point where the first Ritz values converge: beyond it
    # both recurrences lose orthogonality in different rounding patterns and
    # agree only to the accuracy of the converged shifts
    for k in (3, 8, 15, 20):
        r = m.lanczos(b, k, 0.0)
        G, res = S.lanczos_galerkin(r["alpha"], r["beta"], n2, z)
        G2, res2, it = S.shifted_cocg(m, b + 0j, z, k, 0.0, seed=len(z) // 2)
        assert it == k
        assert np.abs(G2 - G).max() < 1e-11 * np.abs(G).max()
        assert np.allclose(res2, res, rtol=1e-10, atol=0)


def test_sz_sum_row_range_is_a_slice_of_the_full_result():
    m = O.Model("HUBBARD", 6, 3, 2, hubbard_terms(6, chain(6), t=1.0, U=2.0))
    rng = np.random.default_rng(3)
    A = rng.normal(size=6) + 1j * rng.normal(size=6)
    x = rng.normal(size=m.dim)
    full = m.sz_sum(x, A)
    for r0, r1 in ((0, 7), (13, 200), (m.dim - 5, m.dim), (40, 40)):
        assert np.array_equal(m.sz_sum(x[r0:r1], A, rows=(r0, r1)), full[r0:r1])
