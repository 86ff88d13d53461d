"""Pins of the oracle's tridiagonal solver and Lanczos driver.

References: numpy/scipy eigensolvers (LAPACK, ARPACK) on independently built
matrices, and closed forms."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle as O
from kron_ref import spin_hamiltonian, spin_sector_indices, hubbard_hamiltonian, hubbard_sector_indices
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_vectors, uniform_couplings


def test_tridiag_eigs_match_lapack():
    rng = np.random.default_rng(1)
    for m in (1, 2, 5, 40, 150):
        a = rng.standard_normal(m) * 3
        b = np.concatenate([[0.0], rng.uniform(0.1, 2.0, m - 1)])
        ref = sla.eigvalsh_tridiagonal(a, b[1:]) if m > 1 else a.copy()
        for k in range(min(m, 4)):
            assert O.tridiag_eig(a, b, k) == pytest.approx(ref[k], abs=1e-13 * (1 + abs(ref[k])))
        # Sturm count between eigenvalues
        if m > 1:
            mid = 0.5 * (ref[0] + ref[1])
            assert O.sturm_count(a, b, mid) == 1
        y = O.tridiag_vec(a, b, ref[0])
        T = np.diag(a) + (np.diag(b[1:], 1) + np.diag(b[1:], -1) if m > 1 else 0)
        assert np.linalg.norm(T @ y - ref[0] * y) < 1e-10 * (1 + abs(ref[0]))


@pytest.mark.parametrize("N,seed", [(10, 1), (12, 2)])
def test_lanczos_ground_state_matches_dense(N, seed):
    Js = uniform_couplings(N, 0.5, 1.5, seed)
    terms = heisenberg_terms(chain(N), Js)
    m = O.Model("SPIN_HALF", N, N // 2, 0, terms)
    H = O.dense_matrix(m)
    w, V = np.linalg.eigh(H)
    v0 = random_vectors(m.dim, 1, seed)[:, 0]
    r = m.lanczos(v0, 300, 1e-12, want_gs=True)
    assert r["status"] == 0
    assert r["e0"] == pytest.approx(w[0], rel=1e-12)
    assert abs(np.dot(r["gs"], V[:, 0])) > 1 - 1e-10
    assert np.linalg.norm(H @ r["gs"] - r["e0"] * r["gs"]) < 1e-9


def test_lanczos_hubbard_matches_jordan_wigner():
    N = 5
    terms = hubbard_terms(N, chain(N), t=1.0, U=4.0)
    m = O.Model("HUBBARD", N, 2, 3, terms)
    Hk = hubbard_hamiltonian(N, terms)
    idx = hubbard_sector_indices(N, 2, 3)
    e_ref = np.linalg.eigvalsh(Hk[idx][:, idx].toarray())[0]
    r = m.lanczos(random_vectors(m.dim, 1, 8)[:, 0], 200, 1e-12)
    assert r["e0"] == pytest.approx(e_ref, rel=1e-12)


def test_lanczos_chain16_matches_independent_arpack():
    """The N=16 periodic Heisenberg chain, S^z=0 sector (12,870 states): the
    oracle's Lanczos against ARPACK on the Kronecker-built matrix."""
    N = 16
    terms = heisenberg_terms(chain(N), 1.0)
    Hk = spin_hamiltonian(N, terms)
    idx = spin_sector_indices(N, N // 2)
    Hs = Hk[idx][:, idx].tocsr()
    e_ref = spla.eigsh(Hs, k=1, which="SA", tol=1e-14)[0][0]
    m = O.Model("SPIN_HALF", N, N // 2, 0, terms)
    r = m.lanczos(random_vectors(m.dim, 1, 1)[:, 0], 300, 1e-12, want_gs=True)
    assert r["status"] == 0
    assert r["e0"] == pytest.approx(e_ref, rel=1e-11)
    # textbook cross-check (Bethe-ansatz value of the 16-site ring, to 5 digits)
    assert r["e0"] == pytest.approx(-7.14230, abs=2e-5)


def test_lanczos_exact_steps_and_breakdown():
    # a 2-dimensional space: the Krylov space is exhausted after 2 steps
    m = O.Model("SPIN_HALF", 2, 1, 0, heisenberg_terms([(0, 1)]))
    r = m.lanczos(np.array([1.0, 0.3]), 10, 0.0)
    assert r["status"] == 2 and r["steps"] == 2
    assert r["e0"] == pytest.approx(-0.75, abs=1e-14)
