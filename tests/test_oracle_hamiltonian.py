"""Pins of the oracle's matrix elements and H*x.

References: Kronecker / Jordan-Wigner constructions (kron_ref.py), closed forms
(two-site singlet -3J/4, 4-site ring -2J, Hubbard dimer, free fermions), trace
identities of the Heisenberg model, and dense products."""
import itertools
import math
import random

import numpy as np
import pytest

import oracle as O
from kron_ref import (spin_hamiltonian, hubbard_hamiltonian, spin_sector_indices, hubbard_sector_indices,
                      project)
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_regular_graph


def _random_spin_terms(N, nb, seed):
    rng = random.Random(seed)
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), nb)
    terms = []
    for k, (i, j) in enumerate(pairs):
        if k % 2:
            terms.append(("EXCHANGE", j, i, 0, rng.uniform(-1, 2), 0.0))
        else:
            terms.append(("XXZ", i, j, 0, rng.uniform(-1, 2), rng.uniform(-1, 2)))
    terms.append(terms[0])          # a duplicated bond is summed
    return terms


@pytest.mark.parametrize("N,n_up,seed", [(6, 3, 1), (7, 2, 2), (8, 4, 3), (9, 5, 4), (5, 0, 5), (5, 5, 6)])
def test_spin_sector_matches_kronecker(N, n_up, seed):
    terms = _random_spin_terms(N, min(10, N * (N - 1) // 2), seed)
    m = O.Model("SPIN_HALF", N, n_up, 0, terms, use_lists=(seed % 2 == 0))
    Hk = project(spin_hamiltonian(N, terms), spin_sector_indices(N, n_up))
    assert np.allclose(O.dense_matrix(m), Hk, atol=1e-14, rtol=0)


@pytest.mark.parametrize("N,seed", [(4, 1), (7, 2), (9, 3)])
def test_spin_full_space_matches_kronecker(N, seed):
    terms = _random_spin_terms(N, min(8, N * (N - 1) // 2), seed)
    m = O.Model("SPIN_HALF_GC", N, 0, 0, terms)
    Hk = spin_hamiltonian(N, terms).toarray()
    assert np.allclose(O.dense_matrix(m), Hk, atol=1e-14, rtol=0)


def _random_hubbard_terms(N, seed):
    rng = random.Random(seed)
    terms = []
    for (i, j) in rng.sample(list(itertools.combinations(range(N), 2)), min(5, N * (N - 1) // 2)):
        a, b = (i, j) if rng.random() < 0.5 else (j, i)
        terms.append(("HOP", a, b, rng.choice([-1, 0, 1]), rng.uniform(-1.5, 1.5), 0.0))
    for i in range(N):
        terms.append(("HUBBARD_U", i, i, 0, rng.uniform(0, 6), 0.0))
    i, j = rng.sample(range(N), 2)
    terms.append(("DENS_DENS", i, j, 0, rng.uniform(-1, 1), 0.0))
    return terms


@pytest.mark.parametrize("N,nu,nd,seed", [(3, 1, 2, 1), (4, 2, 2, 2), (4, 3, 1, 3), (5, 2, 3, 4), (5, 3, 3, 5)])
def test_hubbard_matches_jordan_wigner(N, nu, nd, seed):
    terms = _random_hubbard_terms(N, seed)
    m = O.Model("HUBBARD", N, nu, nd, terms, use_lists=(seed % 2 == 1))
    Hk = project(hubbard_hamiltonian(N, terms), hubbard_sector_indices(N, nu, nd))
    assert np.allclose(O.dense_matrix(m), Hk, atol=1e-14, rtol=0)


def test_two_site_singlet():
    for J in (1.0, 0.37, 2.5):
        m = O.Model("SPIN_HALF", 2, 1, 0, heisenberg_terms([(0, 1)], J))
        assert np.linalg.eigvalsh(O.dense_matrix(m))[0] == pytest.approx(-0.75 * J, abs=1e-15)


def test_four_site_ring():
    m = O.Model("SPIN_HALF", 4, 2, 0, heisenberg_terms(chain(4), 1.3))
    assert np.linalg.eigvalsh(O.dense_matrix(m))[0] == pytest.approx(-2.0 * 1.3, abs=1e-14)


def test_fully_polarised_sector():
    bonds = square(4, 3)
    Js = np.linspace(0.3, 1.7, len(bonds))
    terms = [("XXZ", i, j, 0, float(J), 0.8) for (i, j), J in zip(bonds, Js)]
    for n_up in (0, 12):
        m = O.Model("SPIN_HALF", 12, n_up, 0, terms)
        assert m.dim == 1
        assert O.dense_matrix(m)[0, 0] == pytest.approx(Js.sum() / 4, abs=1e-14)


@pytest.mark.parametrize("t,U", [(1.0, 0.0), (1.0, 4.0), (0.7, 8.0), (-1.0, 2.0)])
def test_hubbard_dimer(t, U):
    m = O.Model("HUBBARD", 2, 1, 1, hubbard_terms(2, [(0, 1)], t=t, U=U))
    e0 = np.linalg.eigvalsh(O.dense_matrix(m))[0]
    assert e0 == pytest.approx((U - math.sqrt(U * U + 16 * t * t)) / 2, abs=1e-14)


@pytest.mark.parametrize("Lx,Ly,nu,nd", [(4, 2, 4, 4), (3, 2, 2, 3), (6, 1, 3, 3)])
def test_free_fermions(Lx, Ly, nu, nd):
    N = Lx * Ly
    bonds = square(Lx, Ly) if Ly > 1 else chain(Lx)
    m = O.Model("HUBBARD", N, nu, nd, hubbard_terms(N, bonds, t=1.0, U=0.0))
    # single-particle levels of -t * adjacency
    A = np.zeros((N, N))
    for i, j in bonds:
        A[i, j] -= 1.0
        A[j, i] -= 1.0
    eps = np.linalg.eigvalsh(A)
    exact = eps[:nu].sum() + eps[:nd].sum()
    assert np.linalg.eigvalsh(O.dense_matrix(m))[0] == pytest.approx(exact, abs=1e-12)


def test_free_fermions_4x4_level_scheme():
    # the single-particle spectrum -2t(cos kx + cos ky) of the 4x4 torus
    bonds = square(4, 4)
    A = np.zeros((16, 16))
    for i, j in bonds:
        A[i, j] -= 1.0
        A[j, i] -= 1.0
    eps = np.sort(np.linalg.eigvalsh(A))
    levels = sorted(-2 * (math.cos(2 * math.pi * a / 4) + math.cos(2 * math.pi * b / 4))
                    for a in range(4) for b in range(4))
    assert np.allclose(eps, levels, atol=1e-12)
    # half filling, 8 fermions per species: -4 + 4*(-2) + 3*0 per species
    assert 2 * sum(levels[:8]) == pytest.approx(-24.0, abs=1e-12)


def test_atomic_limit_t0():
    N = 4
    m = O.Model("HUBBARD", N, 3, 2, hubbard_terms(N, chain(N), t=0.0, U=5.0))
    # minimum number of doubly occupied sites with 3 up and 2 down on 4 sites is 1
    assert np.linalg.eigvalsh(O.dense_matrix(m))[0] == pytest.approx(5.0, abs=1e-14)


def test_heisenberg_traces_full_space():
    bonds = random_regular_graph(10, 3, 11)
    Js = np.linspace(0.5, 1.5, len(bonds))
    terms = heisenberg_terms(bonds, Js)
    H = O.dense_matrix(O.Model("SPIN_HALF_GC", 10, 0, 0, terms))
    assert np.trace(H) == pytest.approx(0.0, abs=1e-11)
    assert np.trace(H @ H) / 1024 == pytest.approx(3.0 / 16.0 * (Js ** 2).sum(), rel=1e-13)


@pytest.mark.parametrize("model,N,nu,nd", [("SPIN_HALF", 10, 5, 0), ("SPIN_HALF_GC", 8, 0, 0),
                                          ("HUBBARD", 5, 2, 3)])
def test_apply_matches_dense_and_is_symmetric(model, N, nu, nd):
    if model == "HUBBARD":
        terms = _random_hubbard_terms(N, 9)
    else:
        terms = _random_spin_terms(N, 12, 9)
    m = O.Model(model, N, nu, nd, terms)
    H = O.dense_matrix(m)
    assert np.array_equal(H, H.T)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((m.dim, 3))
    y0 = rng.standard_normal((m.dim, 3))
    y = m.apply(x, alpha=0.7, beta=-0.4, y=y0.copy())
    assert np.allclose(y, 0.7 * H @ x - 0.4 * y0, atol=1e-13, rtol=1e-13)
    # a row range leaves the other rows alone
    y2 = m.apply(x[:, 0].copy(), rows=(3, 9))
    assert np.allclose(y2[3:9], (H @ x[:, 0])[3:9], atol=1e-13) and not y2[:3].any()


def test_pattern_merges_duplicates_and_sorts():
    terms = [("EXCHANGE", 0, 1, 0, 1.0, 0.0), ("EXCHANGE", 1, 0, 0, 0.5, 0.0), ("EXCHANGE", 1, 2, 0, 1.0, 0.0)]
    m = O.Model("SPIN_HALF", 3, 1, 0, terms)
    rowptr, cols, vals = m.pattern()
    for r in range(m.dim):
        c = cols[rowptr[r]:rowptr[r + 1]]
        assert list(c) == sorted(set(c)) and r in c


def test_invalid_models_rejected():
    with pytest.raises(ValueError):
        O.Model("SPIN_HALF", 4, 2, 0, [("HOP", 0, 1, 0, 1.0, 0.0)])
    with pytest.raises(ValueError):
        O.Model("HUBBARD", 4, 2, 2, [("EXCHANGE", 0, 1, 0, 1.0, 0.0)])
    with pytest.raises(ValueError):
        O.Model("SPIN_HALF", 4, 2, 0, [("EXCHANGE", 0, 0, 0, 1.0, 0.0)])
    with pytest.raises(ValueError):
        O.Model("SPIN_HALF", 4, 2, 0, [("EXCHANGE", 0, 4, 0, 1.0, 0.0)])


@pytest.mark.parametrize("N,nu,nd,seed", [(4, 2, 2, 11), (5, 2, 3, 12), (6, 3, 2, 13)])
def test_pattern_terms_signs_and_ids_match_jordan_wigner(N, nu, nd, seed):
    """Every off-diagonal entry of the unmerged pattern, sign x (-t of its
    term), equals the Jordan-Wigner matrix element, and the bits its term
    moves are the ones row and column differ in.  Hops are on distinct pairs
    so that each (row, col) has a single source term."""
    rng = random.Random(seed)
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), min(6, N * (N - 1) // 2))
    terms = []
    for (i, j) in pairs:
        a, b = (i, j) if rng.random() < 0.5 else (j, i)
        terms.append(("HOP", a, b, rng.choice([-1, 0, 1]), rng.uniform(0.5, 1.5), 0.0))
    terms.append(("HUBBARD_U", 0, 0, 0, 3.0, 0.0))
    m = O.Model("HUBBARD", N, nu, nd, terms)
    Hk = project(hubbard_hamiltonian(N, terms), hubbard_sector_indices(N, nu, nd))
    rows, cols, signs, tids = m.pattern_terms(0, m.dim)
    assert len(rows) > 0 and set(np.unique(signs)) <= {-1, 1}
    assert -1 in signs  # the cases reach odd fermion strings
    order = np.lexsort((tids, rows))
    assert np.array_equal(order, np.arange(len(rows)))  # (row, term) order
    mask = (1 << N) - 1
    for r, c, sg, k in zip(rows, cols, signs, tids):
        kind, i, j, spin, t, _ = terms[k]
        assert kind == "HOP"
        assert Hk[r, c] == pytest.approx(-t * sg, abs=1e-14)
        su, sd = m.row_state(int(r))
        cu, cd = m.row_state(int(c))
        flip = (1 << i) | (1 << j)
        assert ((su ^ cu) == flip and sd == cd and spin in (-1, 0)) or \
               ((sd ^ cd) == flip and su == cu and spin in (-1, 1))
    # every nonzero off-diagonal element of H is listed exactly once
    nz = [(a, b) for a, b in zip(*np.nonzero(Hk)) if a != b]
    assert sorted(nz) == sorted(zip(rows.tolist(), cols.tolist()))


def test_pattern_terms_spin_signs_are_positive_and_ids_follow_bonds():
    terms = _random_spin_terms(8, 10, 21)
    m = O.Model("SPIN_HALF", 8, 4, 0, terms)
    rows, cols, signs, tids = m.pattern_terms(0, m.dim)
    assert np.all(signs == 1)
    for r, c, k in zip(rows[:500], cols[:500], tids[:500]):
        _, i, j, _, _, _ = terms[k]
        assert m.row_state(int(r))[0] ^ m.row_state(int(c))[0] == (1 << i) | (1 << j)
