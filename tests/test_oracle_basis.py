"""Pins of the oracle's basis enumeration, ranking and two-table index.

Independent references: itertools combinations, Python's bisect on a plain
sorted list, and the counting definitions of the Lin tables."""
import bisect
import itertools
import random

import numpy as np
import pytest

import oracle as O
from kron_ref import strings_with_popcount


@pytest.mark.parametrize("N,n", [(1, 0), (1, 1), (4, 2), (8, 3), (10, 5), (12, 0), (12, 12), (13, 6)])
def test_enumeration_matches_combinations(N, n):
    got = O.enumerate_states(N, n)
    want = strings_with_popcount(N, n)
    assert list(map(int, got)) == want
    assert len(got) == O.binom(N, n)


@pytest.mark.parametrize("N,n", [(6, 3), (12, 4), (16, 8), (18, 9)])
def test_colex_rank_is_position(N, n):
    states = strings_with_popcount(N, n)
    for k, s in enumerate(states):
        assert O.rank_colex(s) == k
        assert O.unrank_colex(k, n) == s


def test_colex_rank_large_n_against_enumeration():
    # N=26: 10,400,600 states; compare random ones with bisect on the oracle's enumeration
    N, n = 26, 13
    states = O.enumerate_states(N, n)
    assert len(states) == 10400600
    lst = states.tolist()
    rng = random.Random(5)
    for _ in range(2000):
        k = rng.randrange(len(lst))
        s = lst[k]
        assert bisect.bisect_left(lst, s) == k
        assert O.rank_colex(s) == k
        assert O.unrank_colex(k, n) == s


def test_colex_rank_n32_sector_edges():
    # first / last states of the 4x8 S^z=0 sector (C(32,16) = 601,080,390)
    D = O.binom(32, 16)
    assert D == 601080390
    assert O.unrank_colex(0, 16) == (1 << 16) - 1
    assert O.unrank_colex(D - 1, 16) == ((1 << 16) - 1) << 16
    rng = random.Random(7)
    for _ in range(500):
        bits = rng.sample(range(32), 16)
        s = sum(1 << b for b in bits)
        assert O.unrank_colex(O.rank_colex(s), 16) == s


@pytest.mark.parametrize("N,n", [(4, 2), (7, 3), (10, 5), (12, 6), (13, 6), (16, 8), (16, 3)])
def test_lin_tables_index_every_state(N, n):
    ja, jb = O.lin_tables(N, n)
    nlo = N - N // 2
    states = strings_with_popcount(N, n)
    lowmask = (1 << nlo) - 1
    for k, s in enumerate(states):
        assert int(ja[s & lowmask]) + int(jb[s >> nlo]) == k
    # definition-level checks of both tables
    for l in range(1 << nlo):
        assert ja[l] == sum(1 for l2 in range(l) if bin(l2).count("1") == bin(l).count("1"))
    for h in range(1 << (N // 2)):
        need = n - bin(h).count("1")
        if need < 0 or need > nlo:
            assert jb[h] == np.uint64(0xFFFFFFFFFFFFFFFF)
        else:
            assert int(jb[h]) == sum(1 for s in states if (s >> nlo) < h)


def test_lin_tables_n32_shape_and_totals():
    ja, jb = O.lin_tables(32, 16)
    assert ja.shape == (65536,) and jb.shape == (65536,)
    assert int(ja.max()) == O.binom(16, 8) - 1 == 12869
    valid = jb != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert valid.all()           # every high half occurs when n = N/2
    assert int(jb[-1]) + 1 == O.binom(32, 16)   # last high half pairs with one low half (popcount 0)


@pytest.mark.parametrize("N,nu,nd", [(4, 2, 2), (5, 2, 3), (6, 3, 1)])
def test_hubbard_row_layout(N, nu, nd):
    m = O.Model("HUBBARD", N, nu, nd, [], use_lists=True)
    m2 = O.Model("HUBBARD", N, nu, nd, [], use_lists=False)
    ups = strings_with_popcount(N, nu)
    dns = strings_with_popcount(N, nd)
    assert m.dim == len(ups) * len(dns)
    for r in range(m.dim):
        su, sd = m.row_state(r)
        assert (su, sd) == (ups[r // len(dns)], dns[r % len(dns)])
        assert m2.row_state(r) == (su, sd)
        assert m.state_row(su, sd) == r == m2.state_row(su, sd)
