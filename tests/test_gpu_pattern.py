"""GPU matrix pattern against the oracle: columns bit-exact, values to rounding."""
import itertools
import random

import numpy as np
import pytest

from gpu_util import pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_regular_graph, uniform_couplings

pytestmark = pytest.mark.gpu


def _cmp(m, h, r0, r1):
    orp, oc, ov = m.pattern(r0, r1)
    grp, gc, gv = hphi.hphi_dump_pattern_merged(h, r0, r1)
    _cmp_terms(m, h, r0, r1)
    assert np.array_equal(grp - grp[0], orp - orp[0])
    assert np.array_equal(gc, oc)
    assert np.allclose(gv, ov, rtol=1e-14, atol=1e-14)


def _cmp_terms(m, h, r0, r1):
    """The unmerged (row, col, sign, term id) pattern, bit-exact."""
    orow, ocol, osg, otid = m.pattern_terms(r0, r1)
    grow, gcol, gsg, gtid = hphi.hphi_dump_pattern(h, r0, r1)
    assert np.array_equal(grow, orow) and np.array_equal(gcol, ocol)
    assert np.array_equal(gsg, osg) and np.array_equal(gtid, otid)


def _random_spin_terms(N, nb, seed):
    rng = random.Random(seed)
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), nb)
    out = []
    for k, (i, j) in enumerate(pairs):
        if k % 3 == 0:
            out.append(("XXZ", j, i, 0, rng.uniform(-1, 2), rng.uniform(-1, 2)))
        elif k % 3 == 1:
            out.append(("XXZ", i, j, 0, rng.uniform(-1, 2), 0.0))      # Ising only
        else:
            out.append(("EXCHANGE", i, j, 0, rng.uniform(-1, 2), 0.0))
    out.append(out[-1])  # duplicate bond
    return out


@pytest.mark.parametrize("model,N,nu", [("SPIN_HALF", 8, 4), ("SPIN_HALF", 11, 3), ("SPIN_HALF", 16, 8),
                                        ("SPIN_HALF", 13, 13), ("SPIN_HALF_GC", 9, 0), ("SPIN_HALF_GC", 12, 0)])
def test_spin_pattern_random_bonds(model, N, nu):
    terms = _random_spin_terms(N, min(3 * N, N * (N - 1) // 2), N)
    m, b, h = pair(model, N, nu, 0, terms)
    _cmp(m, h, 0, m.dim)


def test_square_4x8_sampled_rows():
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    rng = np.random.default_rng(3)
    for r0 in list(rng.integers(0, m.dim - 600, 6)) + [0, m.dim - 600]:
        _cmp(m, h, int(r0), int(r0) + 600)


@pytest.mark.parametrize("N,nu,nd,seed", [(4, 2, 2, 1), (5, 2, 3, 2), (6, 3, 3, 3), (7, 2, 5, 4)])
def test_hubbard_pattern(N, nu, nd, seed):
    rng = random.Random(seed)
    terms = []
    for (i, j) in rng.sample(list(itertools.combinations(range(N), 2)), min(7, N * (N - 1) // 2)):
        terms.append(("HOP", j, i, rng.choice([-1, 0, 1]), rng.uniform(-1.5, 1.5), 0.0))
    terms += [("HUBBARD_U", i, i, 0, rng.uniform(0, 6), 0.0) for i in range(N)]
    terms.append(("DENS_DENS", 0, N - 1, 0, 0.7, 0.0))
    m, b, h = pair("HUBBARD", N, nu, nd, terms)
    _cmp(m, h, 0, m.dim)


def test_hubbard_4x4_sampled_rows():
    m, b, h = pair("HUBBARD", 16, 8, 8, hubbard_terms(16, square(4, 4), t=1.0, U=8.0))
    rng = np.random.default_rng(4)
    for r0 in list(rng.integers(0, m.dim - 300, 5)) + [0, m.dim - 300]:
        _cmp(m, h, int(r0), int(r0) + 300)


def test_rrg_gc_sampled_rows():
    bonds = random_regular_graph(26, 3, 4)
    terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004))
    m, b, h = pair("SPIN_HALF_GC", 26, 0, 0, terms)
    for r0 in (0, 12345678, (1 << 26) - 500):
        _cmp(m, h, r0, r0 + 500)


@pytest.mark.parametrize("N,nu,nd,seed", [(6, 3, 3, 7), (8, 4, 3, 8), (10, 5, 5, 9)])
def test_hubbard_terms_with_duplicates_and_cancellations(N, nu, nd, seed):
    """Duplicate hops, a hop listed with the opposite orientation and a
    cancelling pair (t and -t on the same bond): every term keeps its own
    entries, signs included, bit for bit; the merged matrix still agrees."""
    rng = random.Random(seed)
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), 6)
    terms = [("HOP", i, j, -1, rng.uniform(0.5, 1.5), 0.0) for (i, j) in pairs]
    i, j = pairs[0]
    terms.append(("HOP", j, i, -1, terms[0][4], 0.0))          # duplicate, reversed
    terms.append(("HOP", pairs[1][0], pairs[1][1], 0, 0.8, 0.0))
    terms.append(("HOP", pairs[1][0], pairs[1][1], 0, -0.8, 0.0))  # cancels the previous one
    terms.append(("HOP", 0, N - 1, 1, 1.1, 0.0))                # long hop: long fermion strings
    terms += [("HUBBARD_U", s, s, 0, 4.0, 0.0) for s in range(N)]
    m, b, h = pair("HUBBARD", N, nu, nd, terms)
    rows, cols, signs, tids = hphi.hphi_dump_pattern(h, 0, m.dim)
    assert -1 in signs and 1 in signs
    _cmp(m, h, 0, m.dim)


def test_pattern_export_capacity_and_range_errors():
    m, b, h = pair("SPIN_HALF", 8, 4, 0, heisenberg_terms(chain(8), 1.0))
    ctx = h.ctx
    import ctypes as C
    cnt = C.c_int64(0)
    st = ctx.lib.hphi_dump_pattern(ctx.h, h.h, 0, 5, None, None, None, None, C.byref(cnt))
    assert st == -1 and cnt.value == len(m.pattern_terms(0, 5)[0])
    with pytest.raises(hphi.HphiError):
        hphi.hphi_dump_pattern(h, 5, 5)
    with pytest.raises(hphi.HphiError):
        hphi.hphi_dump_pattern(h, 0, m.dim + 1)
