"""GPU basis tables and ranking against the oracle (bit-exact)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ctx
from paper_2307_13222_gb300 import hphi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n", [(2, 1), (5, 2), (12, 3), (16, 8), (17, 8), (20, 10), (24, 0), (24, 24), (32, 16)])
def test_lin_tables_bit_exact(N, n):
    b = hphi.Basis(ctx(), "SPIN_HALF", N, n)
    ja, jb = b.export_tables(0)
    oja, ojb = O.lin_tables(N, n)
    assert np.array_equal(ja, oja)
    assert np.array_equal(jb, ojb)
    assert b.dim == O.binom(N, n)


@pytest.mark.parametrize("N,n", [(10, 5), (16, 8), (21, 7), (32, 16)])
def test_states_and_rank(N, n):
    b = hphi.Basis(ctx(), "SPIN_HALF", N, n)
    rng = np.random.default_rng(N)
    rows = np.unique(np.concatenate([[0, b.dim - 1], rng.integers(0, b.dim, 3000)]))
    for r0 in rows[:50]:
        su, _ = b.states(int(r0), 1)
        assert int(su.item()) == O.unrank_colex(int(r0), n)
    # a contiguous run, ranked back
    r0 = int(rows[len(rows) // 2])
    k = min(5000, b.dim - r0)
    su, _ = b.states(r0, k)
    want = [O.unrank_colex(r, n) for r in range(r0, r0 + k)]
    assert su.cpu().numpy().tolist() == want
    back = b.rank(su)
    assert back.cpu().numpy().tolist() == list(range(r0, r0 + k))
    # outside the sector: wrong popcount, bits beyond N
    bad = torch.tensor([0, (1 << N) | 1, ((1 << N) - 1)], dtype=torch.int64, device="cuda") if n not in (0, N) else None
    if bad is not None:
        assert (b.rank(bad).cpu() == -1).all()


@pytest.mark.parametrize("N,nu,nd", [(4, 2, 2), (6, 3, 2), (8, 4, 4), (16, 8, 8)])
def test_hubbard_rows(N, nu, nd):
    b = hphi.Basis(ctx(), "HUBBARD", N, nu, nd)
    m = O.Model("HUBBARD", N, nu, nd, [])
    assert b.dim == m.dim
    rng = np.random.default_rng(1)
    rows = rng.integers(0, b.dim, 400)
    su, sd = b.states(0, b.dim) if b.dim < 100000 else (None, None)
    for r in rows:
        s1, s2 = b.states(int(r), 1)
        assert (int(s1.item()), int(s2.item())) == m.row_state(int(r))
    for sp, n in ((0, nu), (1, nd)):
        ja, jb = b.export_tables(sp)
        oja, ojb = O.lin_tables(N, n)
        assert np.array_equal(ja, oja) and np.array_equal(jb, ojb)


def test_gc_identity_rank():
    b = hphi.Basis(ctx(), "SPIN_HALF_GC", 20)
    assert b.dim == 1 << 20
    su, _ = b.states(12345, 10)
    assert su.cpu().numpy().tolist() == list(range(12345, 12355))
    na, nb = b.export_tables(0) if False else (None, None)


def test_invalid_sizes_rejected():
    c = ctx()
    for args in (("SPIN_HALF", 41, 3), ("SPIN_HALF", 10, 11), ("SPIN_HALF_GC", 37), ("HUBBARD", 33, 1, 1),
                 ("HUBBARD", 4, 5, 1)):
        with pytest.raises(hphi.HphiError) as ei:
            hphi.Basis(c, *args)
        assert ei.value.code == -1
