"""The named workloads: lattices, couplings, sectors and solver settings.

Each builder returns a dict with the model, sizes, term list and solver
parameters.  Only inputs live here; dimensions quoted in the docstrings are the
binomial counts of the sectors.
"""
from __future__ import annotations

from .lattice import chain, square, ladder, random_regular_graph, uniform_couplings
from .terms import heisenberg_terms, hubbard_terms


def heisenberg_chain16():
    """Spin-1/2 Heisenberg chain, N=16, periodic, J=1, Sz=0 (12,870 states);
    Lanczos to residual 1e-12 from a seeded Gaussian start vector (seed 1)."""
    N = 16
    return dict(name="heisenberg_chain_N16_Sz0", model="SPIN_HALF", n_sites=N, n_up=N // 2, n_dn=0,
                terms=heisenberg_terms(chain(N), 1.0), seed=1, tol=1e-12, max_steps=300, dim=12870)


def heisenberg_square4x8():
    """Spin-1/2 Heisenberg J1 model, 4x8 periodic square lattice (Lx=8, Ly=4,
    site = x + 8y), N=32, Sz=0 (601,080,390 states); 150 Lanczos steps plus
    the ground-state vector."""
    N = 32
    return dict(name="heisenberg_square_4x8_Sz0", model="SPIN_HALF", n_sites=N, n_up=16, n_dn=0,
                terms=heisenberg_terms(square(8, 4), 1.0), seed=2, lanczos_steps=150, dim=601080390)


def hubbard_square4x4(U=8.0):
    """Fermi-Hubbard 4x4 periodic square, t=1, U=8, N_up=N_dn=8
    (12,870^2 = 165,636,900 states)."""
    N = 16
    return dict(name="hubbard_square_4x4_half", model="HUBBARD", n_sites=N, n_up=8, n_dn=8,
                terms=hubbard_terms(N, square(4, 4), t=1.0, U=U), seed=3, tol=1e-10, max_steps=200,
                dim=12870 * 12870)


def ctpq_random_regular(N=26, n_vec=16, seed=4):
    """cTPQ on the full 2^N space of a Heisenberg model on a seeded random
    3-regular graph with J_ij ~ U[0.5, 1.5]; a block of n_vec complex Gaussian
    vectors; nmax=6, dtau=0.02 (the paper's cTPQ benchmark values, Sec. 3.5.2),
    2000 steps (beta up to 40)."""
    bonds = random_regular_graph(N, 3, seed)
    Js = uniform_couplings(len(bonds), 0.5, 1.5, seed + 1000)
    return dict(name=f"ctpq_rrg3_N{N}_B{n_vec}", model="SPIN_HALF_GC", n_sites=N, n_up=0, n_dn=0,
                terms=heisenberg_terms(bonds, Js), seed=seed, n_vec=n_vec, nmax=6, dtau=0.02,
                steps=2000, dim=1 << N)


def small_chain(N, J=1.0, n_up=None, pbc=True):
    return dict(model="SPIN_HALF", n_sites=N, n_up=N // 2 if n_up is None else n_up, n_dn=0,
                terms=heisenberg_terms(chain(N, pbc), J))


def small_hubbard_chain(N, t=1.0, U=4.0, n_up=None, n_dn=None, pbc=True):
    return dict(model="HUBBARD", n_sites=N, n_up=N // 2 if n_up is None else n_up,
                n_dn=N // 2 if n_dn is None else n_dn, terms=hubbard_terms(N, chain(N, pbc), t=t, U=U))


def ladder_terms(L, J=1.0):
    return heisenberg_terms(ladder(L), J)
