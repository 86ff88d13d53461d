"""Interaction-term lists (the paper's J / t / U terms) as plain tuples.

A term is (kind, i, j, spin, v0, v1) with kind one of TERM_KINDS:
  EXCHANGE   J S_i.S_j                         v0 = J
  XXZ        Jz S^z_i S^z_j + Jxy (S^x S^x + S^y S^y)   v0 = Jz, v1 = Jxy
  HOP        -t (c^+_{i s} c_{j s} + h.c.)       v0 = t, spin 0 (up), 1 (down), -1 (both)
  HUBBARD_U  U n_{i up} n_{i down}              v0 = U (j == i)
  DENS_DENS  V n_i n_j                          v0 = V
Each side (the CUDA library and the oracle) maps the kind names to its own codes.
"""
from __future__ import annotations

TERM_KINDS = ("EXCHANGE", "XXZ", "HOP", "HUBBARD_U", "DENS_DENS")


def heisenberg_terms(bonds, J=1.0):
    """J S_i.S_j on every bond; J may be a scalar or one value per bond."""
    Js = [J] * len(bonds) if isinstance(J, (int, float)) else list(J)
    return [("EXCHANGE", i, j, 0, float(v), 0.0) for (i, j), v in zip(bonds, Js)]


def xxz_terms(bonds, Jz, Jxy):
    return [("XXZ", i, j, 0, float(Jz), float(Jxy)) for (i, j) in bonds]


def hubbard_terms(n_sites, bonds, t=1.0, U=0.0, V=0.0):
    terms = [("HOP", i, j, -1, float(t), 0.0) for (i, j) in bonds]
    if U != 0.0:
        terms += [("HUBBARD_U", i, i, 0, float(U), 0.0) for i in range(n_sites)]
    if V != 0.0:
        terms += [("DENS_DENS", i, j, 0, float(V), 0.0) for (i, j) in bonds]
    return terms
