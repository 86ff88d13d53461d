"""Shared helpers of the GPU parity tests (CUDA library vs CPU oracle)."""
import numpy as np

import oracle as O
from paper_2307_13222_gb300 import hphi

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        import paper_2307_13222_gb300 as P
        P.build()
        O.build()
        _CTX = hphi.Context(0)
    return _CTX


def pair(model, N, nu, nd, terms, use_lists=False):
    """(oracle model, GPU basis, GPU hamiltonian) for the same problem."""
    c = ctx()
    b = hphi.Basis(c, model, N, nu, nd)
    h = hphi.Hamiltonian(c, b, terms)
    m = O.Model(model, N, nu, nd, terms, use_lists=use_lists)
    assert b.dim == m.dim
    return m, b, h


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
