"""LOBPCG (Sec. 3.3) against the dense spectrum and the oracle's sector
ground states: the m lowest levels with their degeneracies."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_vectors, uniform_couplings

pytestmark = pytest.mark.gpu


def _start(dim, m, seed):
    return torch.from_numpy(random_vectors(dim, m, seed)).cuda().contiguous()


@pytest.mark.parametrize("case", ["gc10", "sector14", "hubbard6"])
@pytest.mark.parametrize("m", [1, 4, 12])
def test_lowest_levels_against_dense(case, m):
    if case == "gc10":
        mm, b, h = pair("SPIN_HALF_GC", 10, 0, 0, heisenberg_terms(chain(10), uniform_couplings(10, 0.5, 1.5, 4)))
    elif case == "sector14":
        mm, b, h = pair("SPIN_HALF", 14, 7, 0, heisenberg_terms(chain(14), 1.0))
    else:
        mm, b, h = pair("HUBBARD", 6, 3, 3, hubbard_terms(6, chain(6), t=1.0, U=4.0))
    E, U = np.linalg.eigh(O.dense_matrix(mm))
    X = _start(mm.dim, m, 7 + m)
    r = hphi.hphi_lobpcg(h, X, 2000, 1e-9)
    assert r["converged"], r
    assert np.allclose(r["evals"], E[:m], rtol=0, atol=1e-9 * max(1.0, abs(E[0]))), (r["evals"], E[:m])
    Xh = X.cpu().numpy()
    assert np.allclose(Xh.T @ Xh, np.eye(m), atol=1e-10)
    H = O.dense_matrix(mm)
    res = np.linalg.norm(H @ Xh - Xh * r["evals"], axis=0)
    assert res.max() <= 1e-9 * max(1.0, abs(E[0])) * 1.01


def test_square_4x4_multiplets():
    """Full space of the 4x4 Heisenberg model (65,536 states): the lowest level
    is the S^z=0 ground state (a singlet), the lowest S^z=1 state appears three
    times (a triplet) and the lowest S^z=2 state five times (a quintuplet), with
    the energies of the oracle's sector ground states."""
    terms = heisenberg_terms(square(4, 4), 1.0)
    mm, b, h = pair("SPIN_HALF_GC", 16, 0, 0, terms)
    esec = {}
    for mz in (0, 1, 2):
        ms = O.Model("SPIN_HALF", 16, 8 + mz, 0, terms)
        esec[mz] = ms.lanczos(random_vectors(ms.dim, 1, 3)[:, 0], 400, 1e-12)["e0"]
    X = _start(mm.dim, 16, 21)
    r = hphi.hphi_lobpcg(h, X, 3000, 1e-9)
    assert r["converged"]
    ev = r["evals"]
    assert abs(ev[0] - esec[0]) < 1e-9
    for mz, mult in ((1, 3), (2, 5)):
        assert int(np.sum(np.abs(ev - esec[mz]) < 1e-8)) == mult, (mz, ev, esec[mz])


def test_rank_deficient_start_block_is_reported():
    mm, b, h = pair("SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0))
    X = _start(mm.dim, 3, 2)
    X[:, 2] = X[:, 0]
    with pytest.raises(hphi.HphiError):
        hphi.hphi_lobpcg(h, X, 100, 1e-9)
