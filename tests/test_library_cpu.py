"""Host-side checks of the CUDA library that need no GPU: the shared library
loads, exports every entry point the header declares, its host tridiagonal
solver matches LAPACK, and the Matrix Market writer reproduces the paper's
example."""
import io
import os
import re

import numpy as np
import pytest
import scipy.linalg as sla

import paper_2307_13222_gb300 as P
from paper_2307_13222_gb300 import hphi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    P.build()
    return hphi.load_library()


def _declared():
    txt = open(os.path.join(ROOT, "include", "hphi.h")).read()
    return sorted(set(re.findall(r"HPHI_API\s+[\w\s\*]*?\b(hphi_\w+)\s*\(", txt)))


def test_header_declares_and_library_exports_every_symbol(lib):
    declared = _declared()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(hphi.exported_symbols()) == declared


def test_tridiag_eigen_matches_lapack(lib):
    rng = np.random.default_rng(2)
    for n in (1, 2, 3, 17, 120):
        a = rng.standard_normal(n)
        b = np.concatenate([[0.0], rng.uniform(0.05, 1.5, n - 1)])
        ev, Z = hphi.hphi_tridiag_eigen(a, b)
        ref = sla.eigvalsh_tridiagonal(a, b[1:]) if n > 1 else a
        assert np.allclose(ev, ref, atol=1e-12 * (1 + np.abs(ref).max()))
        T = np.diag(a) + (np.diag(b[1:], 1) + np.diag(b[1:], -1) if n > 1 else 0)
        assert np.allclose(T @ Z, Z * ev, atol=1e-11)
        assert np.allclose(Z.T @ Z, np.eye(n), atol=1e-11)
        assert (Z[0] >= 0).all()


def test_tridiag_eigen_degenerate_and_split():
    # a zero off-diagonal splits the matrix; repeated eigenvalues
    a = np.array([1.0, 1.0, 2.0, 2.0])
    b = np.array([0.0, 0.0, 0.5, 0.0])
    ev, Z = hphi.hphi_tridiag_eigen(a, b)
    T = np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1)
    assert np.allclose(ev, np.linalg.eigvalsh(T), atol=1e-14)
    assert np.allclose(T @ Z, Z * ev, atol=1e-13)


def test_matrix_market_writer_reproduces_paper_example():
    gold = open(os.path.join(ROOT, "tests", "golden", "matrix_market_2by2.txt")).read().split("\n")
    f = io.StringIO()
    rowptr = np.array([0, 2, 4])
    cols = np.array([0, 1, 0, 1])
    vals = np.array([1.0, -1j, 1j, -1.0])
    hphi.write_matrix_market(f, 2, rowptr, cols, vals, comment="2by2")
    got = [" ".join(l.split()) for l in f.getvalue().strip().split("\n")]
    want = [" ".join(l.split()) for l in gold if l.strip()]
    assert got == want


def test_no_gpu_means_loud_failure():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        hphi.Context(0)
