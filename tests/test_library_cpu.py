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


def test_library_bootstrap_matches_the_oracle(lib):
    """hphi_tpq_bootstrap (host code of the library) against the oracle's
    bootstrap on random sample data, with the same explicit resamplings and
    with the seeded draws (library Philox vs the input generator's)."""
    import oracle as O
    from workloads import bootstrap_picks
    rng = np.random.default_rng(3)
    e = rng.normal(size=(12, 30))
    h2 = e * e + rng.random(size=(12, 30))
    ln = np.cumsum(rng.normal(scale=0.1, size=(12, 30)), axis=1)
    beta = 0.05 * np.arange(30)
    for picks in (rng.integers(0, 12, size=(6, 12)), None):
        got = hphi.hphi_tpq_bootstrap(e, h2, ln, P=12, M=6, beta=beta, picks=picks, seed=5)
        ref = O.bootstrap_tpq(e, h2, ln, P=12, M=6, picks=picks if picks is not None else bootstrap_picks(6, 12, 12, 5))
        assert np.allclose(got["e_mean"], ref["H"][0], rtol=1e-13) and np.allclose(got["e_sd"], ref["H"][1], rtol=1e-11)
        assert np.allclose(got["c_mean"], beta ** 2 * ref["fluct"][0], rtol=1e-12, atol=1e-15)
        assert np.allclose(got["c_sd"], beta ** 2 * ref["fluct"][1], rtol=1e-10, atol=1e-15)


def test_library_bootstrap_hand_case_and_errors(lib):
    """The four ordered resamplings of two samples (weights 1, 3; <H> = 1, 2):
    mean 13/8, sigma^2 = (9/16)/(M-1) = 3/16; bad picks are refused."""
    import math
    e = np.array([[1.0], [2.0]])
    h2 = np.array([[2.0], [5.0]])
    ln = np.array([[0.0], [math.log(3.0)]])
    picks = np.array([[0, 0], [0, 1], [1, 0], [1, 1]])
    got = hphi.hphi_tpq_bootstrap(e, h2, ln, P=2, M=4, picks=picks)
    assert got["e_mean"][0] == pytest.approx(13 / 8, rel=1e-15)
    assert got["e_sd"][0] == pytest.approx(math.sqrt(3 / 16), rel=1e-14)
    assert got["c_mean"][0] == pytest.approx(35 / 32, rel=1e-15)
    assert got["c_sd"][0] == pytest.approx(math.sqrt(3 / 256), rel=1e-13)
    with pytest.raises(hphi.HphiError):
        hphi.hphi_tpq_bootstrap(e, h2, ln, P=2, M=1, picks=np.array([[0, 2]]))
