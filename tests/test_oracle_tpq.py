"""Pins of the oracle's cTPQ step, thermodynamics and bootstrap.

References: scipy.linalg.expm (the Taylor sum converges to it with a known
remainder), exact canonical ensembles from dense spectra (the paper's check of
cTPQ against full diagonalisation, Sec. 3.5.2), two-level closed forms."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from workloads import chain, heisenberg_terms, random_vectors, random_regular_graph, uniform_couplings


def _model(N=8, seed=3):
    bonds = random_regular_graph(N, 3, seed)
    Js = uniform_couplings(len(bonds), 0.5, 1.5, seed + 1)
    return O.Model("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(bonds, Js)), Js


@pytest.mark.parametrize("cplx", [False, True])
def test_tpq_step_converges_to_expm(cplx):
    m, _ = _model()
    H = O.dense_matrix(m)
    dtau = 0.02
    V = random_vectors(m.dim, 3, 9, complex_=cplx)
    V0 = V.copy()
    e, h2, d = m.tpq_step(V, dtau, 6)
    U = sla.expm(-0.5 * dtau * H)
    Hn = np.linalg.norm(H, 2)
    bound = (0.5 * dtau * Hn) ** 7 / math.factorial(7) * math.exp(0.5 * dtau * Hn)
    for q in range(3):
        phi = V0[:, q]
        ex = U @ phi
        assert np.linalg.norm(V[:, q] - ex / np.linalg.norm(ex)) < 4 * bound + 1e-14
        nn = np.vdot(phi, phi).real
        assert e[q] == pytest.approx(np.vdot(phi, H @ phi).real / nn, rel=1e-13)
        assert h2[q] == pytest.approx(np.vdot(H @ phi, H @ phi).real / nn, rel=1e-13)
        assert d[q] == pytest.approx(np.vdot(ex, ex).real / nn, rel=1e-11)


def test_tpq_high_temperature_moments():
    # beta = 0: <H> -> Tr H / d = 0 and <H^2> -> Tr H^2 / d = sum 3 J^2 / 16 (averaged over vectors)
    m, Js = _model(N=12, seed=5)
    V = random_vectors(m.dim, 16, 21)
    e, h2, d = m.tpq_step(V, 0.02, 6)
    s2 = 3.0 / 16.0 * (np.array(Js) ** 2).sum()
    assert abs(e.mean()) < 5 * math.sqrt(s2 / m.dim)
    assert h2.mean() == pytest.approx(s2, rel=0.05)


def test_ctpq_reproduces_canonical_ensemble():
    """cTPQ (nmax=6, dtau=0.02) on a 10-site chain over 2^10 states against
    the exact canonical averages from the dense spectrum."""
    N = 10
    m = O.Model("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(chain(N), 1.0))
    evals = np.linalg.eigvalsh(O.dense_matrix(m))
    nvec, steps, dtau = 24, 100, 0.02
    V = random_vectors(m.dim, nvec, 33)
    E = np.zeros((nvec, steps))
    E2 = np.zeros((nvec, steps))
    logn = np.zeros((nvec, steps))
    acc = np.zeros(nvec)
    for k in range(steps):
        e, h2, d = m.tpq_step(V, dtau, 6)
        E[:, k], E2[:, k], logn[:, k] = e, h2, acc
        acc = acc + np.log(d)
    betas = dtau * np.arange(steps)
    bs = O.bootstrap_tpq(E, E2, logn, P=nvec, M=nvec // 2, seed=1)
    mean, sd = bs["H"]
    for k in (25, 50, 99):
        ex, _ = O.canonical_thermo(evals, np.array([1.0 / betas[k]]))
        assert abs(mean[k] - ex[0]) < 4 * sd[k] + 0.02 * abs(ex[0])
    # norm bookkeeping: Z(beta)/Z(0) = Tr e^{-beta H} / d_H estimated by the mean of N_k / N_0
    k = 99
    z_est = np.exp(logn[:, k]).mean()
    z_ex = np.exp(-betas[k] * evals).sum() / len(evals)
    assert z_est == pytest.approx(z_ex, rel=0.15)


def test_canonical_thermo_two_level():
    gap = 1.7
    for T in (0.3, 1.0, 4.0):
        E, Cv = O.canonical_thermo(np.array([0.0, gap]), np.array([T]))
        x = gap / T
        assert E[0] == pytest.approx(gap / (1 + math.exp(x)), rel=1e-13)
        assert Cv[0] == pytest.approx(x * x * math.exp(x) / (1 + math.exp(x)) ** 2, rel=1e-12)


def test_bootstrap_identical_samples_have_zero_spread():
    K = 5
    E = np.tile(np.linspace(-1, 0, K), (8, 1))
    E2 = E ** 2 + 0.1
    logn = np.zeros((8, K))
    bs = O.bootstrap_tpq(E, E2, logn, P=8, M=4, seed=0)
    assert np.allclose(bs["H"][0], E[0]) and np.allclose(bs["H"][1], 0)
    assert np.allclose(bs["fluct"][0], 0.1)


def test_mtpq_step_is_the_first_order_operator():
    """mTPQ (Sec. 3.5.1): U_m = 1 - (dtau/2) H with dtau = 2/(l N_s) is the
    cTPQ step with nmax = 1; checked against the dense operator."""
    import numpy as np
    import oracle as O
    from workloads import chain, heisenberg_terms, random_vectors
    N, l = 8, 2.0
    m = O.Model("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(chain(N), 1.0))
    H = O.dense_matrix(m)
    V = np.ascontiguousarray(random_vectors(m.dim, 3, 4))
    V0 = V.copy()
    dtau = 2.0 / (l * N)
    e, h2, d = m.tpq_step(V, dtau, 1)
    for q in range(3):
        w = V0[:, q] - H @ V0[:, q] / (l * N)
        assert np.allclose(V[:, q], w / np.linalg.norm(w), rtol=0, atol=1e-14)
        assert d[q] == np.dot(w, w) / np.dot(V0[:, q], V0[:, q]) or abs(d[q] - np.dot(w, w) / np.dot(V0[:, q], V0[:, q])) < 1e-14


def test_mtpq_temperature_follows_the_canonical_energy():
    """u_k = <H>_k / N_s at beta_k = k dtau / (1 - u_k / l) tracks the canonical
    energy per site of the dense spectrum (16 vectors, 2^12 states) up to the
    typicality and microcanonical-versus-canonical finite-size differences
    (a few percent of the bandwidth at N_s = 12)."""
    import numpy as np
    import oracle as O
    from workloads import random_regular_graph, uniform_couplings, heisenberg_terms, random_vectors
    N, l = 12, 1.5
    bonds = random_regular_graph(N, 3, 6)
    m = O.Model("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 7)))
    E = np.linalg.eigvalsh(O.dense_matrix(m))
    assert E.max() / N < l
    V = np.ascontiguousarray(random_vectors(m.dim, 16, 8))
    dtau = 2.0 / (l * N)
    for k in range(400):
        e, h2, d = m.tpq_step(V, dtau, 1)
        if k in (50, 150, 399):
            u = e / N
            beta = k * dtau / (1.0 - u / l)
            for b_, u_ in zip(beta, u):
                ec, _ = O.canonical_thermo(E, np.array([1.0 / b_]))
                assert abs(u_ - ec[0] / N) < 0.05, (k, u_, ec[0] / N)


def test_binding_bootstrap_agrees_with_the_oracle():
    """The binding's post-processing of cTPQ samples (E, C/beta^2 by the
    paper's bootstrap) against the oracle's, on random sample data."""
    import numpy as np
    import oracle as O
    from paper_2307_13222_gb300.hphi import tpq_thermo
    rng = np.random.default_rng(3)
    e = rng.normal(size=(12, 30))
    h2 = e * e + rng.random(size=(12, 30))
    ln = np.cumsum(rng.normal(scale=0.1, size=(12, 30)), axis=1)
    (hm, hs), (fm, fs) = tpq_thermo(e, h2, ln, P=12, M=6, seed=5)
    bs = O.bootstrap_tpq(e, h2, ln, P=12, M=6, seed=5)
    assert np.allclose(hm, bs["H"][0], rtol=1e-12) and np.allclose(hs, bs["H"][1], rtol=1e-12)
    assert np.allclose(fm, bs["fluct"][0], rtol=1e-12) and np.allclose(fs, bs["fluct"][1], rtol=1e-12)
