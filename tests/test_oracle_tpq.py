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


def _two_sample_set():
    """Two samples at one temperature: weights 1 and 3 (log norms 0, log 3),
    <H> = 1, 2 and <H^2> = 2, 5."""
    num_h = np.array([[1.0], [2.0]])
    num_h2 = np.array([[2.0], [5.0]])
    logn = np.array([[0.0], [math.log(3.0)]])
    return num_h, num_h2, logn


def test_bootstrap_sigma_over_every_resampling_by_hand():
    """All four ordered resamplings of P = 2 from N = 2 (with replacement),
    passed explicitly.  Per resampling <H>_m = sum w H / sum w:
      (0,0): 1,  (0,1), (1,0): (1 + 3*2)/4 = 7/4,  (1,1): 2;
    mean 13/8, squared deviations 25/64, 1/64, 1/64, 9/64 (sum 9/16), so
    sigma^2 = (9/16)/(M-1) = 3/16 (a 1/M divisor gives 9/64).
    <H^2>_m: 2, 17/4, 17/4, 5;  fluctuation <H^2>_m - <H>_m^2: 1, 19/16, 19/16, 1;
    mean 35/32, squared deviations 4 x 9/1024, sigma^2 = (36/1024)/3 = 3/256."""
    num_h, num_h2, logn = _two_sample_set()
    picks = np.array([[0, 0], [0, 1], [1, 0], [1, 1]])
    bs = O.bootstrap_tpq(num_h, num_h2, logn, P=2, M=4, picks=picks)
    mean, sd = bs["H"]
    assert mean[0] == pytest.approx(13 / 8, rel=1e-15)
    assert sd[0] == pytest.approx(math.sqrt(3 / 16), rel=1e-14)
    assert sd[0] != pytest.approx(math.sqrt(9 / 64), rel=1e-3)
    fm, fsd = bs["fluct"]
    assert fm[0] == pytest.approx(35 / 32, rel=1e-15)
    assert fsd[0] == pytest.approx(math.sqrt(3 / 256), rel=1e-13)
    h2m, h2sd = bs["H2"]
    assert h2m[0] == pytest.approx((2 + 17 / 4 + 17 / 4 + 5) / 4, rel=1e-15)


def test_bootstrap_sample_zero_normalisation_cancels():
    """Dividing every norm by sample 0's (the paper's W) changes nothing:
    shifting all log norms of a temperature by a constant leaves the result."""
    num_h, num_h2, logn = _two_sample_set()
    picks = np.array([[0, 1], [1, 1], [0, 0]])
    a = O.bootstrap_tpq(num_h, num_h2, logn, P=2, M=3, picks=picks)
    b = O.bootstrap_tpq(num_h, num_h2, logn + 40.0, P=2, M=3, picks=picks)
    for k in ("H", "H2", "fluct"):
        assert np.allclose(a[k][0], b[k][0], rtol=1e-14) and np.allclose(a[k][1], b[k][1], rtol=1e-12)


def test_bootstrap_draws_are_uniform_with_replacement():
    """The seeded resamplings draw with replacement: for N = P = 2 half of the
    resamplings repeat an index (none would without replacement), and every
    index is equally likely."""
    from workloads import bootstrap_picks
    M = 20000
    picks = bootstrap_picks(M, 2, 2, seed=7)
    rep = np.mean(picks[:, 0] == picks[:, 1])
    assert abs(rep - 0.5) < 4 * math.sqrt(0.25 / M)
    p10 = bootstrap_picks(4000, 25, 10, seed=8)
    counts = np.bincount(p10.reshape(-1), minlength=10)
    n = p10.size
    assert p10.min() == 0 and p10.max() == 9
    assert np.all(np.abs(counts / n - 0.1) < 4 * math.sqrt(0.09 / n))
    # the seeded path of the oracle uses exactly these picks
    num_h, num_h2, logn = _two_sample_set()
    a = O.bootstrap_tpq(num_h, num_h2, logn, P=2, M=50, seed=3)
    b = O.bootstrap_tpq(num_h, num_h2, logn, P=2, M=50, picks=bootstrap_picks(50, 2, 2, 3))
    assert np.array_equal(a["H"][1], b["H"][1])
