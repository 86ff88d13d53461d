"""Pins of the real-time evolution oracle (Sec. 3.4): Phi(t + dt) =
sum_{n<=nmax} (-i dt H)^n / n! Phi(t).

Against scipy's matrix exponential within the Taylor remainder bound, the
two-site Rabi oscillation in closed form, norm and energy conservation, and
the interaction quench of the Hubbard chain (the paper's example) whose
initial double occupancy is 1/4 exactly."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from workloads import chain, heisenberg_terms, hubbard_terms, random_vectors


def _cvec(dim, seed):
    v = random_vectors(dim, 1, seed, complex_=True).reshape(-1)
    return np.ascontiguousarray(v / np.linalg.norm(v))


@pytest.mark.parametrize("model,N,nu,nd", [("SPIN_HALF", 8, 4, 0), ("SPIN_HALF_GC", 6, 0, 0), ("HUBBARD", 4, 2, 2)])
@pytest.mark.parametrize("nmax", [1, 4, 10])
def test_step_matches_expm_within_remainder(model, N, nu, nd, nmax):
    terms = hubbard_terms(N, chain(N), t=1.0, U=3.0) if model == "HUBBARD" else heisenberg_terms(chain(N), 1.0)
    m = O.Model(model, N, nu, nd, terms)
    H = O.dense_matrix(m)
    dt = 0.05
    V = np.ascontiguousarray(np.stack([_cvec(m.dim, 3), _cvec(m.dim, 4)], axis=1))
    V0 = V.copy()
    n2, e, n2n = m.time_step(V, dt, nmax)
    U = sla.expm(-1j * dt * H)
    hn = np.linalg.norm(H, 2)
    bound = (hn * dt) ** (nmax + 1) / math.factorial(nmax + 1) * math.exp(hn * dt)
    for q in range(2):
        assert np.linalg.norm(V[:, q] - U @ V0[:, q]) <= bound + 1e-14
        assert n2[q] == pytest.approx(1.0, abs=1e-14)
        assert e[q] == pytest.approx(np.vdot(V0[:, q], H @ V0[:, q]).real, abs=1e-13)
        assert n2n[q] == pytest.approx(np.vdot(V[:, q], V[:, q]).real, rel=1e-14)


def test_two_site_rabi_oscillation():
    """H = -J/4 + (J/2) sigma_x on {|up dn>, |dn up>}: from |up dn>,
    <up dn|Phi(t)> = e^{i J t/4} cos(J t / 2)."""
    J = 1.7
    m = O.Model("SPIN_HALF", 2, 1, 0, [("EXCHANGE", 0, 1, 0, J, 0.0)])
    V = np.zeros((2, 1), dtype=np.complex128)
    V[m.state_row(0b01), 0] = 1.0
    dt, K = 0.01, 300
    for k in range(K):
        m.time_step(V, dt, 10)
    t = dt * K
    a = V[m.state_row(0b01), 0]
    assert abs(a - np.exp(1j * J * t / 4) * np.cos(J * t / 2)) < 1e-12
    assert abs(abs(V[m.state_row(0b10), 0]) ** 2 - np.sin(J * t / 2) ** 2) < 1e-12


def test_norm_and_energy_conservation_improve_with_nmax():
    m = O.Model("SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0))
    drift = {}
    for nmax in (2, 4, 8):
        V = _cvec(m.dim, 5)[:, None].copy()
        n2, e0, _ = m.time_step(V.copy(), 0.05, nmax)
        for k in range(40):
            n2, e, n2n = m.time_step(V, 0.05, nmax)
        drift[nmax] = (abs(n2n[0] - 1.0), abs(e[0] - e0[0]))
    assert drift[8][0] < 1e-12 and drift[8][1] < 1e-11
    assert drift[2][0] > drift[4][0] > drift[8][0]


def test_hubbard_quench_double_occupancy():
    """U = 0 ground state of the half-filled 6-site ring (closed shell, unique),
    then evolution with U = 8: d(0) = 1/4, E and the norm are conserved, and
    d(t) follows the exact exponential."""
    N = 6
    m0 = O.Model("HUBBARD", N, 3, 3, hubbard_terms(N, chain(N), t=1.0, U=0.0))
    E0, U0 = np.linalg.eigh(O.dense_matrix(m0))
    assert E0[1] - E0[0] > 1e-6
    mq = O.Model("HUBBARD", N, 3, 3, hubbard_terms(N, chain(N), t=1.0, U=8.0))
    docc = O.Model("HUBBARD", N, 3, 3, [("HUBBARD_U", i, i, 0, 1.0 / N, 0.0) for i in range(N)])
    Hq = O.dense_matrix(mq)
    V = U0[:, :1].astype(np.complex128).copy()

    def d_of(v):
        return (np.vdot(v, docc.apply(np.ascontiguousarray(v.real)) + 1j * docc.apply(np.ascontiguousarray(v.imag)))).real

    assert d_of(V[:, 0]) == pytest.approx(0.25, abs=1e-13)
    dt, K = 0.01, 100
    _, e_start, _ = m_e = mq.time_step(V.copy(), dt, 10)
    for k in range(K):
        n2, e, n2n = mq.time_step(V, dt, 10)
    assert abs(e[0] - e_start[0]) < 1e-11 and abs(n2n[0] - 1.0) < 1e-12
    exact = sla.expm(-1j * dt * K * Hq) @ U0[:, 0]
    assert np.linalg.norm(V[:, 0] - exact) < 1e-11
    assert d_of(V[:, 0]) == pytest.approx(d_of(exact), abs=1e-12)
    assert d_of(V[:, 0]) < 0.25  # the repulsive quench removes double occupancy
