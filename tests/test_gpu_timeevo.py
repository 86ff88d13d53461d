"""GPU real-time evolution step (Sec. 3.4) against the oracle's literal
Taylor sum.

Tolerances: FP64 vectors follow the oracle to 1e-12 relative over 10 steps
(summation order differs, nmax stages each ~1e-16); FP32 (C64) storage
rounds every stage to 2^-24, so 2e-5 after 10 steps."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, square, heisenberg_terms, hubbard_terms, random_regular_graph, uniform_couplings, \
    random_vectors

pytestmark = pytest.mark.gpu

CASES = {
    "sector": ("SPIN_HALF", 12, 6, 0, lambda: heisenberg_terms(chain(12), 1.0)),
    "full": ("SPIN_HALF_GC", 12, 0, 0, lambda: heisenberg_terms(random_regular_graph(12, 3, 5),
                                                               uniform_couplings(18, 0.5, 1.5, 8))),
    "hubbard": ("HUBBARD", 6, 3, 2, lambda: hubbard_terms(6, chain(6), t=1.0, U=4.0)),
}


def _start(dim, nvec, seed):
    V = random_vectors(dim, nvec, seed, complex_=True)
    return np.ascontiguousarray(V / np.linalg.norm(V, axis=0))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("nvec,nmax", [(1, 10), (3, 4), (16, 6), (2, 1)])
def test_steps_match_oracle(case, dtype, nvec, nmax):
    model, N, nu, nd, terms = CASES[case]
    m, b, h = pair(model, N, nu, nd, terms())
    V0 = _start(m.dim, nvec, 40 + nvec)
    Vg = torch.from_numpy(V0).to(dtype).cuda().contiguous()
    Vo = Vg.cpu().numpy().astype(np.complex128).copy()
    tol = 1e-12 if dtype == torch.complex128 else 2e-5
    for step in range(10):
        n2, e, h2, n2n = hphi.hphi_time_step(h, Vg, 0.03, nmax)
        on2, oe, on2n = m.time_step(Vo, 0.03, nmax)
        assert np.allclose(n2, on2, rtol=tol), step
        assert np.allclose(e, oe, rtol=tol, atol=tol), step
        assert np.allclose(n2n, on2n, rtol=tol), step
    assert np.abs(Vg.cpu().numpy() - Vo).max() < 10 * tol


def test_h2_output_and_padded_columns():
    """<H Phi|H Phi> of the step and a leading dimension wider than nvec."""
    m, b, h = pair("SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0))
    H = O.dense_matrix(m)
    V0 = _start(m.dim, 2, 3)
    big = torch.zeros((m.dim, 5), dtype=torch.complex128, device="cuda")
    big[:, 1:3] = torch.from_numpy(V0)
    n2, e, h2, n2n = hphi.hphi_time_step(h, big[:, 1:3], 0.02, 8)
    for q in range(2):
        assert h2[q] == pytest.approx(np.linalg.norm(H @ V0[:, q]) ** 2, rel=1e-12)
    assert (big[:, [0, 3, 4]] == 0).all()


def test_two_site_rabi_closed_form():
    J = 1.7
    m, b, h = pair("SPIN_HALF", 2, 1, 0, [("EXCHANGE", 0, 1, 0, J, 0.0)])
    V = torch.zeros(2, dtype=torch.complex128, device="cuda")
    r0, r1 = m.state_row(0b01), m.state_row(0b10)
    V[r0] = 1.0
    for _ in range(300):
        hphi.hphi_time_step(h, V, 0.01, 10)
    t = 3.0
    a = V.cpu().numpy()
    assert abs(a[r0] - np.exp(1j * J * t / 4) * np.cos(J * t / 2)) < 1e-12
    assert abs(abs(a[r1]) ** 2 - np.sin(J * t / 2) ** 2) < 1e-12


def test_hubbard_quench_pipeline():
    """U = 0 ground state of the half-filled 10-site ring (GPU Lanczos), then
    U = 8 evolution: d(0) = 1/4, energy and norm conserved, d(t) as the
    oracle's own evolution from its own ground state."""
    N = 10
    m0, b0, h0 = pair("HUBBARD", N, 5, 5, hubbard_terms(N, chain(N), t=1.0, U=0.0))
    mq, bq, hq = pair("HUBBARD", N, 5, 5, hubbard_terms(N, chain(N), t=1.0, U=8.0))
    md, bd, hd = pair("HUBBARD", N, 5, 5, [("HUBBARD_U", i, i, 0, 1.0 / N, 0.0) for i in range(N)])
    v0 = torch.empty(m0.dim, dtype=torch.float64, device="cuda")
    hphi.hphi_random_vector(b0.ctx, v0, 5)
    gs = torch.empty_like(v0)
    r = hphi.hphi_lanczos(h0, v0, 300, 1e-12, gs_out=gs)
    assert r["converged"]
    V = gs.to(torch.complex128).contiguous()
    HV = torch.empty_like(V)

    def d_gpu():
        hphi.hphi_apply_H(hd, V, HV)
        return float(torch.vdot(V, HV).real)

    og = m0.lanczos(random_vectors(m0.dim, 1, 5).reshape(-1), 300, 1e-12, want_gs=True)["gs"]
    Vo = og.astype(np.complex128)[:, None].copy()

    def d_orc():
        x = Vo[:, 0]
        y = md.apply(np.ascontiguousarray(x.real)) + 1j * md.apply(np.ascontiguousarray(x.imag))
        return float(np.vdot(x, y).real)

    assert d_gpu() == pytest.approx(0.25, abs=1e-9)
    assert d_orc() == pytest.approx(0.25, abs=1e-9)
    e_first = None
    for step in range(60):
        n2, e, h2, n2n = hphi.hphi_time_step(hq, V, 0.01, 10)
        mq.time_step(Vo, 0.01, 10)
        e_first = e[0] if e_first is None else e_first
        assert abs(e[0] - e_first) < 1e-9 and abs(n2n[0] - 1.0) < 1e-9
        if step % 20 == 19:
            assert d_gpu() == pytest.approx(d_orc(), abs=1e-8)
    assert d_gpu() < 0.25


def test_full_size_conservation():
    """4x4 Hubbard at half filling (165,636,900 rows, one C128 vector) and the
    N=26 full space with 16 C64 vectors: the step's norms agree with an
    independent norm and stay unitary to the truncation bound; its energy
    agrees with <Phi|H|Phi> through the H*x entry point."""
    m, b, h = pair("HUBBARD", 16, 8, 8, hubbard_terms(16, square(4, 4), t=1.0, U=8.0))
    V = torch.empty(m.dim, dtype=torch.complex128, device="cuda")
    hphi.hphi_random_vector(b.ctx, V, 12)
    V /= torch.linalg.vector_norm(V)
    HV = torch.empty_like(V)
    hphi.hphi_apply_H(h, V, HV)
    e_ref = float(torch.vdot(V, HV).real)
    del HV
    n2, e, h2, n2n = hphi.hphi_time_step(h, V, 0.01, 10)
    assert n2[0] == pytest.approx(1.0, abs=1e-12)
    assert e[0] == pytest.approx(e_ref, rel=1e-12, abs=1e-12)
    assert n2n[0] == pytest.approx(1.0, abs=1e-9)  # truncation: ~2 (|H| dt)^12 / 11!
    assert n2n[0] == pytest.approx(float(torch.vdot(V, V).real), rel=1e-13)
    del V
    torch.cuda.empty_cache()
    bonds = random_regular_graph(26, 3, 4)
    m, b, h = pair("SPIN_HALF_GC", 26, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004)))
    V = torch.empty((m.dim, 16), dtype=torch.complex64, device="cuda")
    hphi.hphi_random_vector(b.ctx, V, 13)
    n2, e, h2, n2n = hphi.hphi_time_step(h, V, 0.02, 6)
    nn = torch.linalg.vector_norm(V.to(torch.complex128), dim=0).cpu().numpy() ** 2
    assert np.allclose(n2n, nn, rtol=1e-5)
    assert np.allclose(n2n, n2, rtol=1e-5)
    del V
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N", [12, 20])
def test_tiled_block_kernel_pair_swap(N):
    """16 complex C64 columns through the tiled two-pass kernel: the pair swap
    of the real-time step (multiplication by -i dt / j) in its second pass."""
    bonds = random_regular_graph(N, 3, 5)
    m, b, h = pair("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 8)))
    h.set_tuning(variant=5)
    V0 = _start(m.dim, 16, 77)
    Vg = torch.from_numpy(V0).to(torch.complex64).cuda().contiguous()
    Vo = Vg.cpu().numpy().astype(np.complex128).copy()
    for step in range(3 if N <= 12 else 1):
        n2, e, h2, n2n = hphi.hphi_time_step(h, Vg, 0.03, 6)
        on2, oe, on2n = m.time_step(Vo, 0.03, 6)
        assert np.allclose(n2, on2, rtol=2e-5) and np.allclose(e, oe, rtol=2e-5, atol=2e-5), step
    assert h.ctx.last_kernel().startswith("k_tile<f32,")
    assert np.abs(Vg.cpu().numpy() - Vo).max() < 2e-4
