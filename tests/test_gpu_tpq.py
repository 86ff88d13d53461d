"""GPU canonical-TPQ step (Horner) against the oracle's literal Taylor sum."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, heisenberg_terms, random_regular_graph, uniform_couplings, random_vectors

pytestmark = pytest.mark.gpu


def _model(N=10, seed=3):
    bonds = random_regular_graph(N, 3, seed)
    return heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, seed + 1000))


@pytest.mark.parametrize("dtype,nvec,nmax", [(torch.float64, 3, 6), (torch.complex128, 4, 6), (torch.float64, 2, 1),
                                             (torch.complex128, 16, 6), (torch.float32, 3, 6),
                                             (torch.complex64, 2, 3)])
def test_tpq_steps_match_oracle(dtype, nvec, nmax):
    m, b, h = pair("SPIN_HALF_GC", 10, 0, 0, _model())
    cplx = dtype.is_complex
    V0 = random_vectors(m.dim, nvec, 17, complex_=cplx)
    Vg = torch.from_numpy(V0).to(dtype).cuda().contiguous()
    Vo = Vg.cpu().numpy().astype(np.complex128 if cplx else np.float64).copy()
    norm2 = np.zeros(nvec)
    tol = 1e-11 if dtype in (torch.float64, torch.complex128) else 2e-5
    for step in range(25):
        e, h2, logd = hphi.hphi_tpq_step(h, Vg, 0.02, nmax, norm2)
        eo, h2o, do = m.tpq_step(Vo, 0.02, nmax)
        assert np.allclose(e, eo, rtol=tol, atol=tol), (step, e, eo)
        assert np.allclose(h2, h2o, rtol=tol), step
        assert np.allclose(logd, np.log(do), rtol=tol, atol=tol), step
    got = Vg.cpu().numpy() / np.sqrt(norm2)
    assert np.abs(got - Vo).max() < 50 * tol


def test_tpq_sector_model():
    m, b, h = pair("SPIN_HALF", 12, 6, 0, heisenberg_terms(chain(12), 1.0))
    V0 = random_vectors(m.dim, 2, 3)
    Vg = torch.from_numpy(V0).cuda().contiguous()
    Vo = V0.copy()
    norm2 = np.zeros(2)
    for _ in range(10):
        e, h2, logd = hphi.hphi_tpq_step(h, Vg, 0.05, 6, norm2)
        eo, h2o, do = m.tpq_step(Vo, 0.05, 6)
    assert np.allclose(e, eo, rtol=1e-12) and np.allclose(logd, np.log(do), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("coop", [-1, 0, 1])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_tpq_block_of_16_complex_vectors(coop, dtype):
    """16 complex vectors = 32-column rows, the fused <x,Hx>, |Hx|^2, |x|^2
    reductions of the wide-row kernel in both bond-sharing modes."""
    m, b, h = pair("SPIN_HALF_GC", 12, 0, 0, _model(12, 5))
    h.set_tuning(variant=1, coop=coop)
    V0 = random_vectors(m.dim, 16, 23, complex_=True)
    Vg = torch.from_numpy(V0).to(dtype).cuda().contiguous()
    Vo = Vg.cpu().numpy().astype(np.complex128).copy()
    norm2 = np.zeros(16)
    tol = 1e-11 if dtype == torch.complex128 else 2e-5
    for step in range(12):
        e, h2, logd = hphi.hphi_tpq_step(h, Vg, 0.05, 6, norm2)
        eo, h2o, do = m.tpq_step(Vo, 0.05, 6)
        assert np.allclose(e, eo, rtol=tol, atol=tol), (step, e, eo)
        assert np.allclose(h2, h2o, rtol=tol), step
        assert np.allclose(logd, np.log(do), rtol=tol, atol=tol), step


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex64])
def test_mtpq_steps_match_oracle(dtype):
    """mTPQ step = cTPQ step with nmax = 1 and dtau = 2 / (l N_s)."""
    N, l = 10, 1.8
    m, b, h = pair("SPIN_HALF_GC", N, 0, 0, _model(N, 4))
    cplx = dtype.is_complex
    V0 = random_vectors(m.dim, 4, 31, complex_=cplx)
    Vg = torch.from_numpy(V0).to(dtype).cuda().contiguous()
    Vo = Vg.cpu().numpy().astype(np.complex128 if cplx else np.float64).copy()
    norm2 = np.zeros(4)
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    for step in range(20):
        e, h2, logd = hphi.hphi_mtpq_step(h, Vg, l, N, norm2)
        eo, h2o, do = m.tpq_step(Vo, 2.0 / (l * N), 1)
        assert np.allclose(e, eo, rtol=tol, atol=tol) and np.allclose(logd, np.log(do), rtol=tol, atol=tol), step
        beta = hphi.mtpq_beta(step, l, N, e)
        assert np.allclose(beta, step * (2.0 / (l * N)) / (1.0 - eo / N / l), rtol=tol, atol=tol)
