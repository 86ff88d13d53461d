"""GPU vector kernels: dot / nrm2 / axpy / scal / random start vectors."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, rel_err
from paper_2307_13222_gb300 import hphi
from workloads import philox_gaussian, random_vectors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex128, torch.complex64])
@pytest.mark.parametrize("n,nvec", [(1, 1), (1000, 1), (100003, 3), (50000, 16), (7777, 40)])
def test_dot_nrm2(dtype, n, nvec):
    c = ctx()
    cplx = dtype.is_complex
    x = torch.from_numpy(random_vectors(n, nvec, 1, complex_=cplx, normalize=False)).to(dtype).cuda()
    y = torch.from_numpy(random_vectors(n, nvec, 2, complex_=cplx, normalize=False)).to(dtype).cuda()
    xd = x.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    yd = y.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    got = hphi.hphi_dot(c, x, y)
    want = (np.conj(xd) * yd).sum(axis=0)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.sqrt(n))
    nr = hphi.hphi_nrm2(c, x)
    assert np.allclose(nr, np.linalg.norm(xd, axis=0), rtol=1e-13)
    # bitwise reproducible
    assert np.array_equal(hphi.hphi_dot(c, x, y), got)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex128])
def test_axpy_scal(dtype):
    c = ctx()
    cplx = dtype.is_complex
    n, nvec = 30001, 5
    x = torch.from_numpy(random_vectors(n, nvec, 3, complex_=cplx, normalize=False)).to(dtype).cuda()
    y = torch.from_numpy(random_vectors(n, nvec, 4, complex_=cplx, normalize=False)).to(dtype).cuda()
    a = (np.arange(nvec) + 0.5) * (1 - 0.7j if cplx else 1.0)
    want = y.cpu().numpy() + a * x.cpu().numpy()
    hphi.hphi_axpy(c, a, x, y)
    assert rel_err(y.cpu().numpy(), want) < (1e-15 if dtype != torch.float32 else 1e-6)
    want2 = a * x.cpu().numpy()
    hphi.hphi_scal(c, a, x)
    assert rel_err(x.cpu().numpy(), want2) < (1e-15 if dtype != torch.float32 else 1e-6)


def test_random_vector_matches_host_philox():
    c = ctx()
    for n, nvec, seed in ((5000, 1, 7), (1000, 3, 123456789012), (333, 2, 0)):
        x = torch.empty((n, nvec), dtype=torch.float64, device="cuda")
        hphi.hphi_random_vector(c, x, seed)
        want = philox_gaussian(0, n * nvec, seed).reshape(n, nvec)
        assert np.allclose(x.cpu().numpy(), want, rtol=1e-13, atol=1e-13)
    xc = torch.empty((100, 2), dtype=torch.complex128, device="cuda")
    hphi.hphi_random_vector(c, xc, 5)
    want = philox_gaussian(0, 400, 5).reshape(100, 4)
    got = torch.view_as_real(xc).reshape(100, 4).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_empty_vectors():
    c = ctx()
    x = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    assert (hphi.hphi_dot(c, x, x) == 0).all()


@pytest.mark.parametrize("dtype,nvec", [(torch.float32, 4), (torch.float32, 32), (torch.float64, 2),
                                        (torch.float64, 16), (torch.complex64, 2), (torch.complex64, 16),
                                        (torch.complex128, 8)])
def test_axpy_scal_contiguous_rows(dtype, nvec):
    """Rows of several contiguous columns whose width divides the 16-byte vector
    stride take the flat kernel (complex scaling uses the pair term in place)."""
    c = ctx()
    cplx = dtype.is_complex
    n = 40001
    x = torch.from_numpy(random_vectors(n, nvec, 5, complex_=cplx, normalize=False)).to(dtype).cuda()
    y = torch.from_numpy(random_vectors(n, nvec, 6, complex_=cplx, normalize=False)).to(dtype).cuda()
    a = (np.arange(nvec) - 1.5) * (0.3 + 0.8j if cplx else 1.0)
    want = y.cpu().numpy() + a * x.cpu().numpy()
    hphi.hphi_axpy(c, a, x, y)
    assert rel_err(y.cpu().numpy(), want) < (1e-15 if dtype in (torch.float64, torch.complex128) else 1e-6)
    want2 = a * x.cpu().numpy()
    hphi.hphi_scal(c, a, x)
    assert rel_err(x.cpu().numpy(), want2) < (1e-15 if dtype in (torch.float64, torch.complex128) else 1e-6)
