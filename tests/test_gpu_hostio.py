"""hphi_apply_H_host: H*x on a batch of host vectors with the copies
overlapping the products.  Its results must be bit-identical to
hphi_apply_H on the same inputs (the same kernels run), for one, two and
several vectors, real and complex, pinned and pageable host memory."""
import numpy as np
import pytest
import torch

from gpu_util import pair, rel_err
from paper_2307_13222_gb300 import hphi
from workloads import square, heisenberg_terms, random_vectors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,nvec", [(torch.float64, 1), (torch.float32, 1), (torch.complex64, 2),
                                        (torch.float64, 3)])
@pytest.mark.parametrize("nbatch", [1, 2, 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_batch_matches_device_apply(dtype, nvec, nbatch, pinned):
    m, b, h = pair("SPIN_HALF", 16, 8, 0, heisenberg_terms(square(4, 4), 1.0))
    shape = (nbatch, m.dim) if nvec == 1 else (nbatch, m.dim, nvec)
    arr = random_vectors(m.dim, nbatch * nvec, 7 + nbatch, complex_=dtype.is_complex, normalize=False)
    arr = arr.reshape(m.dim, nbatch * nvec)
    xh = torch.from_numpy(np.stack([arr[:, k * nvec:(k + 1) * nvec] for k in range(nbatch)]))
    xh = xh.to(dtype).reshape(shape).contiguous()
    if pinned:
        xh = xh.pin_memory()
    yh = torch.empty(shape, dtype=dtype, pin_memory=pinned)
    hphi.hphi_apply_H_host(h, xh, yh, 0.7)
    for k in range(nbatch):
        xd = xh[k].cuda()
        yd = torch.empty_like(xd)
        hphi.hphi_apply_H(h, xd, yd, 0.7)
        assert torch.equal(yd.cpu(), yh[k])
    # and against the oracle for the first vector
    x0 = xh[0].numpy().astype(np.complex128 if dtype.is_complex else np.float64).reshape(m.dim, nvec)
    for c in range(nvec):
        want = 0.7 * (m.apply(np.ascontiguousarray(x0[:, c].real)) + 1j * m.apply(np.ascontiguousarray(x0[:, c].imag))
                      if dtype.is_complex else m.apply(np.ascontiguousarray(x0[:, c])))
        got = yh[0].numpy().reshape(m.dim, nvec)[:, c]
        assert rel_err(got, want) < (1e-13 if dtype == torch.float64 else 2e-6)


def test_host_batch_edge_cases():
    m, b, h = pair("SPIN_HALF", 12, 6, 0, heisenberg_terms(square(4, 3), 1.0))
    x = torch.zeros((0, m.dim), dtype=torch.float64)
    hphi.hphi_apply_H_host(h, x, torch.zeros_like(x))  # empty batch
    x = torch.ones((2, m.dim), dtype=torch.float64)
    with pytest.raises(ValueError):
        hphi.hphi_apply_H_host(h, x, torch.zeros((2, m.dim), dtype=torch.float32))
    with pytest.raises(ValueError):
        hphi.hphi_apply_H_host(h, x.cuda(), x.cuda())
    with pytest.raises(hphi.HphiError):  # x and y the same memory
        hphi.hphi_apply_H_host(h, x, x)
