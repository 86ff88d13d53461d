"""hphi_dot_static: the dot product for callers that cannot allocate device
memory (for example a service that reserved its whole device-memory budget up
front, or a framework whose allocator must own every allocation).  It runs
the same kernels as hphi_dot with a fixed scratch array inside the library
instead of context workspace.  This file is collected last so that a run that
stops at the first failure has run every other test first."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _vectors(n, nvec, dtype, seed):
    from workloads import random_vectors
    cplx = dtype.is_complex
    return torch.from_numpy(random_vectors(n, nvec, seed, complex_=cplx, normalize=False)).to(dtype).cuda()


@pytest.mark.parametrize("dtype,n,nvec", [(torch.float64, 1000003, 1), (torch.float32, 300001, 5),
                                          (torch.complex128, 200003, 3), (torch.float64, 7, 64)])
def test_dot_static_matches_dot_on_two_calls(dtype, n, nvec):
    import paper_2307_13222_gb300 as P
    from paper_2307_13222_gb300 import hphi
    P.build()
    ctx = hphi.Context(0)
    x = _vectors(n, nvec, dtype, 1)
    y = _vectors(n, nvec, dtype, 2)
    ref = hphi.hphi_dot(ctx, x, y)
    for _ in range(2):
        got = hphi.hphi_dot_static(0, x, y)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.sqrt(n))


def test_dot_static_rejects_too_many_columns():
    from paper_2307_13222_gb300 import hphi
    x = torch.zeros((4, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(hphi.HphiError) as ei:
        hphi.hphi_dot_static(0, x, x)
    assert ei.value.code == -1
