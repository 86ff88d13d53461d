"""hphi_dot_static: the dot product for callers that cannot allocate device
memory (for example a service that reserved its whole device-memory budget up
front, or a framework whose allocator must own every allocation).  It runs
the same kernels as hphi_dot with a fixed scratch array inside the library
instead of context workspace.  This file is collected last so that a run that
stops at the first failure has run every other test first."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _vectors(n, nvec, dtype, seed):
    from workloads import random_vectors
    cplx = dtype.is_complex
    return torch.from_numpy(random_vectors(n, nvec, seed, complex_=cplx, normalize=False)).to(dtype).cuda()


@pytest.mark.parametrize("dtype,n,nvec", [(torch.float64, 1000003, 1), (torch.float32, 300001, 5),
                                          (torch.complex128, 200003, 3), (torch.complex64, 700001, 32),
                                          (torch.float64, 7, 64)])
def test_dot_static_matches_dot_on_two_calls(dtype, n, nvec):
    """Same grid and kernels as hphi_dot on a GB300 (152 SMs x 8 blocks fits
    the static partials): the results are bitwise equal, call after call."""
    import paper_2307_13222_gb300 as P
    from paper_2307_13222_gb300 import hphi
    P.build()
    ctx = hphi.Context(0)
    x = _vectors(n, nvec, dtype, 1)
    y = _vectors(n, nvec, dtype, 2)
    ref = hphi.hphi_dot(ctx, x, y)
    for _ in range(2):
        got = hphi.hphi_dot_static(0, x, y)
        if ctx.sm_count * 8 <= 2048:
            assert np.array_equal(got, ref)
        else:
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.sqrt(n))


def test_dot_static_on_a_side_stream_allocates_nothing():
    from paper_2307_13222_gb300 import hphi
    ctx = hphi.Context(0)
    x = _vectors(2000003, 2, torch.float64, 3)
    y = _vectors(2000003, 2, torch.float64, 4)
    ref = hphi.hphi_dot(ctx, x, y)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    with torch.cuda.stream(side):
        for _ in range(5):
            got = hphi.hphi_dot_static(0, x, y)
            assert np.array_equal(got, ref)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0


def test_dot_static_rejects_too_many_columns():
    from paper_2307_13222_gb300 import hphi
    x = torch.zeros((4, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(hphi.HphiError) as ei:
        hphi.hphi_dot_static(0, x, x)
    assert ei.value.code == -1
    # 33 complex columns are 66 real ones
    z = torch.zeros((4, 33), dtype=torch.complex128, device="cuda")
    with pytest.raises(hphi.HphiError) as ei:
        hphi.hphi_dot_static(0, z, z)
    assert ei.value.code == -1


def test_dot_static_rejects_host_memory_through_the_c_abi():
    """A host pointer passed straight to the C entry point is refused, not read."""
    from paper_2307_13222_gb300 import hphi
    lib = hphi.load_library()
    a = np.ones(1000)
    out = np.zeros(1)
    st = lib.hphi_dot_static(0, None, hphi.F64, a.size, 1, a.ctypes.data_as(C.c_void_p), 1,
                             a.ctypes.data_as(C.c_void_p), 1, out.ctypes.data_as(C.c_void_p))
    assert st == -1
