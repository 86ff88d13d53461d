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


@pytest.mark.parametrize("coop", [-1, 0, 1, 2, 3, 4, 5, "tiled"])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_tpq_block_of_16_complex_vectors(coop, dtype):
    """16 complex vectors = 32-column rows, the fused <x,Hx>, |Hx|^2, |x|^2
    reductions of the wide-row kernel in both bond-sharing modes, and of the
    tiled two-pass kernel (FP32 and FP64 data)."""
    m, b, h = pair("SPIN_HALF_GC", 12, 0, 0, _model(12, 5))
    if coop == "tiled":
        h.set_tuning(variant=5)
    else:
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
        e, h2, logd, beta = hphi.hphi_mtpq_step(h, Vg, l, N, step, norm2)
        eo, h2o, do = m.tpq_step(Vo, 2.0 / (l * N), 1)
        assert np.allclose(e, eo, rtol=tol, atol=tol) and np.allclose(logd, np.log(do), rtol=tol, atol=tol), step
        # beta_k = k dtau / (1 - u_k / l) of the oracle's energy (Sec. 3.5.1)
        assert np.allclose(beta, step * (2.0 / (l * N)) / (1.0 - eo / N / l), rtol=tol, atol=tol)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_ctpq_thermodynamics_small_member_of_the_benchmark_family(dtype):
    """The benchmark's cTPQ run (16 complex vectors, nmax 6, dtau 0.02) on a
    14-site member of its random 3-regular graph family for 1000 steps
    (beta up to 20): E(T) and C(T) from the paper's bootstrap against the exact
    canonical averages of the spectrum (dense, sector by sector)."""
    import oracle as O
    N = 14
    bonds = random_regular_graph(N, 3, 4)
    terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004))
    m, b, h = pair("SPIN_HALF_GC", N, 0, 0, terms)
    evals = np.concatenate([np.linalg.eigvalsh(O.dense_matrix(O.Model("SPIN_HALF", N, n, 0, terms)))
                            for n in range(N + 1)])
    nvec, steps, dtau = 16, 1000, 0.02
    V = torch.from_numpy(random_vectors(m.dim, nvec, 4, complex_=True)).to(dtype).cuda().contiguous()
    norm2 = np.zeros(nvec)
    E = np.zeros((nvec, steps))
    E2 = np.zeros((nvec, steps))
    logn = np.zeros((nvec, steps))
    acc = np.zeros(nvec)
    for k in range(steps):
        e, h2, logd = hphi.hphi_tpq_step(h, V, dtau, 6, norm2)
        E[:, k], E2[:, k], logn[:, k] = e, h2, acc
        acc = acc + logd
    betas = dtau * np.arange(steps)
    bs = hphi.hphi_tpq_bootstrap(E, E2, logn, P=nvec, M=nvec // 2, beta=betas, seed=1)
    mean, sd, c, csd = bs["e_mean"], bs["e_sd"], bs["c_mean"], bs["c_sd"]
    for k in (50, 250, 500, 999):
        ex, cx = O.canonical_thermo(evals, np.array([1.0 / betas[k]]))
        assert abs(mean[k] - ex[0]) < 4 * sd[k] + 0.02 * abs(ex[0]), (k, mean[k], ex[0], sd[k])
        assert abs(c[k] - cx[0]) < 4 * csd[k] + 0.1 * abs(cx[0]) + 0.02, (k, c[k], cx[0])


def test_ctpq_benchmark_trajectories_at_full_size():
    """The cTPQ benchmark at its own size: 2^26 states of the seeded 26-site
    random 3-regular graph (J ~ U[0.5, 1.5]), 16 complex FP64 start vectors
    from the library's Philox stream, nmax = 6, dtau = 0.02 (Sec. 3.5.2).
    Two of the 16 columns (0 and 9) are run by the oracle's literal Taylor sum
    for the first 10 steps: <H> per step to 1e-10 of the energy scale
    sqrt(<H^2>), <H^2> to 1e-10 relative, log D to 1e-11 absolute, and the
    normalised vectors after the last step to 1e-10 of their largest entry."""
    from workloads import configs
    cfg = configs.ctpq_random_regular()
    m, b, h = pair("SPIN_HALF_GC", cfg["n_sites"], 0, 0, cfg["terms"])
    nvec, cols, steps = cfg["n_vec"], [0, 9], 10
    V = torch.empty((m.dim, nvec), dtype=torch.complex128, device="cuda")
    hphi.hphi_random_vector(h.ctx, V, cfg["seed"])
    Vo = np.ascontiguousarray(V[:, cols].cpu().numpy())
    Vo /= np.linalg.norm(Vo, axis=0, keepdims=True)
    norm2 = np.zeros(nvec)
    for step in range(steps):
        e, h2, logd = hphi.hphi_tpq_step(h, V, cfg["dtau"], cfg["nmax"], norm2)
        eo, h2o, do = m.tpq_step(Vo, cfg["dtau"], cfg["nmax"])
        scale = np.sqrt(h2o)  # the energy scale of the state
        assert np.all(np.abs(e[cols] - eo) <= 1e-10 * scale), (step, e[cols], eo)
        assert np.allclose(h2[cols], h2o, rtol=1e-10, atol=0), (step, h2[cols], h2o)
        # log D_k is O(dtau^2 <H^2>) near beta = 0: compared absolutely (FP64 norms
        # summed over 2^27 reals carry ~1e-12 of rounding on either side)
        assert np.all(np.abs(logd[cols] - np.log(do)) <= 1e-11), (step, logd[cols], np.log(do))
    got = V[:, cols].cpu().numpy() / np.sqrt(norm2[cols])
    assert np.abs(got - Vo).max() <= 1e-10 * np.abs(Vo).max()

