"""GPU H*x against the oracle, element by element.

Tolerances: FP64 results agree with the oracle's FP64 sums to a few ulps of
the row magnitude (different summation order): 1e-13 relative to max|y|.
FP32 storage/arithmetic: the inputs are rounded to FP32 (2^-24) and each row
sums <= ~70 terms, so 2e-6 relative to max|y|."""
import itertools
import random

import numpy as np
import pytest
import torch

from gpu_util import pair, rel_err
from paper_2307_13222_gb300 import hphi
from workloads import (chain, square, heisenberg_terms, hubbard_terms, random_regular_graph, uniform_couplings,
                       random_vectors)

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-13, torch.float32: 2e-6, torch.complex128: 1e-13, torch.complex64: 2e-6}


def _check(m, h, dtype, nvec, alpha=1.0, beta=0.0, ld_pad=0, seed=0):
    cplx = dtype in (torch.complex128, torch.complex64)
    x = random_vectors(m.dim, nvec, seed + 11, complex_=cplx, normalize=False)
    y0 = random_vectors(m.dim, nvec, seed + 12, complex_=cplx, normalize=False)
    ld = nvec + ld_pad
    xd = torch.zeros((m.dim, ld), dtype=dtype, device="cuda")
    yd = torch.zeros((m.dim, ld), dtype=dtype, device="cuda")
    xd[:, :nvec] = torch.from_numpy(x).to(dtype)
    yd[:, :nvec] = torch.from_numpy(y0).to(dtype)
    xs, ys = xd[:, :nvec], yd[:, :nvec]
    hphi.hphi_apply_H(h, xs, ys, alpha, beta)
    # oracle on the same (rounded) inputs
    xr = xs.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    yr0 = torch.from_numpy(y0).to(dtype).numpy().astype(np.complex128 if cplx else np.float64)
    if cplx:
        want = np.empty_like(xr)
        want.real = m.apply(np.ascontiguousarray(xr.real), alpha, beta, np.ascontiguousarray(yr0.real))
        want.imag = m.apply(np.ascontiguousarray(xr.imag), alpha, beta, np.ascontiguousarray(yr0.imag))
    else:
        want = m.apply(xr, alpha, beta, yr0.copy())
    got = ys.cpu().numpy()
    assert rel_err(got, want) < TOL[dtype], (dtype, nvec, rel_err(got, want))
    if ld_pad:  # padding columns untouched
        assert (yd[:, nvec:] == 0).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nvec", [1, 2, 3, 8, 32, 33])
def test_spin_chain_sector(dtype, nvec):
    m, b, h = pair("SPIN_HALF", 14, 7, 0, heisenberg_terms(chain(14), 1.0))
    _check(m, h, dtype, nvec, alpha=0.7, beta=-0.3 if nvec % 2 else 0.0, seed=nvec)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex128, torch.complex64])
def test_random_xxz_sector(dtype):
    rng = random.Random(5)
    N = 15
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), 40)
    terms = [("XXZ", i, j, 0, rng.uniform(-1, 2), rng.uniform(-1, 2)) for i, j in pairs]
    m, b, h = pair("SPIN_HALF", N, 6, 0, terms)
    _check(m, h, dtype, 2, alpha=1.3, beta=0.5, ld_pad=3, seed=2)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nvec", [1, 4, 16])
def test_full_space_random_graph(dtype, nvec):
    bonds = random_regular_graph(14, 3, 9)
    terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 10))
    m, b, h = pair("SPIN_HALF_GC", 14, 0, 0, terms)
    _check(m, h, dtype, nvec, seed=3)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex128])
@pytest.mark.parametrize("geom", ["chain8", "square3x3", "random"])
def test_hubbard(dtype, geom):
    if geom == "chain8":
        N, terms = 8, hubbard_terms(8, chain(8), t=1.0, U=4.0)
        nu, nd = 4, 3
    elif geom == "square3x3":
        N, terms = 9, hubbard_terms(9, square(3, 3), t=0.8, U=6.0, V=0.5)
        nu, nd = 4, 5
    else:
        rng = random.Random(7)
        N = 8
        terms = [("HOP", j, i, rng.choice([-1, 0, 1]), rng.uniform(-1, 1), 0.0)
                 for i, j in rng.sample(list(itertools.combinations(range(N), 2)), 12)]
        terms += [("HUBBARD_U", i, i, 0, rng.uniform(0, 5), 0.0) for i in range(N)]
        terms += [("DENS_DENS", 1, 6, 0, -0.4, 0.0)]
        nu, nd = 3, 4
    m, b, h = pair("HUBBARD", N, nu, nd, terms)
    _check(m, h, dtype, 1, alpha=-0.9, beta=0.25, seed=4)


def test_edge_cases():
    # one-state sectors, no terms, two sites
    for (model, N, nu, terms) in [("SPIN_HALF", 6, 6, heisenberg_terms(chain(6), 1.0)),
                                  ("SPIN_HALF", 6, 0, heisenberg_terms(chain(6), 1.0)),
                                  ("SPIN_HALF", 6, 3, []), ("SPIN_HALF", 2, 1, heisenberg_terms([(0, 1)], 1.0)),
                                  ("SPIN_HALF_GC", 2, 0, heisenberg_terms([(0, 1)], 2.0))]:
        m, b, h = pair(model, N, nu, 0, terms)
        _check(m, h, torch.float64, 1)
    m, b, h = pair("HUBBARD", 4, 0, 0, hubbard_terms(4, chain(4), 1.0, 3.0))
    _check(m, h, torch.float64, 1)
    m, b, h = pair("HUBBARD", 4, 4, 4, hubbard_terms(4, chain(4), 1.0, 3.0))
    _check(m, h, torch.float64, 1)


def test_alias_and_bad_arguments_rejected():
    m, b, h = pair("SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0))
    x = torch.ones(m.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(hphi.HphiError):
        hphi.hphi_apply_H(h, x, x)
    y = torch.ones(m.dim + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        hphi.hphi_apply_H(h, x, y)


def test_hermitian_on_gpu():
    m, b, h = pair("SPIN_HALF", 20, 10, 0, heisenberg_terms(square(5, 4), 1.0))
    u = torch.from_numpy(random_vectors(m.dim, 1, 1)[:, 0]).cuda()
    v = torch.from_numpy(random_vectors(m.dim, 1, 2)[:, 0]).cuda()
    hu, hv = torch.empty_like(u), torch.empty_like(v)
    hphi.hphi_apply_H(h, u, hu)
    hphi.hphi_apply_H(h, v, hv)
    a, c = torch.dot(u, hv).item(), torch.dot(hu, v).item()
    assert abs(a - c) < 1e-13 * max(abs(a), 1.0)


def _sampled_rows(m, h, dtype, nvec, rows, seed):
    """Full-size check: x drawn on the device, y at sampled rows from the
    oracle's row entries and the gathered x values."""
    ctx = h.ctx
    x = torch.empty((m.dim, nvec) if nvec > 1 else (m.dim,), dtype=dtype, device="cuda")
    hphi.hphi_random_vector(ctx, x, seed)
    y = torch.empty_like(x)
    hphi.hphi_apply_H(h, x, y)
    torch.cuda.synchronize()
    worst = 0.0
    for r in rows:
        cols, vals, _ = m.row_entries(int(r))
        xv = x[torch.from_numpy(cols).cuda()].cpu().numpy().astype(np.float64)
        want = (vals[:, None] * xv.reshape(len(cols), -1)).sum(axis=0)
        got = y[int(r)].cpu().numpy().astype(np.float64).reshape(-1)
        scale = np.abs(vals).sum() * np.abs(xv).max()
        worst = max(worst, float(np.abs(got - want).max() / scale))
    del x, y
    torch.cuda.empty_cache()
    return worst


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_square_4x8_full_size_sampled(dtype):
    """The N=32 S^z=0 sector of the 4x8 lattice (601,080,390 rows)."""
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    rng = np.random.default_rng(8)
    rows = np.concatenate([[0, 1, m.dim - 1], rng.integers(0, m.dim, 400)])
    assert _sampled_rows(m, h, dtype, 1, rows, 42) < (1e-15 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("variant", [-1, 0])
def test_hubbard_4x4_full_size_sampled(variant):
    """165,636,900 rows: the bond-major kernel (automatic) and the generic one."""
    m, b, h = pair("HUBBARD", 16, 8, 8, hubbard_terms(16, square(4, 4), t=1.0, U=8.0))
    h.set_tuning(variant=variant)
    rng = np.random.default_rng(9)
    rows = np.concatenate([[0, m.dim - 1], rng.integers(0, m.dim, 300)])
    assert _sampled_rows(m, h, torch.float64, 1, rows, 43) < 1e-15
    assert _sampled_rows(m, h, torch.float32, 1, rows, 44) < 1e-6


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rrg26_block32_full_size_sampled(dtype):
    """2^26 rows x 32 real columns (16 complex TPQ vectors)."""
    bonds = random_regular_graph(26, 3, 4)
    terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004))
    m, b, h = pair("SPIN_HALF_GC", 26, 0, 0, terms)
    rng = np.random.default_rng(10)
    rows = np.concatenate([[0, m.dim - 1], rng.integers(0, m.dim, 200)])
    assert _sampled_rows(m, h, dtype, 32, rows, 44) < (1e-15 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("variant,split,hints,inner", [(-1, 1, 1, -1), (0, 1, 1, -1), (1, 1, 1, -1),
                                                       (0, 3, 0, 2), (1, 2, 0, 1), (1, 4, 1, 0), (-1, 8, 1, 32),
                                                       (2, 1, 1, -1), (2, 1, 0, 3), (3, 1, 1, -1)])
@pytest.mark.parametrize("shape", ["sector", "full", "hubbard"])
@pytest.mark.parametrize("nvec", [1, 2, 32])
def test_kernel_variants_and_knobs(variant, split, hints, inner, shape, nvec):
    """Every H*x kernel (generic, table-driven, on-the-fly ranks) and launch knob
    gives the oracle's result; the reductions are checked through Lanczos/TPQ."""
    if shape == "sector":
        m, b, h = pair("SPIN_HALF", 14, 7, 0, heisenberg_terms(square(7, 2), 1.0))
    elif shape == "full":
        bonds = random_regular_graph(14, 3, 9)
        m, b, h = pair("SPIN_HALF_GC", 14, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 3)))
    else:
        m, b, h = pair("HUBBARD", 8, 4, 3, hubbard_terms(8, chain(8), t=1.0, U=4.0, V=0.3))
    h.set_tuning(variant=variant, split=split, l2_hints=hints, inner_bits=inner)
    for dtype in (torch.float64, torch.float32):
        _check(m, h, dtype, nvec, alpha=0.9, beta=0.0 if nvec == 32 else 0.4, seed=nvec + split)


@pytest.mark.parametrize("coop", [-1, 0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("split", [1, 3])
@pytest.mark.parametrize("shape", ["sector", "full"])
def test_wide_rows_cooperative_knob(coop, split, shape):
    """32-column rows: bond work shared by the lanes of a row (coop=1) or
    repeated per lane (coop=0) gives the oracle's result, with and without an
    accumulate term."""
    if shape == "sector":
        m, b, h = pair("SPIN_HALF", 16, 8, 0, heisenberg_terms(square(4, 4), 1.0))
    else:
        bonds = random_regular_graph(16, 3, 12)
        m, b, h = pair("SPIN_HALF_GC", 16, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 5)))
    h.set_tuning(variant=1, coop=coop, split=split)
    assert h.get_tuning()["coop"] == coop
    for dtype in (torch.float64, torch.float32):
        _check(m, h, dtype, 32, alpha=1.1, beta=0.0, seed=20 + split)
        _check(m, h, dtype, 32, alpha=-0.6, beta=0.25, seed=21 + split)


@pytest.mark.parametrize("N,nup", [(12, 6), (13, 4), (17, 8), (20, 7), (22, 11)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lists", [0, 1, 2, 3])
def test_staged_kernel(N, nup, dtype, lists):
    """Shared-memory staged kernel (spin sector, one column): low halves of
    4 to 11 bits, every popcount class, random XXZ couplings incl. zero Jxy."""
    rng = random.Random(N * 31 + nup)
    pairs = rng.sample(list(itertools.combinations(range(N), 2)), 3 * N)
    terms = [("XXZ", i, j, 0, rng.uniform(-1, 2), rng.uniform(-1, 2) if k % 7 else 0.0)
             for k, (i, j) in enumerate(pairs)]
    m, b, h = pair("SPIN_HALF", N, nup, 0, terms)
    h.set_tuning(variant=2, staged_lists=lists)
    _check(m, h, dtype, 1, alpha=0.8, beta=0.0, seed=N)
    _check(m, h, dtype, 1, alpha=-1.1, beta=0.35, seed=N + 1)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lists", [0, 1, 2, 3])
def test_staged_square_4x8_full_size_sampled(dtype, lists):
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    h.set_tuning(variant=2, staged_lists=lists)
    rng = np.random.default_rng(18)
    rows = np.concatenate([[0, 1, m.dim - 1], rng.integers(0, m.dim, 400)])
    assert _sampled_rows(m, h, dtype, 1, rows, 52) < (1e-15 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("N,nup", [(2, 1), (12, 6), (13, 4), (17, 8), (20, 7), (22, 11), (24, 12)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_bond_major_kernel(N, nup, dtype):
    """Bond-major kernel (spin sector, one column): every popcount class, low
    halves of 1 to 12 bits, random XXZ couplings incl. zero Jxy, so lists of
    every length from empty up; with and without the accumulate term."""
    rng = random.Random(N * 37 + nup)
    pairs = list(itertools.combinations(range(N), 2))
    pairs = rng.sample(pairs, min(len(pairs), 3 * N))
    terms = [("XXZ", i, j, 0, rng.uniform(-1, 2), rng.uniform(-1, 2) if k % 7 else 0.0)
             for k, (i, j) in enumerate(pairs)]
    m, b, h = pair("SPIN_HALF", N, nup, 0, terms)
    h.set_tuning(variant=3)
    _check(m, h, dtype, 1, alpha=0.8, beta=0.0, seed=N)
    _check(m, h, dtype, 1, alpha=-1.1, beta=0.35, seed=N + 1)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_bond_major_square_4x8_full_size_sampled(dtype):
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    h.set_tuning(variant=3)
    rng = np.random.default_rng(19)
    rows = np.concatenate([[0, 1, m.dim - 1], rng.integers(0, m.dim, 400)])
    assert _sampled_rows(m, h, dtype, 1, rows, 53) < (1e-15 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("shape", ["sector", "full", "hubbard"])
@pytest.mark.parametrize("dtype,nvec", [(torch.float32, 1), (torch.float64, 1), (torch.complex64, 16)])
def test_autotune_keeps_results(shape, dtype, nvec):
    if shape == "sector":
        m, b, h = pair("SPIN_HALF", 16, 8, 0, heisenberg_terms(square(4, 4), 1.0))
    elif shape == "full":
        bonds = random_regular_graph(14, 3, 9)
        m, b, h = pair("SPIN_HALF_GC", 14, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 3)))
    else:
        m, b, h = pair("HUBBARD", 8, 4, 3, hubbard_terms(8, chain(8), t=1.0, U=4.0, V=0.3))
    ms, tried = h.autotune(dtype, nvec, reps=2)
    assert ms > 0 and tried >= 2
    _check(m, h, dtype, nvec, alpha=0.9, beta=0.0, seed=5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_hubbard_large_down_sector_falls_back(dtype):
    """D_dn = C(18, 8) = 43,758 down states: the block of one up string does not
    fit in shared memory, so one-column launches take the generic kernel."""
    m, b, h = pair("HUBBARD", 18, 1, 8, hubbard_terms(18, chain(18), t=1.0, U=4.0))
    _check(m, h, dtype, 1, alpha=0.9, beta=0.3, seed=3)
    assert not h.ctx.last_kernel().startswith("k_hvp")


def test_last_kernel_names_the_launch():
    """hphi_last_kernel reports the instance that ran and the source hash the
    library was built from (what the bench matches profiles against)."""
    import importlib
    build = importlib.import_module("paper_2307_13222_gb300.build")
    m, b, h = pair("SPIN_HALF", 16, 8, 0, heisenberg_terms(square(4, 4), 1.0))
    x = torch.ones(m.dim, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    hphi.hphi_apply_H(h, x, y)
    torch.cuda.synchronize()
    name = h.ctx.last_kernel()
    assert name.startswith("k_hvp<f32,512,RED0,MINB2>@") and name.endswith("@" + build.source_tag("hv_phased.cu"))
    h.set_tuning(variant=0)
    hphi.hphi_apply_H(h, x, y)
    assert h.ctx.last_kernel().startswith("k_hvl<f32,")


@pytest.mark.parametrize("N,nup", [(2, 1), (5, 2), (9, 4), (12, 6), (13, 4), (17, 8), (20, 7), (22, 11), (24, 12)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_segment_kernel(N, nup, dtype):
    """High-high pass plus bond-major kernel (variant 4; spin sector, one
    column): low halves of 1 to 12 bits (0 to 4 bits above the lowest 8, so
    one to 16 chunks), every popcount class, random XXZ couplings incl. zero
    Jxy; the accumulate form (beta != 0) keeps the high-high terms in the
    context buffer, the plain one in y."""
    rng = random.Random(N * 41 + nup)
    pairs = list(itertools.combinations(range(N), 2))
    pairs = rng.sample(pairs, min(len(pairs), 3 * N))
    terms = [("XXZ", i, j, 0, rng.uniform(-1, 2), rng.uniform(-1, 2) if k % 7 else 0.0)
             for k, (i, j) in enumerate(pairs)]
    m, b, h = pair("SPIN_HALF", N, nup, 0, terms)
    h.set_tuning(variant=4)
    _check(m, h, dtype, 1, alpha=0.8, beta=0.0, seed=N)
    assert h.ctx.last_kernel().startswith("k_hhs+k_hvp<"), h.ctx.last_kernel()
    _check(m, h, dtype, 1, alpha=-1.1, beta=0.35, seed=N + 1)


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (6, 4), (5, 5), (6, 5)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_segment_kernel_square_lattices(Lx, Ly, dtype):
    """Periodic square lattices up to 30 sites (S^z = 0) through variant 4."""
    N = Lx * Ly
    m, b, h = pair("SPIN_HALF", N, N // 2, 0, heisenberg_terms(square(Lx, Ly), 1.0))
    h.set_tuning(variant=4)
    if m.dim <= 3_000_000:
        _check(m, h, dtype, 1, alpha=1.0, beta=0.0, seed=N)
    else:
        rng = np.random.default_rng(N)
        rows = np.concatenate([[0, 1, m.dim - 1], rng.integers(0, m.dim, 300)])
        assert _sampled_rows(m, h, dtype, 1, rows, 60 + N) < (1e-15 if dtype == torch.float64 else 1e-6)
    assert h.ctx.last_kernel().startswith("k_hhs+k_hvp<")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_segment_square_4x8_full_size_sampled(dtype):
    m, b, h = pair("SPIN_HALF", 32, 16, 0, heisenberg_terms(square(8, 4), 1.0))
    h.set_tuning(variant=4)
    rng = np.random.default_rng(29)
    rows = np.concatenate([[0, 1, m.dim - 1], rng.integers(0, m.dim, 400)])
    assert _sampled_rows(m, h, dtype, 1, rows, 63) < (1e-15 if dtype == torch.float64 else 1e-6)
    assert h.ctx.last_kernel().startswith("k_hhs+k_hvp<")


@pytest.mark.parametrize("variant", [3, 4])
def test_fused_reductions_one_column_sector(variant):
    """<x, Hx>, |Hx|^2, |x|^2 of one sector column (the cTPQ step on one
    column and the FP64 Rayleigh quotient take this launch form)."""
    m, b, h = pair("SPIN_HALF", 16, 8, 0, heisenberg_terms(square(4, 4), 1.0))
    h.set_tuning(variant=variant)
    V0 = random_vectors(m.dim, 1, 5)
    Vg = torch.from_numpy(V0).cuda().contiguous()
    Vo = V0.copy()
    norm2 = np.zeros(1)
    for _ in range(4):
        e, h2, logd = hphi.hphi_tpq_step(h, Vg, 0.05, 6, norm2)
        eo, h2o, do = m.tpq_step(Vo, 0.05, 6)
        assert np.allclose(e, eo, rtol=1e-12) and np.allclose(h2, h2o, rtol=1e-12)
        assert np.allclose(logd, np.log(do), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("N,seed", [(12, 9), (20, 3), (22, 4)])
def test_tiled_block_kernel(N, seed, dtype):
    """Tiled two-pass block kernel (variant 5; full space, 32 FP32 columns):
    one tile holding every row (N = 12) and two passes over tiles of the
    bond-graph split (N = 20, 22), plain and with the accumulate term."""
    bonds = random_regular_graph(N, 3, seed)
    m, b, h = pair("SPIN_HALF_GC", N, 0, 0, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, seed + 7)))
    h.set_tuning(variant=5)
    _check(m, h, dtype, 32, alpha=1.1, beta=0.0, seed=30 + N)
    want = "k_tile<f32," if dtype == torch.float32 else "k_tile<f64,"
    assert h.ctx.last_kernel().startswith(want), h.ctx.last_kernel()
    _check(m, h, dtype, 32, alpha=-0.6, beta=0.25, seed=31 + N)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_tiled_block_rrg26_full_size_sampled(dtype):
    """The cTPQ block shape at full size (2^26 rows x 16 complex columns, FP32
    and FP64) through the tiled kernel: two passes over L2-sized tiles."""
    bonds = random_regular_graph(26, 3, 4)
    terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004))
    m, b, h = pair("SPIN_HALF_GC", 26, 0, 0, terms)
    h.set_tuning(variant=5)
    rng = np.random.default_rng(11)
    rows = np.concatenate([[0, m.dim - 1], rng.integers(0, m.dim, 200)])
    assert _sampled_rows(m, h, dtype, 32, rows, 45) < (1e-6 if dtype == torch.float32 else 1e-14)
    assert h.ctx.last_kernel().startswith("k_tile<f32," if dtype == torch.float32 else "k_tile<f64,")
