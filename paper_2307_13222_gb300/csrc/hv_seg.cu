// High-high pass of the one-column H*x for the spin-1/2 S^z sector, run before
// the bond-major kernel (hv_phased.cu), which then skips its high-high phase.
//
// A sector state is (h, l): h the high half, l the low half of popcount p.
// Its row is jb[h] + ja[l], and a bond with both sites in h (Sec. 3.1.1: the
// exchange term Jxy/2 (S+S- + S-S+) flips two antiparallel spins) maps row
// jb[h] + ja[l] to jb[h ^ m] + ja[l]: the same offset in another row block.
// Taken block by block, these terms read about a dozen other blocks spread
// over the whole high space, which have left L2 again by the time their
// neighbours need them (the single-pass kernel moves about 7x its algorithmic
// bytes from DRAM, mostly for these terms).
//
// Here the rows are cut along the low half instead.  Split l into its lowest
// n0 = min(8, N_lo) bits and the upper n1 = N_lo - n0 bits l1: the rows of
// one block whose l1 lies in [t0, t0 + W) are contiguous, from SO[p][t0] to
// SO[p][t0 + W] (SO[p][t] = number of class-p low halves whose upper part is
// below t), and a high-high term keeps l1.  So the work is walked chunk by
// chunk of W consecutive l1 values, every block within one chunk before the
// next chunk: the slices of all blocks in one chunk (D x W / 2^n1 rows, sized
// to a fraction of L2) stay in L2 while every thread block works on that
// chunk, and each slice comes from DRAM about once.  A warp owns one (chunk,
// block) slice, lists the block's applicable high-high bonds as row offsets,
// and streams:
//   t[row] = sum_k c_k x[row + jb[h ^ m_k] - jb[h]]      (coalesced, from L2).
// t lives in y when y's old value is not read (beta = 0 and v != y), else in
// a context buffer; the bond-major kernel adds t[row] to its diagonal term.
#include "hvcommon.cuh"

#include <vector>

namespace hphi {

namespace {

constexpr int kHhsWarps = 8;  // warps per thread block; each owns one slice at a time

template <typename T>
__global__ void __launch_bounds__(32 * kHhsWarps, 6)
    k_hhs(const HvTables P, const SegArgs s, int wbits, const T *__restrict__ X, T *__restrict__ Tout) {
    __shared__ int32_t gdel[kHhsWarps][kMaxHH];
    __shared__ T gco[kHhsWarps][kMaxHH];
    const HamDesc &D = *P.desc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nH = (int64_t)1 << s.nhi;
    const int nchunk = 1 << (s.n1 - wbits);
    const int64_t units = nH * nchunk;
    // unit u: chunk u / nH, block u % nH; consecutive warps take consecutive blocks
    // of the same chunk
    for (int64_t u = (int64_t)blockIdx.x * kHhsWarps + warp; u < units; u += (int64_t)gridDim.x * kHhsWarps) {
        const int j = (int)(u / nH);
        const int64_t h = u - (int64_t)j * nH;
        const uint64_t jbh = P.jb[h];
        if (jbh == ~0ull) continue;
        const int p = s.n - __popcll((unsigned long long)h);
        if (p < 0 || p > s.nlo) continue;
        const uint32_t t0 = (uint32_t)j << wbits, t1 = t0 + (1u << wbits);
        const uint32_t r0 = s.so[(p << s.n1) | t0];
        const uint32_t r1 = t1 < (1u << s.n1) ? s.so[(p << s.n1) | t1] : P.loff[p + 1] - P.loff[p];
        if (r0 >= r1) continue;
        int ng = 0;
        for (int k0 = 0; k0 < D.n_hh; k0 += 32) {
            const int k = k0 + lane;
            bool app = false;
            int32_t del = 0;
            T cf = (T)0;
            if (k < D.n_hh) {
                const HHBond &bd = D.hh[k];
                if (bd.cxy != 0.0 && (((h >> bd.i) ^ (h >> bd.j)) & 1)) {
                    const uint64_t h2 = (uint64_t)h ^ ((1ull << bd.i) | (1ull << bd.j));
                    del = (int32_t)((int64_t)P.jb[h2] - (int64_t)jbh);
                    cf = (T)bd.cxy;
                    app = true;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, app);
            const int pos = ng + __popc(m & lt);
            if (app && pos < kMaxHH) {
                gdel[warp][pos] = del;
                gco[warp][pos] = cf;
            }
            ng += __popc(m);
        }
        ng = ng < kMaxHH ? ng : kMaxHH;
        __syncwarp();
        const T *xb = X + jbh;
        T *tb = Tout + jbh;
        // two rows per lane, eight bonds per batch: sixteen loads in flight
        for (uint32_t r = r0 + lane; r < r1; r += 64) {
            const bool two = r + 32 < r1;
            const uint32_t rb = two ? r + 32 : r;
            T acc0 = (T)0, acc1 = (T)0;
            for (int k = 0; k < ng; k += 8) {
                T v0[8], v1[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int kk = k + q < ng ? k + q : ng - 1;
                    v0[q] = __ldg(xb + (int64_t)r + gdel[warp][kk]);
                    v1[q] = __ldg(xb + (int64_t)rb + gdel[warp][kk]);
                }
#pragma unroll
                for (int q = 0; q < 8; q++)
                    if (k + q < ng) {
                        acc0 = fma(gco[warp][k + q], v0[q], acc0);
                        acc1 = fma(gco[warp][k + q], v1[q], acc1);
                    }
            }
            tb[r] = acc0;
            if (two) tb[rb] = acc1;
        }
        __syncwarp();
    }
}

}  // namespace

// The split of the low half and the table SO of a spin S^z-sector Hamiltonian
// with N_lo <= 16 (nothing is built otherwise and variant 4 is not offered).
int build_seg_tables(hphi_ctx *ctx, hphi_ham *H) {
    const hphi_basis *B = H->basis;
    if (B->model != HPHI_SPIN_HALF || H->nlo > 16 || H->nlo < 1 || H->host.n_hh > kMaxHH) return HPHI_OK;
    SegArgs s{};
    s.nlo = H->nlo;
    s.nhi = H->host.nhi;
    s.n = H->host.n;
    s.n0 = H->nlo < 8 ? H->nlo : 8;
    s.n1 = H->nlo - s.n0;
    const int n0 = s.n0, n1 = s.n1;
    auto binom = [](int n, int k) -> int64_t {
        if (k < 0 || k > n) return 0;
        int64_t r = 1;
        for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
        return r;
    };
    std::vector<uint16_t> so((size_t)(H->nlo + 1) << n1);
    for (int p = 0; p <= H->nlo; p++) {
        int64_t acc = 0;
        for (uint32_t l1 = 0; l1 < (1u << n1); l1++) {
            if (acc > 65535) return HPHI_OK;
            so[((size_t)p << n1) | l1] = (uint16_t)acc;
            acc += binom(n0, p - __builtin_popcount(l1));
        }
    }
    cudaError_t e = cudaMalloc((void **)&H->seg_so, so.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemcpy(H->seg_so, so.data(), so.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(ctx, e, "segment table");
    s.so = H->seg_so;
    H->seg = new (std::nothrow) SegArgs(s);
    if (!H->seg) return set_err(ctx, HPHI_E_NOMEM, "segment table");
    return HPHI_OK;
}

template <typename T>
int launch_seg(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, int red_mode, int *grid) {
    if (!ham->seg || !a.P.ph_ent)
        return set_err(ctx, HPHI_E_INVAL, "high-high pass: no segment table or bond lists for this Hamiltonian");
    const SegArgs &s = *ham->seg;
    // t in y when y's old value is not read (beta = 0 and v is not y); else a context buffer
    T *tbuf = nullptr;
    if (a.beta == 0.0 && (a.v == nullptr || a.v != a.y)) {
        tbuf = a.y;
    } else {
        const size_t need = (size_t)ham->D * sizeof(T);
        if (ctx->seg_tmp_bytes < need) {
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(ctx->seg_tmp);
            ctx->seg_tmp = nullptr;
            ctx->seg_tmp_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->seg_tmp, need);
            if (e != cudaSuccess) return cuda_err(ctx, e, "high-high pass buffer");
            ctx->seg_tmp_bytes = need;
        }
        tbuf = (T *)ctx->seg_tmp;
    }
    // chunk width: the x slices of one chunk take at most 30 % of L2
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess || l2 <= 0) {
        cudaGetLastError();
        l2 = 64 << 20;
    }
    const double per_l1 = (double)ham->D * sizeof(T) / (double)(1u << s.n1);
    int wbits = 0;
    while (wbits < s.n1 && per_l1 * (double)(2u << wbits) <= 0.3 * (double)l2) wbits++;
    const int occ = dyn_occupancy(ctx, (const void *)k_hhs<T>, 32 * kHhsWarps, 0);
    const int64_t units = ((int64_t)1 << s.nhi) << (s.n1 - wbits);
    int64_t g = (int64_t)(occ > 0 ? occ : 1) * ctx->sm_count;
    const int64_t need_blocks = (units + kHhsWarps - 1) / kHhsWarps;
    if (g > need_blocks) g = need_blocks;
    if (g < 1) g = 1;
    // one timing slot covers both launches (the H*x is the pair)
    const int slot = prof_begin(ctx, PROF_HV);
    k_hhs<T><<<(int)g, 32 * kHhsWarps, 0, ctx->stream>>>(a.P, s, wbits, a.x, tbuf);
    HPHI_CUDA(ctx, cudaGetLastError());
    a.tin = tbuf;
    const bool prof = ctx->prof;
    ctx->prof = false;
    const int st = launch_phased<T>(ctx, ham, a, red_mode, grid);
    ctx->prof = prof;
    prof_end(ctx, slot);
    a.tin = nullptr;
    if (st) return st;
    char name[sizeof ctx->last_kernel];
    snprintf(name, sizeof name, "k_hhs+%s", ctx->last_kernel);
    snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "%s", name);
    return HPHI_OK;
}

template int launch_seg<float>(hphi_ctx *, const hphi_ham *, HvArgs<float> &, int, int *);
template int launch_seg<double>(hphi_ctx *, const hphi_ham *, HvArgs<double> &, int, int *);

}  // namespace hphi
