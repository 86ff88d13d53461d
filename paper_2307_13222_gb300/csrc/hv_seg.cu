// Two-pass segment H*x kernel for the spin-1/2 S^z sector, one column.
//
// A sector state s = (h, l1, l0): h the high half (N_hi bits), and the low
// half l (N_lo bits) split into l0, its lowest n0 = min(8, N_lo) bits, and l1,
// the remaining n1 = N_lo - n0 bits.  Lin's rank of s is jb[h] + ja[l] with
// ja[l] = SO[p][l1] + r8[l0]: p = pop(l), SO[p][l1] the number of class-p low
// halves whose upper part is below l1, r8[l0] the rank of l0 among the n0-bit
// strings of its popcount.  The rows of one (h, l1) are therefore a contiguous
// "segment" of C(n0, p - pop(l1)) rows, ordered by l0, and every segment of
// the same l0 class c0 lists the same l0 strings in the same order.
//
// Each exchange bond (Sec. 3.1.1: J S_i.S_j, here Jxy/2 (S+S- + S-S+) off the
// diagonal) moves one up spin between its two sites, and where those sites
// lie decides how the target row is found:
//   G  both in h:        same (l1, l0), block h ^ m: target = source + jb[h^m] - jb[h]
//   E  l0 bit i, h bit a: block h ^ 2^a, same l1, l0 ^ 2^i
//   A  both in l0:        same segment, l0 ^ m
//   B  l0 bit i, l1 bit b: same block, segment l1 ^ 2^b, l0 ^ 2^i
//   C  both in l1:        same block, segment l1 ^ m, same l0
//   F  l1 bit b, h bit a: block h ^ 2^a, segment l1 ^ 2^b, same l0
// G and E keep l1: all their sources lie in the "strip" of one l1, i.e. the
// segments (h, l1) of every h, a few MB for the 4x8 sector (2.4 GB / 256).
// A, B, C and F keep h or flip one bit of it.
//
// Pass 1 (k_sgs) walks the strips one after another: while every thread block
// works on the same strip, the strip stays in L2 and the G and E sources,
// spread over the whole high space, come from L2 instead of DRAM.  A warp owns
// one segment; each lane one row (register accumulation, no lists):
//   t[row] = sum_G c x[row + dG] + sum_{E applicable} c x[jb[h^2^a] + SO + r8[l0^2^i]].
// Pass 2 (k_sgb) walks the row blocks h like the other staged kernels: the
// block's x in shared memory, SO and r8 in shared memory; each lane owns a row:
//   acc = diag x[row] + t[row] + A, B, C terms from shared memory + F terms
//   from block h ^ 2^a (the traversal varies the F bonds' high bits first, so
//   those blocks are the ones just staged by neighbouring thread blocks),
// then the epilogue y = alpha acc + beta y + gamma v with the fused
// reductions.  Each row sums its terms in a fixed order: deterministic.
// t lives in y when y's old value is not needed (beta = 0 and v != y), else in
// a context buffer.
#include "hvcommon.cuh"

#include <vector>

namespace hphi {

namespace {

template <typename T>
constexpr int seg_threads() { return sizeof(T) == 4 ? 512 : 1024; }
template <typename T>
constexpr int seg_minb() { return sizeof(T) == 4 ? 3 : 1; }
constexpr int kSgsWarps = 8;  // warps (segments in flight) per thread block of pass 1

// Pass 1: G and E terms of every row, strip by strip.
template <typename T>
__global__ void __launch_bounds__(32 * kSgsWarps, 4)
    k_sgs(const SegArgs s, const HvTables P, const T *__restrict__ X, T *__restrict__ Tout) {
    __shared__ uint8_t r8s[256], uns[256];
    __shared__ int32_t gdel[kSgsWarps][kMaxHH];
    __shared__ T gco[kSgsWarps][kMaxHH];
    __shared__ int64_t ebase[kSgsWarps][kSegMax];
    __shared__ uint8_t eneed[kSgsWarps][kSegMax];
    __shared__ T eco[kSegMax];
    const int n0s = 1 << s.n0;
    for (int i = threadIdx.x; i < n0s; i += blockDim.x) {
        r8s[i] = s.r8[i];
        uns[i] = s.un8[i];
    }
    for (int i = threadIdx.x; i < s.nE; i += blockDim.x) eco[i] = (T)s.cE[i];
    __syncthreads();
    const HamDesc &D = *P.desc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nH = (int64_t)1 << s.nhi;
    const int64_t nhc = (nH + kSgsWarps - 1) / kSgsWarps;
    const int64_t items = nhc << s.n1;
    for (int64_t c = blockIdx.x; c < items; c += gridDim.x) {
        const uint32_t t = (uint32_t)(c / nhc);
        const int64_t h = (c - (int64_t)t * nhc) * kSgsWarps + warp;
        if (h >= nH) continue;
        const uint64_t jbh = P.jb[h];
        if (jbh == ~0ull) continue;
        const int p = s.n - __popcll((unsigned long long)h);
        const int c0 = p - __popc(t);
        if (c0 < 0 || c0 > s.n0 || p < 0 || p > s.nlo) continue;
        const int64_t seg = (int64_t)jbh + s.so[(p << s.n1) | t];
        const int len = s.off8[c0 + 1] - s.off8[c0];
        // G: the high-high bonds whose bits differ in h, as offsets to block h ^ m
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
        // E: segment (h ^ 2^a, t) of each bond; the term applies where bit i of l0
        // equals 1 - bit a of h (the target then lies in the sector)
        for (int e = lane; e < s.nE; e += 32) {
            const int a = s.E1[e];
            const uint64_t h2 = (uint64_t)h ^ (1ull << a);
            const int p2 = s.n - __popcll((unsigned long long)h2);
            const uint64_t j2 = P.jb[h2];
            const bool ok = j2 != ~0ull && p2 >= 0 && p2 <= s.nlo;
            ebase[warp][e] = ok ? (int64_t)j2 + s.so[(p2 << s.n1) | t] : (int64_t)0;
            eneed[warp][e] = ok ? (uint8_t)(1 - ((h >> a) & 1)) : (uint8_t)2;
        }
        __syncwarp();
        const int ob = s.off8[c0];
        for (int r = lane; r < len; r += 32) {
            const uint32_t l0 = uns[ob + r];
            const T *xr = X + seg + r;
            T acc = (T)0;
            int k = 0;
            for (; k + 4 <= ng; k += 4) {
                T v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) v[u] = __ldg(xr + gdel[warp][k + u]);
#pragma unroll
                for (int u = 0; u < 4; u++) acc = fma(gco[warp][k + u], v[u], acc);
            }
            for (; k < ng; k++) acc = fma(gco[warp][k], __ldg(xr + gdel[warp][k]), acc);
            for (int e = 0; e < s.nE; e++) {
                const int i = s.E0[e];
                if (((l0 >> i) & 1u) == eneed[warp][e])
                    acc = fma(eco[e], __ldg(X + ebase[warp][e] + r8s[l0 ^ (1u << i)]), acc);
            }
            Tout[seg + r] = acc;
        }
        __syncwarp();
    }
}

// Pass 2: diagonal, t, and the A, B, C, F terms; epilogue and reductions.
template <typename T, int NT, int RED, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_sgb(const HvArgs<T> a, const SegArgs s, const T *Tin, uint32_t xs_len) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *xs = (T *)s_raw;
    uint16_t *sos = (uint16_t *)(s_raw + (((size_t)xs_len * sizeof(T) + 15) & ~(size_t)15));
    const int nso = (s.nlo + 1) << s.n1;
    uint8_t *r8s = (uint8_t *)(sos + nso);
    __shared__ HBlock<T> hb;
    __shared__ int64_t fbase[kSegMax];
    __shared__ int16_t fso[kSegMax];   // row of SO for the target block's class
    __shared__ uint8_t fneed[kSegMax];
    __shared__ T cA[kSegMax], cB[kSegMax], cC[kSegMax], cF[kSegMax];
    const HvTables &P = a.P;
    const int n0s = 1 << s.n0;
    for (int i = threadIdx.x; i < nso; i += NT) sos[i] = s.so[i];
    for (int i = threadIdx.x; i < n0s; i += NT) r8s[i] = s.r8[i];
    for (int i = threadIdx.x; i < kSegMax; i += NT) {
        cA[i] = (T)s.cA[i];
        cB[i] = (T)s.cB[i];
        cC[i] = (T)s.cC[i];
        cF[i] = (T)s.cF[i];
    }
    const uint64_t keep = spol(P.hints, 0), stream = spol(P.hints, 1);
    const T al = (T)(a.alpha_dev ? a.alpha_dev[0] : a.alpha[0]);
    const T ga = (T)(a.gamma_dev ? a.gamma_dev[0] : a.gamma[0]);
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    RedAcc<T> racc[NR > 0 ? NR : 1];
    const T *__restrict__ dlow = (const T *)P.dlow;
    const T *__restrict__ X = a.x;
    const uint32_t m0 = (1u << s.n0) - 1u;
    for (int64_t c = blockIdx.x; c < P.nh; c += gridDim.x) {
        const int64_t h = block_of(P, c);
        __syncthreads();  // the previous block is done with hb and xs
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base, len = hb.len, cp0 = hb.cp0;
        const int p = P.n - __popcll((unsigned long long)h);
        if (threadIdx.x < s.nF) {
            const int k = threadIdx.x, aa = s.F1[k];
            const uint64_t h2 = (uint64_t)h ^ (1ull << aa);
            const int p2 = s.n - __popcll((unsigned long long)h2);
            const uint64_t j2 = P.jb[h2];
            const bool ok = j2 != ~0ull && p2 >= 0 && p2 <= s.nlo;
            fbase[k] = ok ? (int64_t)j2 : (int64_t)0;
            fso[k] = (int16_t)(ok ? (p2 << s.n1) : 0);
            fneed[k] = ok ? (uint8_t)(1 - ((h >> aa) & 1)) : (uint8_t)2;
        }
        for (uint32_t q = threadIdx.x; q < len; q += NT) xs[q] = gload<T>(X + base + q, keep);
        __syncthreads();
        const int pso = p << s.n1;
        for (uint32_t q = threadIdx.x; q < len; q += NT) {
            const uint32_t cp = cp0 + q;
            const uint32_t l = __ldg(P.lstate + cp);
            const uint32_t l0 = l & m0, l1 = l >> s.n0;
            const uint32_t r = r8s[l0];
            const uint32_t sq = q - r;  // this row's segment start
            T d = __ldg(dlow + cp) + hb.dh;
            for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
            const uint32_t row = base + q;
            T acc = fma(d, xs[q], Tin[row]);
            for (int k = 0; k < s.nA; k++) {
                const uint32_t i = s.A0[k], j = s.A1[k];
                if (((l0 >> i) ^ (l0 >> j)) & 1u) acc = fma(cA[k], xs[sq + r8s[l0 ^ ((1u << i) | (1u << j))]], acc);
            }
            for (int k = 0; k < s.nB; k++) {
                const uint32_t i = s.B0[k], b = s.B1[k];
                if (((l0 >> i) ^ (l1 >> b)) & 1u)
                    acc = fma(cB[k], xs[sos[pso | (l1 ^ (1u << b))] + r8s[l0 ^ (1u << i)]], acc);
            }
            for (int k = 0; k < s.nC; k++) {
                const uint32_t b1 = s.C0[k], b2 = s.C1[k];
                if (((l1 >> b1) ^ (l1 >> b2)) & 1u)
                    acc = fma(cC[k], xs[sos[pso | (l1 ^ ((1u << b1) | (1u << b2)))] + r], acc);
            }
            for (int k = 0; k < s.nF; k++) {
                const uint32_t b = s.F0[k];
                if (((l1 >> b) & 1u) == fneed[k])
                    acc = fma(cF[k], gload<T>(X + fbase[k] + sos[fso[k] | (l1 ^ (1u << b))] + r, keep), acc);
            }
            const T xo = xs[q];
            T out = al * acc;
            T *yr = a.y + row;
            if (use_beta) out = fma(be, cload<T>(yr, stream), out);
            if (use_v) out = fma(ga, cload<T>(a.v + row, stream), out);
            cstore<T>(yr, stream, out);
            if constexpr (RED == 1) racc[0].add(xo, out);
            if constexpr (RED == 2) {
                racc[0].add(xo, acc);
                racc[1].add(acc, acc);
                racc[2].add(xo, xo);
            }
            if constexpr (RED == 3) racc[0].add(out, out);
        }
    }
    if constexpr (RED != 0) {
        __shared__ double red_sm[NT / 32][3];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const double v = warp_sum_d(racc[r].value());
            if (lane == 0) red_sm[warp][r] = v;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            const int r = threadIdx.x;
            double sum = 0.0;
            if (r < NR)
                for (int w = 0; w < NT / 32; w++) sum += red_sm[w][r];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol] = sum;
        }
    }
}

template <typename T, int RED>
int go_seg(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, const T *tbuf, int *grid_out) {
    constexpr int NT = seg_threads<T>(), MB = seg_minb<T>();
    const SegArgs &s = *ham->seg;
    const uint32_t xl = staged_block_len(ham);
    const size_t nso = (size_t)(s.nlo + 1) << s.n1;
    const size_t dyn = (((size_t)xl * sizeof(T) + 15) & ~(size_t)15) + nso * sizeof(uint16_t) + 256;
    static int occ[64] = {0};
    static size_t occ_dyn[64] = {0};
    const int dev = ctx->device;
    if (occ[dev] == 0 || occ_dyn[dev] != dyn) {
        cudaFuncSetAttribute(k_sgb<T, NT, RED, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sgb<T, NT, RED, MB>, NT, dyn);
        occ[dev] = n;
        occ_dyn[dev] = dyn;
    }
    if (occ[dev] < 1) return set_err(ctx, HPHI_E_INVAL, "segment H*x: a row block does not fit in shared memory");
    static int occ_s[64] = {0};
    if (occ_s[dev] == 0) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sgs<T>, 32 * kSgsWarps, 0);
        occ_s[dev] = n > 0 ? n : 1;
    }
    const int64_t nitems = (((int64_t)1 << s.nhi) + kSgsWarps - 1) / kSgsWarps << s.n1;
    int64_t g1 = (int64_t)occ_s[dev] * ctx->sm_count;
    if (g1 > nitems) g1 = nitems;
    if (g1 < 1) g1 = 1;
    int64_t g2 = (int64_t)occ[dev] * ctx->sm_count;
    if (g2 > ham->nh) g2 = ham->nh;
    if (g2 < 1) g2 = 1;
    *grid_out = (int)g2;
    const int slot = prof_begin(ctx, PROF_HV);
    k_sgs<T><<<(int)g1, 32 * kSgsWarps, 0, ctx->stream>>>(s, a.P, a.x, (T *)tbuf);
    k_sgb<T, NT, RED, MB><<<(int)g2, NT, dyn, ctx->stream>>>(a, s, tbuf, xl);
    snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_sgs+k_sgb<%s,%d,RED%d,MINB%d>@" HPHI_SRC_TAG, tname<T>(), NT,
             RED, MB);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace

// Segment tables and bond classes of a spin S^z-sector Hamiltonian (N_lo <= 16,
// at most kSegMax bonds of each class); nothing is built otherwise and the
// kernel is not offered.
int build_seg_tables(hphi_ctx *ctx, hphi_ham *H) {
    const hphi_basis *B = H->basis;
    if (B->model != HPHI_SPIN_HALF || H->nlo > 16 || H->nlo < 1) return HPHI_OK;
    const HamDesc &D = H->host;
    SegArgs s{};
    s.nlo = H->nlo;
    s.nhi = D.nhi;
    s.n = D.n;
    s.n0 = H->nlo < 8 ? H->nlo : 8;
    s.n1 = H->nlo - s.n0;
    const int n0 = s.n0, n1 = s.n1;
    auto push = [](int &cnt, uint8_t *x0, uint8_t *x1, double *cf, int u, int v, double c) {
        if (cnt >= kSegMax) return false;
        x0[cnt] = (uint8_t)u;
        x1[cnt] = (uint8_t)v;
        cf[cnt] = c;
        cnt++;
        return true;
    };
    bool ok = true;
    for (int k = 0; k < D.n_ll && ok; k++) {
        const LLBondD &bd = D.ll[k];
        if (bd.cxy == 0.0) continue;
        const int i = bd.i < bd.j ? bd.i : bd.j, j = bd.i < bd.j ? bd.j : bd.i;
        if (j < n0) ok = push(s.nA, s.A0, s.A1, s.cA, i, j, bd.cxy);
        else if (i < n0) ok = push(s.nB, s.B0, s.B1, s.cB, i, j - n0, bd.cxy);
        else ok = push(s.nC, s.C0, s.C1, s.cC, i - n0, j - n0, bd.cxy);
    }
    for (int k = 0; k < D.n_lh && ok; k++) {
        const LHBond &bd = D.lh[k];
        if (bd.cxy == 0.0) continue;
        if (bd.b < n0) ok = push(s.nE, s.E0, s.E1, s.cE, bd.b, bd.a, bd.cxy);
        else ok = push(s.nF, s.F0, s.F1, s.cF, bd.b - n0, bd.a, bd.cxy);
    }
    if (!ok || D.n_hh > kMaxHH) return HPHI_OK;
    // n0-bit strings by (popcount, value): ranks and the class-ordered list
    std::vector<uint8_t> r8((size_t)1 << n0), un((size_t)1 << n0);
    int pos = 0;
    for (int c = 0; c <= n0; c++) {
        s.off8[c] = (uint16_t)pos;
        int rk = 0;
        for (uint32_t v = 0; v < (1u << n0); v++)
            if (__builtin_popcount(v) == c) {
                r8[v] = (uint8_t)rk++;
                un[pos++] = (uint8_t)v;
            }
    }
    for (int c = n0 + 1; c <= 9; c++) s.off8[c] = (uint16_t)pos;
    // SO[p][l1]: class-p low halves whose upper part is below l1
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
    auto up = [&](auto **dst, const auto &v) -> int {
        const size_t bytes = v.size() * sizeof(v[0]);
        cudaError_t e = cudaMalloc((void **)dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err(ctx, e, "segment tables");
        return HPHI_OK;
    };
    int st;
    if ((st = up(&H->seg_r8, r8)) || (st = up(&H->seg_un, un)) || (st = up(&H->seg_so, so))) return st;
    s.r8 = H->seg_r8;
    s.un8 = H->seg_un;
    s.so = H->seg_so;
    H->seg = new (std::nothrow) SegArgs(s);
    if (!H->seg) return set_err(ctx, HPHI_E_NOMEM, "segment tables");
    return HPHI_OK;
}

// Order of the row blocks of pass 2: the high bits of the F bonds vary first,
// so that the blocks h ^ 2^a an F term reads belong to the same run of blocks.
void seg_traversal(const hphi_ham *ham, HvTables &P) {
    const SegArgs &s = *ham->seg;
    const int nb = s.nhi;
    uint32_t fm = 0;
    for (int k = 0; k < s.nF; k++) fm |= 1u << s.F1[k];
    int k = 0;
    for (int b = 0; b < nb; b++)
        if ((fm >> b) & 1) P.hperm[k++] = (uint8_t)b;
    for (int b = 0; b < nb; b++)
        if (!((fm >> b) & 1)) P.hperm[k++] = (uint8_t)b;
    P.use_perm = 1;
    P.outer_mask = 0;
}

template <typename T>
int launch_seg(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, int red_mode, int *grid) {
    if (!ham->seg) return set_err(ctx, HPHI_E_INVAL, "segment H*x: no segment tables for this Hamiltonian");
    // t in y when y's old value is not read (beta = 0 and v is not y); else a context buffer
    const T *tbuf = nullptr;
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
            if (e != cudaSuccess) return cuda_err(ctx, e, "segment H*x buffer");
            ctx->seg_tmp_bytes = need;
        }
        tbuf = (const T *)ctx->seg_tmp;
    }
    seg_traversal(ham, a.P);
    switch (red_mode) {
    case 0: return go_seg<T, 0>(ctx, ham, a, tbuf, grid);
    case 1: return go_seg<T, 1>(ctx, ham, a, tbuf, grid);
    case 2: return go_seg<T, 2>(ctx, ham, a, tbuf, grid);
    case 3: return go_seg<T, 3>(ctx, ham, a, tbuf, grid);
    default: return HPHI_E_INVAL;
    }
}

template int launch_seg<float>(hphi_ctx *, const hphi_ham *, HvArgs<float> &, int, int *);
template int launch_seg<double>(hphi_ctx *, const hphi_ham *, HvArgs<double> &, int, int *);

}  // namespace hphi
