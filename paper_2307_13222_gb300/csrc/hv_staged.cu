// Staged H*x kernel for the spin-1/2 S^z sector with one column.
//
// The thread block that owns row block h (all states with high half h) first
// copies the block's slice of x into shared memory.  Every low-low bond keeps
// the high half, so its target is in the same block: it is read from shared
// memory.  The target's position is Lin's rank of the flipped low half, which
// the kernel computes from two small shared tables instead of loading it:
// split an N_lo-bit string l with popcount p into its low byte and the rest,
//   rank_p(l) = T1[l & 255] + T2_p[l >> 8],
//   T1[b]     = #{b' < b : popcount(b') = popcount(b)}        (8-bit strings),
//   T2_p[u]   = sum_{u' < u} C(8, p - popcount(u'))           (N_lo - 8 high bits),
// i.e. Lin's two-table rank applied once more to the low half.  A low-low flip
// keeps p; a mixed bond flips one low bit, so its target block (the high half
// with bit a flipped) ranks l ^ 2^b with p - 1 or p + 1.  High-high bonds keep
// the low half: their targets are the same row offset in another block, read
// straight from global memory (coalesced).  The diagonal, the epilogue and the
// reductions are those of the other H*x kernels.
#include "hvcommon.cuh"

namespace hphi {

namespace {

constexpr int kStagedThreads = 512;
constexpr int kMaxLLs = 128;
constexpr int kT2Rows = 17;  // popcounts 0..16 of a low half of <= 16 bits
constexpr int kGathers = 4;  // global gathers in flight per chunk

__device__ __forceinline__ int binom8(int k) {  // C(8, k), 0 outside 0..8
    constexpr int c[9] = {1, 8, 28, 56, 70, 56, 28, 8, 1};
    return (k < 0 || k > 8) ? 0 : c[k];
}

// RED: 0 none; 1 <x,y>; 2 <x,Hx>, |Hx|^2, |x|^2; 3 |y|^2.  Dynamic shared
// memory: xs[max block length] (T), then the 3 * nwarps reduction slots.
// TAB = 0: targets in the block from the shared rank tables (T1, T2_p); TAB = 1:
// from the Hamiltonian's per-low-half lists (low-low targets and coefficient
// indices, ranks of the low half with one bit flipped), read coalesced.
template <typename T, int RED, int TAB, int MINB>
__global__ void __launch_bounds__(kStagedThreads, MINB) k_hvs(const HvArgs<T> a, uint32_t xs_len) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *xs = (T *)s_raw;
    double *red_sm = (double *)(s_raw + ((xs_len * sizeof(T) + 15) & ~(size_t)15));
    __shared__ HBlock<T> hb;
    __shared__ uint32_t ll_m[kMaxLLs];
    __shared__ T ll_c[kMaxLLs];
    __shared__ uint8_t t1[256];
    __shared__ uint16_t t2[kT2Rows][256];
    __shared__ T coef_sm[TAB ? kMaxCoef : 1];
    const HvTables &P = a.P;
    const HamDesc &D = *P.desc;
    if constexpr (TAB)
        for (int i = threadIdx.x; i < D.n_ncoef; i += blockDim.x) coef_sm[i] = (T)D.coef[i];
    const uint32_t L32 = (uint32_t)P.L;
    const int nll = D.n_ll < kMaxLLs ? D.n_ll : kMaxLLs;
    for (int i = threadIdx.x; i < nll; i += blockDim.x) {
        ll_m[i] = (1u << D.ll[i].i) | (1u << D.ll[i].j);
        ll_c[i] = (T)D.ll[i].cxy;
    }
    // T1 and T2_p (the rank tables of the low half)
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        const int pb = __popc(b);
        int r = 0;
        for (int b2 = 0; b2 < b; b2++) r += __popc(b2) == pb;
        t1[b] = (uint8_t)r;
    }
    const int nhi8 = P.nlo > 8 ? P.nlo - 8 : 0;
    for (int e = threadIdx.x; e < kT2Rows * 256; e += blockDim.x) {
        const int p = e >> 8, u = e & 255;
        int s = 0;
        if (u < (1 << nhi8))
            for (int u2 = 0; u2 < u; u2++) s += binom8(p - __popc(u2));
        t2[p][u] = (uint16_t)s;
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
    const uint32_t ld = (uint32_t)a.ldx;

    for (int64_t c = blockIdx.x; c < P.nh; c += gridDim.x) {
        const int64_t h = block_of(P, c);
        __syncthreads();  // the previous block is done with hb and xs
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base, len = hb.len, cp0 = hb.cp0;
        const int nhh = hb.nhh, nlh = hb.nlh;
        const int p = P.n - __popcll((unsigned long long)h);  // popcount of every low half of the block
        const uint16_t *t2c = t2[p];
        const uint16_t *t2m = t2[p > 0 ? p - 1 : 0];
        const uint16_t *t2p = t2[p < kT2Rows - 1 ? p + 1 : p];
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) xs[q] = gload<T>(X + (base + q) * ld, keep);
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) {
            const uint32_t cp = cp0 + q;
            const uint32_t l = __ldg(P.lstate + cp);
            T d = __ldg(dlow + cp) + hb.dh;
            for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
            const T xo = xs[q];
            T acc = d * xo;
            const uint32_t row = base + q;
            // high-high bonds: same low half in block h ^ m (row offset per block)
            for (int k0 = 0; k0 < nhh; k0 += kGathers) {
                T v[kGathers];
#pragma unroll
                for (int u = 0; u < kGathers; u++) {
                    const int k = k0 + u;
                    if (k < nhh)
                        v[u] = gload<T>(X + (row + (uint32_t)hb.hh_delta[k]) * ld, hb.hh_outer[k] ? stream : keep);
                }
#pragma unroll
                for (int u = 0; u < kGathers; u++)
                    if (k0 + u < nhh) acc = fma(hb.hh_coef[k0 + u], v[u], acc);
            }
            // low-low bonds: same block, from shared memory
            if constexpr (TAB) {
                const int cnt = __ldg(P.ll_cnt + cp);
#pragma unroll 4
                for (int e = 0; e < cnt; e++) {
                    const uint32_t pk = __ldg(P.ll_pk + ((uint32_t)e * L32 + cp));
                    acc = fma(coef_sm[pk >> 24], xs[pk & 0xFFFFFFu], acc);
                }
            } else {
#pragma unroll 4
                for (int k = 0; k < nll; k++) {
                    const uint32_t m = ll_m[k], lm = l & m;
                    if (lm != 0 && lm != m) {
                        const uint32_t l2 = l ^ m;
                        acc = fma(ll_c[k], xs[t1[l2 & 255u] + t2c[l2 >> 8]], acc);
                    }
                }
            }
            // mixed bonds: low bit b must equal 1 - bit a of h; target block h ^ 2^a
            for (int k0 = 0; k0 < nlh; k0 += kGathers) {
                T v[kGathers];
                bool ok[kGathers];
#pragma unroll
                for (int u = 0; u < kGathers; u++) {
                    const int k = k0 + u;
                    ok[u] = false;
                    if (k < nlh) {
                        const uint32_t b = hb.lh_b[k], need = hb.lh_need[k];
                        ok[u] = ((l >> b) & 1u) == need;
                        if (ok[u]) {
                            uint32_t r;
                            if constexpr (TAB) {
                                r = __ldg(P.flipq + ((uint32_t)hb.lh_bi[k] * L32 + cp));
                            } else {
                                const uint32_t l2 = l ^ (1u << b);
                                const uint16_t *t2x = need ? t2m : t2p;
                                r = t1[l2 & 255u] + t2x[l2 >> 8];
                            }
                            v[u] = gload<T>(X + ((uint32_t)hb.lh_base[k] + r) * ld, hb.lh_outer[k] ? stream : keep);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kGathers; u++)
                    if (ok[u]) acc = fma(hb.lh_coef[k0 + u], v[u], acc);
            }
            T out = al * acc;
            T *yr = a.y + row * ld;
            if (use_beta) out = fma(be, cload<T>(yr, stream), out);
            if (use_v) out = fma(ga, cload<T>(a.v + row * ld, stream), out);
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
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int nwarp = kStagedThreads / 32;
#pragma unroll
        for (int r = 0; r < NR; r++) {
            double val = racc[r].value();
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
            if (lane == 0) red_sm[warp * 3 + r] = val;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            const int r = threadIdx.x;
            double s = 0.0;
            if (r < NR)
                for (int w = 0; w < nwarp; w++) s += red_sm[w * 3 + r];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol] = s;
        }
    }
}

template <typename T, int RED, int TAB, int MINB>
int go_s(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, uint32_t xs_len, int *grid_out) {
    const size_t dyn = ((xs_len * sizeof(T) + 15) & ~(size_t)15) + 3 * (kStagedThreads / 32) * sizeof(double);
    const int occ = dyn_occupancy(ctx, (const void *)k_hvs<T, RED, TAB, MINB>, kStagedThreads, dyn);
    if (occ < 1) return set_err(ctx, HPHI_E_INVAL, "staged H*x: a row block does not fit in shared memory");
    int64_t g = (int64_t)occ * ctx->sm_count;
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    *grid_out = (int)g;
    const int slot = prof_begin(ctx, PROF_HV);
    k_hvs<T, RED, TAB, MINB><<<(int)g, kStagedThreads, dyn, ctx->stream>>>(a, xs_len);
    snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_hvs<%s,RED%d,TAB%d,MINB%d>@" HPHI_SRC_TAG, tname<T>(), RED, TAB, MINB);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace

// Largest row block: of a spin sector, the class of popcount closest to half of
// the low bits; of a Hubbard model, the D_dn rows of one up string.
uint32_t staged_block_len(const hphi_ham *ham) {
    if (ham->model == HPHI_HUBBARD) return (uint32_t)ham->basis->sp[1].dim;  // D_dn rows per up string
    const std::vector<uint32_t> &lo = ham->basis->sp[0].loff_h;
    uint32_t m = 0;
    for (size_t p = 0; p + 1 < lo.size(); p++) m = lo[p + 1] - lo[p] > m ? lo[p + 1] - lo[p] : m;
    return m;
}

template <typename T, int TAB, int MINB>
int staged_red(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, uint32_t xl, int red_mode, int *grid) {
    switch (red_mode) {
    case 0: return go_s<T, 0, TAB, MINB>(ctx, ham, a, xl, grid);
    case 1: return go_s<T, 1, TAB, MINB>(ctx, ham, a, xl, grid);
    case 2: return go_s<T, 2, TAB, MINB>(ctx, ham, a, xl, grid);
    case 3: return go_s<T, 3, TAB, MINB>(ctx, ham, a, xl, grid);
    default: return HPHI_E_INVAL;
    }
}

template <typename T>
int launch_staged(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid) {
    const uint32_t xl = staged_block_len(ham);
    // tune_staged_lists: bit 0 = the list form (needs the packed low-low lists), bit 1 =
    // registers sized for one more thread block per SM
    // automatic form (measured on the 6x5 and 4x8 sectors): FP32 lists with registers for
    // 3 blocks per SM (-23 %), FP64 rank tables with registers for 2 (-7 to -27 %)
    const int form = ham->tune_staged_lists >= 0 ? ham->tune_staged_lists : (std::is_same<T, float>::value ? 3 : 2);
    const bool lists = (form & 1) && a.P.ll_pk;
    const bool more = (form & 2) != 0;
    if constexpr (std::is_same<T, float>::value) {
        if (more) return lists ? staged_red<T, 1, 3>(ctx, ham, a, xl, red_mode, grid)
                               : staged_red<T, 0, 3>(ctx, ham, a, xl, red_mode, grid);
        return lists ? staged_red<T, 1, 2>(ctx, ham, a, xl, red_mode, grid)
                     : staged_red<T, 0, 2>(ctx, ham, a, xl, red_mode, grid);
    } else {
        if (more) return lists ? staged_red<T, 1, 2>(ctx, ham, a, xl, red_mode, grid)
                               : staged_red<T, 0, 2>(ctx, ham, a, xl, red_mode, grid);
        return lists ? staged_red<T, 1, 1>(ctx, ham, a, xl, red_mode, grid)
                     : staged_red<T, 0, 1>(ctx, ham, a, xl, red_mode, grid);
    }
}

template int launch_staged<float>(hphi_ctx *, const hphi_ham *, const HvArgs<float> &, int, int *);
template int launch_staged<double>(hphi_ctx *, const hphi_ham *, const HvArgs<double> &, int, int *);

}  // namespace hphi
