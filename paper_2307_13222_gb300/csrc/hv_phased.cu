// Bond-major H*x kernel for the spin-1/2 S^z sector and for Hubbard models,
// one column.
//
// Like the staged kernel, the thread block that owns row block h (the states
// with high half h: rows base .. base + len - 1, low halves of popcount p)
// first copies the block's slice of x into shared memory.  It then builds
// (H x) of the block in a second shared array, one bond at a time:
//   1. the diagonal and the high-high bonds, two rows per lane at a time
//      (their targets sit at the same row offset in block h ^ m: coalesced);
//   2. each low-low bond k = (i, j): acc[q] += c_k xs[q'] over the list of the
//      rows of class p whose bits i and j differ, q' = Lin's rank of the
//      flipped low half (same class, so the target is in shared memory);
//   3. each mixed bond (a, b): acc[q] += c x[jb(h ^ 2^a) + r] over the list of
//      the rows whose bit b equals 1 - h_a, r = rank of l ^ 2^b in class p -+ 1
//      (ascending in q, so a warp's loads walk the target block in order);
//   4. the epilogue y = alpha acc + beta y + gamma v with the fused reductions.
// The lists hold only applicable (row, target) pairs, built once per
// Hamiltonian on the host: no lane tests a bond, and none idles on a bond that
// does not apply to its row.  Within one phase each row occurs at most once.
// Warp w owns a fixed range of the block's rows in every phase (the lists
// carry offsets at the range boundaries), so consecutive phases are ordered by
// __syncwarp() alone.  Every row sums its terms in a fixed order, so results
// are deterministic.  (Sec. 3.1.1 and Sec. 5: the spin-1/2 exchange terms and
// their action on the bit-encoded basis.)  Hubbard models take the same path
// with row block = the D_dn rows of one up string: phase 1 carries the
// diagonal and the up hops (whole-block moves with the up string's sign),
// phase 2 the down hops, one list per (hop pair, fermion sign) coefficient;
// there is no phase 3.
#include "hvcommon.cuh"

namespace hphi {

namespace {

constexpr int kPhUnroll = 4;   // list entries in flight per lane (mixed phase; FP64 low-low phase)
// low-low phase: FP32 takes 8 entries per lane per batch (measured 1.7 % faster)
template <typename T> constexpr int kPhUnrollLL = sizeof(T) == 4 ? 8 : 4;
constexpr int kPhGathers = 4;  // high-high gathers in flight per row
constexpr int kPhMaxLL = 128;

// U list entries of one low-low bond per lane (entry i = first + 32 u): acs[q] += c xs[q'].
template <typename T, int U, bool PRED>
__device__ __forceinline__ void ll_batch(const uint32_t *__restrict__ ent, int32_t first, int32_t end, T c,
                                         const T *xs, T *acs) {
    uint32_t pk[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int32_t i = first + 32 * u;
        pk[u] = (!PRED || i < end) ? __ldg(ent + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
        if (!PRED || first + 32 * u < end) {
            const uint32_t q = pk[u] & 0xFFFFu;
            acs[q] = fma(c, xs[pk[u] >> 16], acs[q]);
        }
}

template <typename T, int NT, int RED, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_hvp(const HvArgs<T> a, uint32_t xs_len) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *xs = (T *)s_raw;
    T *acs = xs + xs_len;
    double *red_sm = (double *)(s_raw + ((2 * (size_t)xs_len * sizeof(T) + 15) & ~(size_t)15));
    __shared__ HBlock<T> hb;
    __shared__ T ll_c[kPhMaxLL];
    const HvTables &P = a.P;
    const HamDesc &D = *P.desc;
    // Hubbard: the low-low lists are the down hops, one list per coefficient
    // (hop pair and fermion sign), all in one class (p = 0)
    const bool hub = P.model == kHubbard;
    const int nll = hub ? D.n_ncoef : D.n_ll;
    for (int i = threadIdx.x; i < nll; i += NT) ll_c[i] = (T)(hub ? D.coef[i] : D.ll[i].cxy);
    const uint64_t keep = spol(P.hints, 0), stream = spol(P.hints, 1);
    const T al = (T)(a.alpha_dev ? a.alpha_dev[0] : a.alpha[0]);
    const T ga = (T)(a.gamma_dev ? a.gamma_dev[0] : a.gamma[0]);
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    constexpr int W = NT / 32, RPW = kPhRanges / W;
    static_assert(kPhRanges % W == 0, "row ranges must split evenly over the warps");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *__restrict__ dlow = (const T *)P.dlow;
    const T *__restrict__ X = a.x;
    constexpr uint32_t ld = 1;  // x, y and v are contiguous vectors (the launcher checks)
    const uint32_t *__restrict__ ent = P.ph_ent;
    constexpr int OS = kPhRanges + 1;  // offsets per list group
    // reductions: each warp folds its rows of a block into its slots of red_sm
    // (lane 0 owns them), so no accumulator stays live through the bond phases
    if (RED != 0 && lane == 0)
        for (int r = 0; r < 3; r++) red_sm[warp * 3 + r] = 0.0;

    for (int64_t c = blockIdx.x; c < P.nh; c += gridDim.x) {
        const int64_t h = block_of(P, c);
        __syncthreads();  // the previous block is done with hb, xs and acs
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base, len = hb.len, cp0 = hb.cp0;
        const int p = hub ? 0 : P.n - __popcll((unsigned long long)h);
        for (uint32_t q = threadIdx.x; q < len; q += NT) xs[q] = gload<T>(X + (base + q) * ld, keep);
        __syncthreads();
        const uint32_t q0 = (uint32_t)(((uint64_t)len * (uint32_t)(warp * RPW)) / kPhRanges);
        const uint32_t q1 = (uint32_t)(((uint64_t)len * (uint32_t)((warp + 1) * RPW)) / kPhRanges);
        // 1. diagonal and high-high bonds, two rows per lane at a time (twice the
        // gathers in flight); with a.tin the high-high terms come precomputed
        const int nhh = a.tin ? 0 : hb.nhh;
        for (uint32_t q = q0 + lane; q < q1; q += 64) {
            const bool two = q + 32 < q1;
            T acc[2];
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const uint32_t qq = q + 32 * t;
                acc[t] = 0;
                if (t == 0 || two) {
                    const uint32_t cp = cp0 + qq;
                    const uint32_t l = hub ? __ldg(P.states_dn + qq) : __ldg(P.lstate + cp);
                    T d = __ldg(dlow + cp) + hb.dh;
                    for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
                    acc[t] = a.tin ? fma(d, xs[qq], a.tin[base + qq]) : d * xs[qq];
                }
            }
            for (int k0 = 0; k0 < nhh; k0 += kPhGathers) {
                T v[2][kPhGathers];
#pragma unroll
                for (int u = 0; u < kPhGathers; u++) {
                    const int k = k0 + u;
                    if (k < nhh) {
                        const uint32_t off = (uint32_t)hb.hh_delta[k];
                        const uint64_t pol = hb.hh_outer[k] ? stream : keep;
                        v[0][u] = gload<T>(X + (base + q + off) * ld, pol);
                        if (two) v[1][u] = gload<T>(X + (base + q + 32 + off) * ld, pol);
                    }
                }
#pragma unroll
                for (int u = 0; u < kPhGathers; u++)
                    if (k0 + u < nhh) {
                        const T c = hb.hh_coef[k0 + u];
                        acc[0] = fma(c, v[0][u], acc[0]);
                        if (two) acc[1] = fma(c, v[1][u], acc[1]);
                    }
            }
            acs[q] = acc[0];
            if (two) acs[q + 32] = acc[1];
        }
        __syncwarp();
        // 2. low-low bonds, targets in shared memory.  Lane j holds the list range
        // of bond k0 + j; the bond loop takes it by shuffle.
        for (int k0 = 0; k0 < nll; k0 += 32) {
            int32_t my0 = 0, my1 = 0;
            if (k0 + lane < nll) {
                const int32_t *o = P.ph_off + ((int64_t)p * nll + k0 + lane) * OS + warp * RPW;
                my0 = __ldg(o);
                my1 = __ldg(o + RPW);
            }
            const int kn = nll - k0 < 32 ? nll - k0 : 32;
            for (int j = 0; j < kn; j++) {
                const int32_t s0 = __shfl_sync(0xffffffffu, my0, j), s1 = __shfl_sync(0xffffffffu, my1, j);
                if (s0 == s1) continue;
                const T ck = ll_c[k0 + j];
                // full batches of kPhUnrollLL entries per lane, then halving batches,
                // then one predicated batch of two: no lane slot idles in a batch but
                // the last (a row occurs once per bond, so batches need no ordering)
                int32_t b = s0;
                for (; b + 32 * kPhUnrollLL<T> <= s1; b += 32 * kPhUnrollLL<T>)
                    ll_batch<T, kPhUnrollLL<T>, false>(ent, b + lane, s1, ck, xs, acs);
                if (kPhUnrollLL<T> > 4 && b + 128 <= s1) {
                    ll_batch<T, 4, false>(ent, b + lane, s1, ck, xs, acs);
                    b += 128;
                }
                if (b + 64 <= s1) {
                    ll_batch<T, 2, false>(ent, b + lane, s1, ck, xs, acs);
                    b += 64;
                }
                if (b < s1) ll_batch<T, 2, true>(ent, b + lane, s1, ck, xs, acs);
                __syncwarp();
            }
        }
        // 3. mixed bonds, targets in block h ^ 2^a.  Lane j holds the list range
        // of mixed bond k0 + j of this block; the loop walks the batches of all
        // of them in order, loading the next batch's entries before it gathers
        // and adds the current one (the first batch of a bond no longer waits for
        // its list after the previous bond ends).
        const int nlh = hb.nlh;
        for (int k0 = 0; k0 < nlh; k0 += 32) {
            int32_t my0 = 0, my1 = 0;
            bool okb = false;
            if (k0 + lane < nlh) {
                const int k = k0 + lane;
                const int g = (p * P.ph_nlb + hb.lh_bi[k]) * 2 + hb.lh_need[k];
                const int32_t *o = P.ph_off + P.ph_mx0 + (int64_t)g * OS + warp * RPW;
                my0 = __ldg(o);
                my1 = __ldg(o + RPW);
                okb = my1 > my0 && hb.lh_base[k] >= 0;
            }
            unsigned ne = __ballot_sync(0xffffffffu, okb);
            if (!ne) continue;
            int j = __ffs(ne) - 1;
            ne &= ne - 1;
            int32_t b0 = __shfl_sync(0xffffffffu, my0, j), s1 = __shfl_sync(0xffffffffu, my1, j);
            uint32_t pk[kPhUnroll];
#pragma unroll
            for (int u = 0; u < kPhUnroll; u++) {
                const int32_t i = b0 + lane + 32 * u;
                pk[u] = i < s1 ? __ldg(ent + i) : 0u;
            }
            while (true) {
                int jn = j;
                int32_t bn = b0 + 32 * kPhUnroll, s1n = s1;
                bool more = true, sw = false;
                if (bn >= s1) {
                    if (ne) {
                        jn = __ffs(ne) - 1;
                        ne &= ne - 1;
                        bn = __shfl_sync(0xffffffffu, my0, jn);
                        s1n = __shfl_sync(0xffffffffu, my1, jn);
                        sw = true;
                    } else {
                        more = false;
                    }
                }
                const int k = k0 + j;
                const T cf = hb.lh_coef[k];
                const uint32_t b2 = (uint32_t)hb.lh_base[k];
                const uint64_t pol = hb.lh_outer[k] ? stream : keep;
                T v[kPhUnroll];
#pragma unroll
                for (int u = 0; u < kPhUnroll; u++)
                    if (b0 + lane + 32 * u < s1) v[u] = gload<T>(X + (b2 + (pk[u] >> 16)) * ld, pol);
                uint32_t pn[kPhUnroll];
#pragma unroll
                for (int u = 0; u < kPhUnroll; u++) {
                    const int32_t i = bn + lane + 32 * u;
                    pn[u] = (more && i < s1n) ? __ldg(ent + i) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kPhUnroll; u++)
                    if (b0 + lane + 32 * u < s1) {
                        const uint32_t q = pk[u] & 0xFFFFu;
                        acs[q] = fma(cf, v[u], acs[q]);
                    }
                if (!more) {
                    __syncwarp();
                    break;
                }
                if (sw) __syncwarp();
                j = jn;
                b0 = bn;
                s1 = s1n;
#pragma unroll
                for (int u = 0; u < kPhUnroll; u++) pk[u] = pn[u];
            }
        }
        // 4. epilogue over the warp's rows
        RedAcc<T> racc[NR > 0 ? NR : 1];
        for (uint32_t q = q0 + lane; q < q1; q += 32) {
            const T acc = acs[q];
            const T xo = xs[q];
            const uint32_t row = base + q;
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
        if constexpr (RED != 0) {
#pragma unroll
            for (int r = 0; r < NR; r++) {
                double val = racc[r].value();
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                if (lane == 0) red_sm[warp * 3 + r] += val;
            }
        }
    }
    if constexpr (RED != 0) {
        __syncthreads();
        if (threadIdx.x < 3) {
            const int r = threadIdx.x;
            double s = 0.0;
            if (r < NR)
                for (int w = 0; w < W; w++) s += red_sm[w * 3 + r];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol] = s;
        }
    }
}

template <typename T, int NT, int RED, int MINB>
int go_p(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, uint32_t xs_len, int *grid_out) {
    const size_t dyn = ((2 * (size_t)xs_len * sizeof(T) + 15) & ~(size_t)15) + 3 * (NT / 32) * sizeof(double);
    const int occ = dyn_occupancy(ctx, (const void *)k_hvp<T, NT, RED, MINB>, NT, dyn);
    if (occ < 1) return set_err(ctx, HPHI_E_INVAL, "bond-major H*x: a row block does not fit in shared memory");
    int64_t g = (int64_t)occ * ctx->sm_count;
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    *grid_out = (int)g;
    const int slot = prof_begin(ctx, PROF_HV);
    k_hvp<T, NT, RED, MINB><<<(int)g, NT, dyn, ctx->stream>>>(a, xs_len);
    snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_hvp<%s,%d,RED%d,MINB%d>@" HPHI_SRC_TAG, tname<T>(), NT, RED, MINB);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace

// FP32: 512 threads with registers for two blocks per SM (x and the
// accumulator of a 12,870-row block take 103 KB of shared memory); FP64: one
// block of 1024 threads (206 KB).
template <typename T>
int launch_phased(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid) {
    const int nlists = ham->model == HPHI_HUBBARD ? ham->host.n_ncoef : ham->host.n_ll;
    if (!a.P.ph_ent || nlists > kPhMaxLL)
        return set_err(ctx, HPHI_E_INVAL, "bond-major H*x: no bond lists for this Hamiltonian");
    if (a.ldx != 1 || a.ldy != 1 || (a.v && a.ldv != 1))
        return set_err(ctx, HPHI_E_INVAL, "bond-major H*x: one contiguous column only");
    const uint32_t xl = staged_block_len(ham);
    constexpr bool F = std::is_same<T, float>::value;
    constexpr int NT = F ? 512 : 1024, MB = F ? 2 : 1;
    switch (red_mode) {
    case 0: return go_p<T, NT, 0, MB>(ctx, ham, a, xl, grid);
    case 1: return go_p<T, NT, 1, MB>(ctx, ham, a, xl, grid);
    case 2: return go_p<T, NT, 2, MB>(ctx, ham, a, xl, grid);
    case 3: return go_p<T, NT, 3, MB>(ctx, ham, a, xl, grid);
    default: return HPHI_E_INVAL;
    }
}

template int launch_phased<float>(hphi_ctx *, const hphi_ham *, const HvArgs<float> &, int, int *);
template int launch_phased<double>(hphi_ctx *, const hphi_ham *, const HvArgs<double> &, int, int *);

}  // namespace hphi
