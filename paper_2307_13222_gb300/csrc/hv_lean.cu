// Lean H*x kernel: one thread per row, CPL consecutive columns per thread.
//
// It computes what the generic kernel computes (hv.cu) for the common shapes:
// x, y and v share one leading dimension, and the reductions are one of the
// driver patterns (none; <x,y>; <x,Hx> |Hx|^2 |x|^2; |y|^2).  Differences that
// make it cheaper:
//   * the leading dimension (1, 2 or 32) and the reduction pattern are template
//     constants, so the row loop carries no runtime switches;
//   * 32-bit element offsets: a gather address is one wide multiply-add, and
//     four gathers are issued before any is used;
//   * L2 eviction priorities: gathered x lines are kept (evict_last) because
//     neighbouring row blocks read them again, while the streaming y / v lines
//     are marked evict_first so they do not push x out of L2.
#include "hvcommon.cuh"

namespace hphi {

namespace {

__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_normal() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// read-only gathers of x (non-coherent path, L2 priority hint)
template <typename T, int CPL>
__device__ __forceinline__ void ld_keep(const T *p, uint64_t pol, T (&v)[CPL]) {
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[0]) : "l"(p), "l"(pol));
        } else if constexpr (CPL == 2) {
            asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v[0]), "=f"(v[1]) : "l"(p), "l"(pol));
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 4)
                asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                    : "=f"(v[k]), "=f"(v[k + 1]), "=f"(v[k + 2]), "=f"(v[k + 3])
                    : "l"(p + k), "l"(pol));
        }
    } else {
        if constexpr (CPL == 1) {
            asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v[0]) : "l"(p), "l"(pol));
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 2)
                asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                    : "=d"(v[k]), "=d"(v[k + 1])
                    : "l"(p + k), "l"(pol));
        }
    }
}

// coherent streaming loads (v may alias y) and stores; volatile keeps their order
template <typename T, int CPL>
__device__ __forceinline__ void ld_stream(const T *p, uint64_t pol, T (&v)[CPL]) {
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[0]) : "l"(p), "l"(pol) : "memory");
        } else if constexpr (CPL == 2) {
            asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                         : "=f"(v[0]), "=f"(v[1])
                         : "l"(p), "l"(pol)
                         : "memory");
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 4)
                asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                             : "=f"(v[k]), "=f"(v[k + 1]), "=f"(v[k + 2]), "=f"(v[k + 3])
                             : "l"(p + k), "l"(pol)
                             : "memory");
        }
    } else {
        if constexpr (CPL == 1) {
            asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v[0]) : "l"(p), "l"(pol) : "memory");
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 2)
                asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                             : "=d"(v[k]), "=d"(v[k + 1])
                             : "l"(p + k), "l"(pol)
                             : "memory");
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void st_stream(T *p, uint64_t pol, const T (&v)[CPL]) {
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v[0]), "l"(pol) : "memory");
        } else if constexpr (CPL == 2) {
            asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v[0]), "f"(v[1]),
                         "l"(pol)
                         : "memory");
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 4)
                asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p + k), "f"(v[k]),
                             "f"(v[k + 1]), "f"(v[k + 2]), "f"(v[k + 3]), "l"(pol)
                             : "memory");
        }
    } else {
        if constexpr (CPL == 1) {
            asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v[0]), "l"(pol) : "memory");
        } else {
#pragma unroll
            for (int k = 0; k < CPL; k += 2)
                asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p + k), "d"(v[k]),
                             "d"(v[k + 1]), "l"(pol)
                             : "memory");
        }
    }
}

constexpr int kGather = 4;  // gathers in flight per chunk

// RED: 0 none; 1 <x,y>; 2 <x,Hx>, |Hx|^2, |x|^2; 3 |y|^2.  Element offsets are
// 32-bit (the launcher checks D * ld < 2^32) so that every gather address is a
// single wide multiply-add from the vector base.  One thread per row; the
// neighbours of a row are taken in chunks of four gathers issued together.
template <typename T, int CPL, int LDC, int RED>
__global__ void __launch_bounds__(kThreads, (CPL >= 4 || sizeof(T) == 8) ? 2 : 3) k_hvl(const HvArgs<T> a) {
    extern __shared__ double red_sm[];  // [nwarps][3][CPL]
    __shared__ HBlock<T> hb;
    __shared__ T coef_sm[kMaxCoef];
    const HvTables &P = a.P;
    const HamDesc &D = *P.desc;
    for (int i = threadIdx.x; i < D.n_ncoef; i += blockDim.x) coef_sm[i] = (T)D.coef[i];
    const uint32_t ld = LDC > 0 ? (uint32_t)LDC : (uint32_t)a.ldx;
    const uint32_t L32 = (uint32_t)P.L;
    const uint64_t keep = P.hints ? policy_keep() : policy_normal();
    const uint64_t stream = P.hints ? policy_stream() : policy_normal();
    const int split = P.split, sub = blockIdx.x % split;
    const int64_t nbg = gridDim.x / split;  // row blocks in flight
    T al[CPL], ga[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k++) {
        al[k] = (T)(a.alpha_dev ? a.alpha_dev[k] : a.alpha[k]);
        ga[k] = (T)(a.gamma_dev ? a.gamma_dev[k] : a.gamma[k]);
    }
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    RedAcc<T> racc[NR > 0 ? NR : 1][CPL];
    const T *__restrict__ dlow = (const T *)P.dlow;
    const T *__restrict__ X = a.x;

    for (int64_t c = blockIdx.x / split; c < P.nh; c += nbg) {
        const int64_t h = block_of(P, c);
        __syncthreads();  // the previous block's rows are done with hb
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base;
        const uint32_t len = hb.len, cp0 = hb.cp0;
        const int nhh = hb.nhh, nlh = hb.nlh;
        for (uint32_t q = threadIdx.x + sub * kThreads; q < len; q += split * kThreads) {
            const uint32_t cp = cp0 + q;
            uint32_t l;
            if (P.model == kSpin) l = __ldg(P.lstate + cp);
            else if (P.model == kSpinGC) l = q;
            else l = __ldg(P.states_dn + q);
            const int cnt = __ldg(P.ll_cnt + cp);
            T d = __ldg(dlow + cp) + hb.dh;
            for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
            const uint32_t roff = (base + q) * ld;
            T xo[CPL], acc[CPL];
            ld_keep<T, CPL>(X + roff, keep, xo);
#pragma unroll
            for (int k = 0; k < CPL; k++) acc[k] = d * xo[k];
            // high-high neighbours (up hops): fixed row offsets of this block
            for (int k0 = 0; k0 < nhh; k0 += kGather) {
                T v[kGather][CPL], cc[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    const int k = k0 + u;
                    if (k < nhh) {
                        cc[u] = hb.hh_coef[k];
                        const uint32_t t = roff + (uint32_t)hb.hh_delta[k] * ld;
                        ld_keep<T, CPL>(X + t, hb.hh_outer[k] ? stream : keep, v[u]);
                    } else {
                        cc[u] = (T)0;
#pragma unroll
                        for (int j = 0; j < CPL; j++) v[u][j] = (T)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < kGather; u++)
#pragma unroll
                    for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            // low-low neighbours (down hops): ELL lists of this low half
            for (int e0 = 0; e0 < cnt; e0 += kGather) {
                uint32_t tg[kGather], cf[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    const uint32_t e = (uint32_t)(e0 + u);
                    if ((int)e < cnt) {
                        const uint32_t off = e * L32 + cp;
                        if (P.ll_pk) {
                            const uint32_t pk = __ldg(P.ll_pk + off);
                            tg[u] = pk & 0xFFFFFFu;
                            cf[u] = pk >> 24;
                        } else {
                            tg[u] = __ldg(P.ll_tgt + off);
                            cf[u] = __ldg(P.ll_cf + off);
                        }
                    }
                }
                T v[kGather][CPL], cc[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    if (e0 + u < cnt) {
                        cc[u] = coef_sm[cf[u]];
                        ld_keep<T, CPL>(X + (base + tg[u]) * ld, keep, v[u]);
                    } else {
                        cc[u] = (T)0;
#pragma unroll
                        for (int j = 0; j < CPL; j++) v[u][j] = (T)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < kGather; u++)
#pragma unroll
                    for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            // mixed bonds: the low bit must match, the target block is h ^ bit a
            for (int k0 = 0; k0 < nlh; k0 += kGather) {
                uint32_t tq[kGather];
                bool ok[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    const int k = k0 + u;
                    ok[u] = k < nlh && ((l >> hb.lh_b[k]) & 1u) == hb.lh_need[k];
                    if (ok[u]) tq[u] = __ldg(P.flipq + ((uint32_t)hb.lh_bi[k] * L32 + cp));
                }
                T v[kGather][CPL], cc[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    if (ok[u]) {
                        cc[u] = hb.lh_coef[k0 + u];
                        const uint32_t t = ((uint32_t)hb.lh_base[k0 + u] + tq[u]) * ld;
                        ld_keep<T, CPL>(X + t, hb.lh_outer[k0 + u] ? stream : keep, v[u]);
                    } else {
                        cc[u] = (T)0;
#pragma unroll
                        for (int j = 0; j < CPL; j++) v[u][j] = (T)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < kGather; u++)
#pragma unroll
                    for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            // epilogue: out = alpha H x (+ beta y) (+ gamma v)
            T out[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) out[k] = al[k] * acc[k];
            if constexpr (CPL % 2 == 0) {
                if (a.swap) {
#pragma unroll
                    for (int k = 0; k < CPL; k++) out[k] = al[k] * acc[k ^ 1];
                }
            }
            T *yr = a.y + roff;
            if (use_beta) {
                T yo[CPL];
                ld_stream<T, CPL>(yr, stream, yo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(be, yo[k], out[k]);
            }
            if (use_v) {
                T vo[CPL];
                ld_stream<T, CPL>(a.v + roff, stream, vo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(ga[k], vo[k], out[k]);
            }
            st_stream<T, CPL>(yr, stream, out);
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                if constexpr (RED == 1) racc[0][k].add(xo[k], out[k]);
                if constexpr (RED == 2) {
                    racc[0][k].add(xo[k], acc[k]);
                    racc[1][k].add(acc[k], acc[k]);
                    racc[2][k].add(xo[k], xo[k]);
                }
                if constexpr (RED == 3) racc[0][k].add(out[k], out[k]);
            }
        }
    }
    if constexpr (RED != 0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int nwarp = kThreads / 32;
#pragma unroll
        for (int r = 0; r < NR; r++) {
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                double val = racc[r][k].value();
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                if (lane == 0) red_sm[(warp * 3 + r) * CPL + k] = val;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * CPL; t += blockDim.x) {
            const int r = t / CPL, c = t % CPL;
            double s = 0.0;
            if (r < NR)
                for (int w = 0; w < nwarp; w++) s += red_sm[(w * 3 + r) * CPL + c];
            a.partials[((int64_t)blockIdx.x * 3 + r) * CPL + c] = s;
        }
    }
}

template <typename T, int CPL, int LDC, int RED>
int go(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int *grid_out) {
    const size_t dyn = RED ? 3 * (kThreads / 32) * CPL * sizeof(double) : 0;
    const int occ = dyn_occupancy(ctx, (const void *)k_hvl<T, CPL, LDC, RED>, kThreads, dyn);
    // a multiple of the split: `split` consecutive thread blocks share a row block
    const int split = a.P.split;
    int64_t g = (int64_t)(occ > 0 ? occ : 1) * ctx->sm_count / split;
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    g *= split;
    *grid_out = (int)g;
    const int slot = prof_begin(ctx, PROF_HV);
    k_hvl<T, CPL, LDC, RED><<<(int)g, kThreads, dyn, ctx->stream>>>(a);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

template <typename T, int CPL, int LDC>
int go_red(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid) {
    switch (red_mode) {
    case 0: return go<T, CPL, LDC, 0>(ctx, ham, a, grid);
    case 1: return go<T, CPL, LDC, 1>(ctx, ham, a, grid);
    case 2: return go<T, CPL, LDC, 2>(ctx, ham, a, grid);
    case 3: return go<T, CPL, LDC, 3>(ctx, ham, a, grid);
    default: return HPHI_E_INVAL;
    }
}

}  // namespace

template <typename T>
int launch_lean(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int cpl, int ldc, int red_mode, int *grid) {
    constexpr int WIDE = std::is_same<T, float>::value ? 8 : 4;  // 32-byte rows of a 32-column slice
    if (cpl == 1 && ldc == 1) return go_red<T, 1, 1>(ctx, ham, a, red_mode, grid);
    if (cpl == 1 && ldc == 0) return go_red<T, 1, 0>(ctx, ham, a, red_mode, grid);
    if (cpl == 2 && ldc == 2) return go_red<T, 2, 2>(ctx, ham, a, red_mode, grid);
    if (cpl == WIDE && ldc == 32) return go_red<T, WIDE, 32>(ctx, ham, a, red_mode, grid);
    return HPHI_E_INVAL;
}

template int launch_lean<float>(hphi_ctx *, const hphi_ham *, const HvArgs<float> &, int, int, int, int *);
template int launch_lean<double>(hphi_ctx *, const hphi_ham *, const HvArgs<double> &, int, int, int, int *);

}  // namespace hphi
