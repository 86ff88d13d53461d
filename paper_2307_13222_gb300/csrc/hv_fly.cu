// H*x kernel for spin models with neighbour ranks computed on the fly.
//
// A row is (h, l).  Its neighbours are
//   high-high bond b:  row + (jb[h ^ m_b] - jb[h])          (per block, shared memory)
//   low-low bond b:    jb[h] + ja[l ^ m_b]                   if bits i, j of l differ
//   mixed bond (a,b):  jb[h ^ 2^a] + ja[l ^ 2^b]             if bit b of l equals 1 - bit a of h
// (full space: ja[l] = l, jb[h] = h << N_lo).  Lin's ja is a 2^N_lo table of
// 16-bit ranks (128 KB at N_lo = 16) that stays in L1, so each gather needs
// one trip to L2/DRAM instead of a table trip followed by the gather.
// G lanes share a row and split its columns (CPL each); 8 gathers are issued
// before any is used.  Same epilogue and reductions as the other kernels.
#include "hvcommon.cuh"

namespace hphi {

namespace {

__device__ __forceinline__ uint64_t pol_of(int hints, int kind) {
    uint64_t p;
    if (!hints) asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    else if (kind) asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

template <typename T, int CPL>
__device__ __forceinline__ void gld(const T *p, uint64_t pol, T (&v)[CPL]) {
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[0]) : "l"(p), "l"(pol));
        } else if constexpr (CPL == 2) {
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                : "=f"(v[0]), "=f"(v[1])
                : "l"(p), "l"(pol));
        } else {
            static_assert(CPL == 4, "float columns per lane: 1, 2 or 4");
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                : "l"(p), "l"(pol));
        }
    } else {
        if constexpr (CPL == 1) {
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v[0]) : "l"(p), "l"(pol));
        } else {
            static_assert(CPL == 2, "double columns per lane: 1 or 2");
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                : "=d"(v[0]), "=d"(v[1])
                : "l"(p), "l"(pol));
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void sld(const T *p, uint64_t pol, T (&v)[CPL]) {  // coherent (may alias y)
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[0]) : "l"(p), "l"(pol) : "memory");
        } else if constexpr (CPL == 2) {
            asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                         : "=f"(v[0]), "=f"(v[1])
                         : "l"(p), "l"(pol)
                         : "memory");
        } else {
            asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                         : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                         : "l"(p), "l"(pol)
                         : "memory");
        }
    } else {
        if constexpr (CPL == 1) {
            asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v[0]) : "l"(p), "l"(pol) : "memory");
        } else {
            asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                         : "=d"(v[0]), "=d"(v[1])
                         : "l"(p), "l"(pol)
                         : "memory");
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void sst(T *p, uint64_t pol, const T (&v)[CPL]) {
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (CPL == 1) {
            asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v[0]), "l"(pol) : "memory");
        } else if constexpr (CPL == 2) {
            asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v[0]), "f"(v[1]),
                         "l"(pol)
                         : "memory");
        } else {
            asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v[0]),
                         "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol)
                         : "memory");
        }
    } else {
        if constexpr (CPL == 1) {
            asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v[0]), "l"(pol) : "memory");
        } else {
            asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v[0]), "d"(v[1]),
                         "l"(pol)
                         : "memory");
        }
    }
}

constexpr int kMaxLLs = 128;  // low-low bonds kept in shared memory

template <typename T, int CPL, int G, int RED>
__global__ void __launch_bounds__(kThreads, (CPL == 1 && sizeof(T) == 4) ? 3 : 2) k_hvo(const HvArgs<T> a) {
    extern __shared__ double red_sm[];  // [nwarps][3][G*CPL]
    __shared__ HBlock<T> hb;
    __shared__ uint32_t ll_m[kMaxLLs];
    __shared__ T ll_c[kMaxLLs];
    const HvTables &P = a.P;
    const HamDesc &D = *P.desc;
    const int nll = D.n_ll < kMaxLLs ? D.n_ll : kMaxLLs;
    for (int i = threadIdx.x; i < nll; i += blockDim.x) {
        ll_m[i] = (1u << D.ll[i].i) | (1u << D.ll[i].j);
        ll_c[i] = (T)D.ll[i].cxy;
    }
    const bool sector = P.model == kSpin;
    const uint32_t ld = (uint32_t)a.ldx;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    constexpr int ngrp = kThreads / G;
    const uint32_t col0 = (uint32_t)(gl * CPL);
    const bool act = (int)col0 < a.ncol;
    const uint64_t keep = pol_of(P.hints, 0), stream = pol_of(P.hints, 1);
    const int split = P.split, sub = blockIdx.x % split;
    const int64_t nbg = gridDim.x / split;
    T al[CPL], ga[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k++) {
        const int c = (int)col0 + k < a.ncol ? (int)col0 + k : 0;
        al[k] = (T)(a.alpha_dev ? a.alpha_dev[c] : a.alpha[c]);
        ga[k] = (T)(a.gamma_dev ? a.gamma_dev[c] : a.gamma[c]);
    }
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    RedAcc<T> racc[NR > 0 ? NR : 1][CPL];
    const T *__restrict__ dlow = (const T *)P.dlow;
    const T *__restrict__ X = a.x;
    const uint16_t *__restrict__ ja = P.ja16;
    constexpr int kCh = CPL == 1 ? 8 : 4;  // gathers in flight per chunk

    for (int64_t c = blockIdx.x / split; c < P.nh; c += nbg) {
        const int64_t h = block_of(P, c);
        __syncthreads();
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base, len = hb.len, cp0 = hb.cp0;
        const int nhh = hb.nhh, nlh = hb.nlh;
        for (uint32_t q = grp + sub * ngrp; q < len; q += split * ngrp) {
            const uint32_t cp = cp0 + q;
            const uint32_t l = sector ? __ldg(P.lstate + cp) : q;
            T d = __ldg(dlow + cp) + hb.dh;
            for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
            const uint32_t roff = (base + q) * ld + col0;
            T xo[CPL], acc[CPL];
            if (act) gld<T, CPL>(X + roff, keep, xo);
#pragma unroll
            for (int k = 0; k < CPL; k++) acc[k] = act ? d * xo[k] : (T)0;
            uint32_t t[kCh];
            T cc[kCh];
            bool ok[kCh];
            uint8_t ob[kCh];
            // high-high neighbours
            for (int k0 = 0; k0 < nhh; k0 += kCh) {
#pragma unroll
                for (int u = 0; u < kCh; u++) {
                    const int k = k0 + u;
                    ok[u] = act && k < nhh;
                    if (ok[u]) {
                        t[u] = roff + (uint32_t)hb.hh_delta[k] * ld;
                        cc[u] = hb.hh_coef[k];
                        ob[u] = hb.hh_outer[k];
                    }
                }
                T v[kCh][CPL];
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u]) gld<T, CPL>(X + t[u], ob[u] ? stream : keep, v[u]);
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u])
#pragma unroll
                        for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            // low-low neighbours: same block, rank of l ^ m
            for (int k0 = 0; k0 < nll; k0 += kCh) {
#pragma unroll
                for (int u = 0; u < kCh; u++) {
                    const int k = k0 + u;
                    ok[u] = false;
                    if (act && k < nll) {
                        const uint32_t m = ll_m[k], lm = l & m;
                        ok[u] = lm != 0 && lm != m && ll_c[k] != (T)0;
                        if (ok[u]) {
                            const uint32_t l2 = l ^ m;
                            t[u] = (base + (sector ? (uint32_t)__ldg(ja + l2) : l2)) * ld + col0;
                            cc[u] = ll_c[k];
                        }
                    }
                }
                T v[kCh][CPL];
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u]) gld<T, CPL>(X + t[u], keep, v[u]);
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u])
#pragma unroll
                        for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            // mixed bonds: bit b of l must equal 1 - bit a of h
            for (int k0 = 0; k0 < nlh; k0 += kCh) {
#pragma unroll
                for (int u = 0; u < kCh; u++) {
                    const int k = k0 + u;
                    ok[u] = false;
                    if (act && k < nlh) {
                        const uint32_t b = hb.lh_b[k];
                        ok[u] = ((l >> b) & 1u) == hb.lh_need[k];
                        if (ok[u]) {
                            const uint32_t l2 = l ^ (1u << b);
                            t[u] = ((uint32_t)hb.lh_base[k] + (sector ? (uint32_t)__ldg(ja + l2) : l2)) * ld + col0;
                            cc[u] = hb.lh_coef[k];
                            ob[u] = hb.lh_outer[k];
                        }
                    }
                }
                T v[kCh][CPL];
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u]) gld<T, CPL>(X + t[u], ob[u] ? stream : keep, v[u]);
#pragma unroll
                for (int u = 0; u < kCh; u++)
                    if (ok[u])
#pragma unroll
                        for (int j = 0; j < CPL; j++) acc[j] = fma(cc[u], v[u][j], acc[j]);
            }
            if (!act) continue;
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
                sld<T, CPL>(yr, stream, yo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(be, yo[k], out[k]);
            }
            if (use_v) {
                T vo[CPL];
                sld<T, CPL>(a.v + roff, stream, vo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(ga[k], vo[k], out[k]);
            }
            sst<T, CPL>(yr, stream, out);
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
        constexpr int nwarp = kThreads / 32, W = G * CPL;
#pragma unroll
        for (int r = 0; r < NR; r++) {
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                double val = racc[r][k].value();
#pragma unroll
                for (int off = 16; off >= G; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                if (lane < G) red_sm[(warp * 3 + r) * W + col0 + k] = val;
            }
        }
        __syncthreads();
        for (int tt = threadIdx.x; tt < 3 * W; tt += blockDim.x) {
            const int r = tt / W, cc2 = tt % W;
            if (cc2 >= a.ncol) continue;
            double s = 0.0;
            if (r < NR)
                for (int w = 0; w < nwarp; w++) s += red_sm[(w * 3 + r) * W + cc2];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol + cc2] = s;
        }
    }
}

// Cooperative variant for wide rows: the G lanes of a row group split the
// candidate bonds of the row (high-high list, low-low bonds, mixed bonds),
// each lane evaluates every G-th candidate, the group ballots the applicable
// ones and broadcasts their targets by shuffle, then every lane gathers its
// CPL columns of each target.  The bond work is done once per row instead of
// once per lane.
// KB: targets broadcast and gathered per batch; MINB: thread blocks per SM the
// register budget is sized for (more resident warps, fewer loads in flight each).
template <typename T, int CPL, int G, int RED, int KB, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_hvc(const HvArgs<T> a) {
    extern __shared__ double red_sm[];  // [nwarps][3][G*CPL]
    __shared__ HBlock<T> hb;
    __shared__ uint32_t ll_m[kMaxLLs];
    __shared__ T ll_c[kMaxLLs];
    const HvTables &P = a.P;
    const HamDesc &D = *P.desc;
    const int nll = D.n_ll < kMaxLLs ? D.n_ll : kMaxLLs;
    for (int i = threadIdx.x; i < nll; i += blockDim.x) {
        ll_m[i] = (1u << D.ll[i].i) | (1u << D.ll[i].j);
        ll_c[i] = (T)D.ll[i].cxy;
    }
    const bool sector = P.model == kSpin;
    const uint32_t ld = (uint32_t)a.ldx;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    constexpr int ngrp = kThreads / G;
    const int gbase = (threadIdx.x & 31) - gl;  // first lane of the group in the warp
    const uint32_t col0 = (uint32_t)(gl * CPL);
    const uint64_t keep = pol_of(P.hints, 0), stream = pol_of(P.hints, 1);
    const int split = P.split, sub = blockIdx.x % split;
    const int64_t nbg = gridDim.x / split;
    T al[CPL], ga[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k++) {
        al[k] = (T)(a.alpha_dev ? a.alpha_dev[col0 + k] : a.alpha[col0 + k]);
        ga[k] = (T)(a.gamma_dev ? a.gamma_dev[col0 + k] : a.gamma[col0 + k]);
    }
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    RedAcc<T> racc[NR > 0 ? NR : 1][CPL];
    const T *__restrict__ dlow = (const T *)P.dlow;
    const T *__restrict__ X = a.x;
    const uint16_t *__restrict__ ja = P.ja16;

    for (int64_t c = blockIdx.x / split; c < P.nh; c += nbg) {
        const int64_t h = block_of(P, c);
        __syncthreads();
        setup_block<T>(P, h, hb);
        if (!hb.valid) continue;
        const uint32_t base = (uint32_t)hb.base, len = hb.len, cp0 = hb.cp0;
        const int nhh = hb.nhh, nlh = hb.nlh;
        const int ncand = nhh + nll + nlh;
        // every thread of the block runs the same number of row iterations
        for (uint32_t q0 = sub * ngrp; q0 < len; q0 += split * ngrp) {
            const uint32_t q = q0 + grp;
            const bool rv = q < len;
            const uint32_t cp = cp0 + (rv ? q : 0);
            const uint32_t l = rv ? (sector ? __ldg(P.lstate + cp) : q) : 0;
            T d = rv ? __ldg(dlow + cp) + hb.dh : (T)0;
            for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
            const uint32_t row = base + q;
            const uint32_t roff = row * ld + col0;
            T xo[CPL], acc[CPL];
            if (rv) gld<T, CPL>(X + roff, keep, xo);
#pragma unroll
            for (int k = 0; k < CPL; k++) acc[k] = rv ? d * xo[k] : (T)0;
            for (int r0 = 0; r0 < ncand; r0 += G) {
                // this lane's candidate
                const int k = r0 + gl;
                bool ok = false;
                uint32_t tr = 0;  // target row
                T cf = (T)0;
                int ob = 0;
                if (rv && k < ncand) {
                    if (k < nhh) {
                        ok = true;
                        tr = row + (uint32_t)hb.hh_delta[k];
                        cf = hb.hh_coef[k];
                        ob = hb.hh_outer[k];
                    } else if (k < nhh + nll) {
                        const int kk = k - nhh;
                        const uint32_t m = ll_m[kk], lm = l & m;
                        cf = ll_c[kk];
                        ok = lm != 0 && lm != m && cf != (T)0;
                        if (ok) {
                            const uint32_t l2 = l ^ m;
                            tr = base + (sector ? (uint32_t)__ldg(ja + l2) : l2);
                        }
                    } else {
                        const int kk = k - nhh - nll;
                        const uint32_t b = hb.lh_b[kk];
                        ok = ((l >> b) & 1u) == hb.lh_need[kk];
                        if (ok) {
                            const uint32_t l2 = l ^ (1u << b);
                            tr = (uint32_t)hb.lh_base[kk] + (sector ? (uint32_t)__ldg(ja + l2) : l2);
                            cf = hb.lh_coef[kk];
                            ob = hb.lh_outer[kk];
                        }
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const unsigned gm = (bal >> gbase) & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u));
                // broadcast the group's targets 8 at a time, then gather
                constexpr int kB = G < KB ? G : KB;
#pragma unroll
                for (int s0 = 0; s0 < G; s0 += kB) {
                    uint32_t ts[kB];
                    T cs[kB];
                    int os[kB];
#pragma unroll
                    for (int u = 0; u < kB; u++) {
                        ts[u] = __shfl_sync(0xffffffffu, tr, gbase + s0 + u);
                        cs[u] = __shfl_sync(0xffffffffu, cf, gbase + s0 + u);
                        os[u] = __shfl_sync(0xffffffffu, ob, gbase + s0 + u);
                    }
                    T v[kB][CPL];
#pragma unroll
                    for (int u = 0; u < kB; u++)
                        if ((gm >> (s0 + u)) & 1u) gld<T, CPL>(X + (ts[u] * ld + col0), os[u] ? stream : keep, v[u]);
#pragma unroll
                    for (int u = 0; u < kB; u++)
                        if ((gm >> (s0 + u)) & 1u)
#pragma unroll
                            for (int j = 0; j < CPL; j++) acc[j] = fma(cs[u], v[u][j], acc[j]);
                }
            }
            if (!rv) continue;
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
                sld<T, CPL>(yr, stream, yo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(be, yo[k], out[k]);
            }
            if (use_v) {
                T vo[CPL];
                sld<T, CPL>(a.v + roff, stream, vo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(ga[k], vo[k], out[k]);
            }
            sst<T, CPL>(yr, stream, out);
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
        constexpr int nwarp = kThreads / 32, W = G * CPL;
#pragma unroll
        for (int r = 0; r < NR; r++) {
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                double val = racc[r][k].value();
#pragma unroll
                for (int off = 16; off >= G; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                if (lane < G) red_sm[(warp * 3 + r) * W + col0 + k] = val;
            }
        }
        __syncthreads();
        for (int tt = threadIdx.x; tt < 3 * W; tt += blockDim.x) {
            const int r = tt / W, cc2 = tt % W;
            double s = 0.0;
            if (r < NR)
                for (int w = 0; w < nwarp; w++) s += red_sm[(w * 3 + r) * W + cc2];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol + cc2] = s;
        }
    }
}

template <typename T, int CPL, int G, int RED, int KB, int MINB>
int go_c(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int *grid_out) {
    const size_t dyn = RED ? 3 * (kThreads / 32) * G * CPL * sizeof(double) : 0;
    const int occ = dyn_occupancy(ctx, (const void *)k_hvc<T, CPL, G, RED, KB, MINB>, kThreads, dyn);
    const int split = a.P.split;
    int64_t g = (int64_t)(occ > 0 ? occ : 1) * ctx->sm_count / split;
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    g *= split;
    *grid_out = (int)g;
    const int slot = prof_begin(ctx, PROF_HV);
    k_hvc<T, CPL, G, RED, KB, MINB><<<(int)g, kThreads, dyn, ctx->stream>>>(a);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

template <typename T, int CPL, int G, int KB, int MINB>
int go_c_red(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid) {
    switch (red_mode) {
    case 0: return go_c<T, CPL, G, 0, KB, MINB>(ctx, ham, a, grid);
    case 1: return go_c<T, CPL, G, 1, KB, MINB>(ctx, ham, a, grid);
    case 2: return go_c<T, CPL, G, 2, KB, MINB>(ctx, ham, a, grid);
    case 3: return go_c<T, CPL, G, 3, KB, MINB>(ctx, ham, a, grid);
    default: return HPHI_E_INVAL;
    }
}

// bond sharing form: 1 = 8 targets per batch, 2 thread blocks per SM;
// 2 = 4 targets, 3 blocks; 3 = 4 targets, 4 blocks; 4 = 4 targets, 5 blocks;
// 5 = 2 targets, 6 blocks
template <typename T, int CPL, int G>
int go_coop(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int form, int red_mode, int *grid) {
    if (form == 2) return go_c_red<T, CPL, G, 4, 3>(ctx, ham, a, red_mode, grid);
    if (form == 3) return go_c_red<T, CPL, G, 4, 4>(ctx, ham, a, red_mode, grid);
    if (form == 4) return go_c_red<T, CPL, G, 4, 5>(ctx, ham, a, red_mode, grid);
    if (form == 5) return go_c_red<T, CPL, G, 2, 6>(ctx, ham, a, red_mode, grid);
    return go_c_red<T, CPL, G, 8, 2>(ctx, ham, a, red_mode, grid);
}

template <typename T, int CPL, int G, int RED>
int go(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int *grid_out) {
    const size_t dyn = RED ? 3 * (kThreads / 32) * G * CPL * sizeof(double) : 0;
    const int occ = dyn_occupancy(ctx, (const void *)k_hvo<T, CPL, G, RED>, kThreads, dyn);
    const int split = a.P.split;
    int64_t g = (int64_t)(occ > 0 ? occ : 1) * ctx->sm_count / split;
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    g *= split;
    *grid_out = (int)g;
    const int slot = prof_begin(ctx, PROF_HV);
    k_hvo<T, CPL, G, RED><<<(int)g, kThreads, dyn, ctx->stream>>>(a);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

template <typename T, int CPL, int G>
int go_red(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid) {
    switch (red_mode) {
    case 0: return go<T, CPL, G, 0>(ctx, ham, a, grid);
    case 1: return go<T, CPL, G, 1>(ctx, ham, a, grid);
    case 2: return go<T, CPL, G, 2>(ctx, ham, a, grid);
    case 3: return go<T, CPL, G, 3>(ctx, ham, a, grid);
    default: return HPHI_E_INVAL;
    }
}

}  // namespace

template <typename T>
int launch_fly(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int G, int cpl, int red_mode, int *grid) {
    if (G == 1 && cpl == 1) return go_red<T, 1, 1>(ctx, ham, a, red_mode, grid);
    if (G == 1 && cpl == 2) return go_red<T, 2, 1>(ctx, ham, a, red_mode, grid);
    // 32-column rows: cooperative target generation unless the per-lane variant was asked for
    // measured: shared bond work with registers for 4 blocks per SM pays for FP32
    // rows (-36 % on the N=26 block); the per-lane form is faster for FP64
    const int coop = ham->tune_coop < 0 ? (std::is_same<T, float>::value ? 3 : 0) : ham->tune_coop;
    if constexpr (std::is_same<T, float>::value) {
        if (G == 8 && cpl == 4) return coop ? go_coop<T, 4, 8>(ctx, ham, a, coop, red_mode, grid)
                                            : go_red<T, 4, 8>(ctx, ham, a, red_mode, grid);
    } else {
        if (G == 16 && cpl == 2) return coop ? go_coop<T, 2, 16>(ctx, ham, a, coop, red_mode, grid)
                                             : go_red<T, 2, 16>(ctx, ham, a, red_mode, grid);
    }
    return HPHI_E_INVAL;
}

template int launch_fly<float>(hphi_ctx *, const hphi_ham *, const HvArgs<float> &, int, int, int, int *);
template int launch_fly<double>(hphi_ctx *, const hphi_ham *, const HvArgs<double> &, int, int, int, int *);

}  // namespace hphi
