// Pieces shared by the generic and the lean H*x kernels.
#pragma once

#include <math.h>

#include "rowvisit.cuh"

namespace hphi {

struct FF {  // float-float accumulator (Knuth TwoSum + exact FMA product)
    float hi, lo;
};
static __device__ __forceinline__ void ff_add_prod(FF &s, float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float t = s.hi + p;
    float bp = t - s.hi;
    float e = (s.hi - (t - bp)) + (p - bp);
    s.hi = t;
    s.lo += e + pe;
}

template <typename T>
struct RedAcc;
template <>
struct RedAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct RedAcc<float> {
    FF s{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) { ff_add_prod(s, a, b); }
    __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};

// L2 cache policies and hinted loads / stores of the staged kernels: the
// vector x is kept (evict_last), streamed rows are evicted first.  Gathers of
// x allocate in L1 (L1::no_allocate measured 3 % slower on the 4x8 Lanczos
// H*x: neighbouring rows share lines).
__device__ __forceinline__ uint64_t spol(int hints, int kind) {
    uint64_t p;
    if (!hints) asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    else if (kind) asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

template <typename T>
__device__ __forceinline__ T gload(const T *p, uint64_t pol) {
    T v;
    if constexpr (std::is_same<T, float>::value)
        asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    else
        asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

template <typename T>
__device__ __forceinline__ T cload(const T *p, uint64_t pol) {  // coherent (v may alias y)
    T v;
    if constexpr (std::is_same<T, float>::value)
        asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol) : "memory");
    else
        asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}

template <typename T>
__device__ __forceinline__ void cstore(T *p, uint64_t pol, T v) {
    if constexpr (std::is_same<T, float>::value)
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
    else
        asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

#ifndef HPHI_SRC_TAG
#define HPHI_SRC_TAG "untagged"
#endif

template <typename T>
inline const char *tname() { return std::is_same<T, float>::value ? "f32" : "f64"; }

template <typename T>
struct HvArgs {
    HvTables P;
    const T *x;
    int64_t ldx;
    T *y;
    int64_t ldy;
    const T *v;
    int64_t ldv;
    int ncol;  // columns of this launch (<= 32)
    double beta;
    double alpha[32];
    double gamma[32];
    const double *alpha_dev;  // override alpha[] when non-null
    const double *gamma_dev;
    int red[3];
    double *partials;  // [grid][3][ncol]
    int swap;          // out[c] takes (H x)[c ^ 1]: multiplication by -i / +i of complex columns
    const T *tin;      // bond-major kernel: the high-high terms of every row, computed by a
                       // separate pass (the kernel then skips its high-high phase); else null
};

inline HvTables make_tables(const hphi_ham *ham, int real_dtype) {
    const hphi_basis *b = ham->basis;
    HvTables P{};
    P.desc = ham->desc;
    P.model = ham->model;
    P.nlo = ham->nlo;
    P.ngroups = ham->host.ngroups;
    P.n = ham->host.n;
    P.nh = ham->nh;
    P.L = ham->L;
    P.ddn = ham->host.ddn;
    P.jb = b->sp[0].jb;
    P.loff = b->sp[0].loff;
    P.lstate = b->sp[0].lstate;
    P.states_up = b->sp[0].states;
    P.states_dn = b->sp[1].states;
    P.dlow = real_dtype == HPHI_F64 ? (const void *)ham->dlow_d : (const void *)ham->dlow_f;
    P.ll_cnt = ham->ll_cnt;
    P.ll_tgt = ham->ll_tgt;
    P.ll_cf = ham->ll_cf;
    P.flipq = ham->flipq;
    P.up_cnt = ham->up_cnt;
    P.up_tgt = ham->up_tgt;
    P.up_cf = ham->up_cf;
    P.aup = ham->aup;
    P.ll_pk = ham->ll_pk;
    P.use_perm = 0;
    P.outer_mask = 0;
    for (int k = 0; k < 32; k++) P.hperm[k] = (uint8_t)k;
    P.split = 1;
    P.hints = ham->tune_hints;
    P.ja16 = ham->ja16;
    P.ph_ent = ham->ph_ent;
    P.ph_off = ham->ph_off;
    P.ph_mx0 = ham->ph_mx0;
    P.ph_nlb = ham->nlb;
    return P;
}

// Traversal order of the row blocks for a launch whose rows occupy
// bytes_per_row in L2.  The high-half bits of h are split into "inner" bits,
// varied first, so that the blocks of one subcube (about half of L2) stay
// resident while they are processed, and "outer" bits.  Every off-diagonal
// bond that touches an outer bit sends its target to another subcube, so the
// outer set is grown greedily by the bit that adds the fewest such bonds (its
// bonds minus those to bits already outer); outer bits with the most bonds
// come first in the counter, so that their flips reach the subcube processed
// just before or after.  Hubbard keeps natural order.
inline void set_traversal(hphi_ctx *ctx, const hphi_ham *ham, HvTables &P, double bytes_per_row) {
    P.use_perm = 0;
    P.outer_mask = 0;
    if (ham->model == HPHI_HUBBARD) return;
    const int nb = ham->host.nhi;
    if (nb <= 0 || nb > 32) return;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess || l2 <= 0) {
        cudaGetLastError();
        return;
    }
    const double block_bytes = (double)ham->D / (double)ham->nh * bytes_per_row;
    int d = (int)floor(log2(0.5 * (double)l2 / (block_bytes > 1.0 ? block_bytes : 1.0)));
    if (ham->tune_inner >= 0) d = ham->tune_inner;
    if (d < 0) d = 0;
    if (d >= nb) return;
    uint32_t adj[32] = {0};
    int deg[32] = {0};
    for (int k = 0; k < ham->host.n_hh; k++) {
        if (ham->host.hh[k].cxy == 0.0) continue;
        adj[ham->host.hh[k].i] |= 1u << ham->host.hh[k].j;
        adj[ham->host.hh[k].j] |= 1u << ham->host.hh[k].i;
        deg[ham->host.hh[k].i]++;
        deg[ham->host.hh[k].j]++;
    }
    for (int k = 0; k < ham->host.n_lh; k++)
        if (ham->host.lh[k].cxy != 0.0) deg[ham->host.lh[k].a]++;
    const int need = nb - d;
    uint32_t outer = 0;
    for (int t = 0; t < need; t++) {
        int best = -1, bc = 1 << 30;
        for (int b = nb - 1; b >= 0; b--) {
            if ((outer >> b) & 1) continue;
            const int c = deg[b] - __builtin_popcount(adj[b] & outer);
            if (c < bc) {
                bc = c;
                best = b;
            }
        }
        outer |= 1u << best;
    }
    int k = 0;
    for (int b = 0; b < nb; b++)
        if (!((outer >> b) & 1)) P.hperm[k++] = (uint8_t)b;
    // outer bits with the most bonds lowest in the counter: those flips go to the
    // subcube processed just before or after
    int maxd = 0;
    for (int b = 0; b < nb; b++) maxd = deg[b] > maxd ? deg[b] : maxd;
    for (int c = maxd; c >= 0; c--)
        for (int b = 0; b < nb; b++)
            if (((outer >> b) & 1) && deg[b] == c) P.hperm[k++] = (uint8_t)b;
    P.use_perm = 1;
    P.outer_mask = outer;
}


// Launchers of the lean kernel (hv_lean.cu).  Returns HPHI_E_INVAL when no
// lean variant covers the request (the caller then uses the generic kernel).
template <typename T>
int launch_lean(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int cpl, int ldc, int red_mode, int *grid);
// On-the-fly-rank kernel (hv_fly.cu), spin models: G lanes per row, CPL columns per lane.
template <typename T>
int launch_fly(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int G, int cpl, int red_mode, int *grid);
// staged kernel (hv_staged.cu): spin sector, one column, N_lo <= 16
template <typename T>
int launch_staged(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid);
template <typename T>
int launch_phased(hphi_ctx *ctx, const hphi_ham *ham, const HvArgs<T> &a, int red_mode, int *grid);
uint32_t staged_block_len(const hphi_ham *ham);
// tiled two-pass block kernel (hv_tile.cu): full space, 32 columns (FP32 or FP64)
template <typename T>
int launch_tile(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, int red_mode, int *grid);
// high-high pass plus the bond-major kernel (hv_seg.cu): spin sector, one column
template <typename T>
int launch_seg(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, int red_mode, int *grid);

}  // namespace hphi
