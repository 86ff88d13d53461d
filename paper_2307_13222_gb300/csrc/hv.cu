// The matrix-free H*x kernel (the product under every iterative method of
// the paper: Sec. 1, Sec. 3.4, Sec. 3.5.1).
//
//   y = alpha_c * (H x) + beta * y + gamma_c * v        (per real column c)
//
// optionally with per-column reductions of <x,Hx>, |Hx|^2, |x|^2, <x,y>, |y|^2
// written as per-block partials (summed later in fixed order, so results are
// bitwise reproducible).  Pull form: every output row is produced by one group
// of G lanes (lanes split the columns), so there are no atomics and x is only
// gathered.  Thread blocks walk the row blocks h in a fixed interleaved order.
#include <type_traits>

#include "rowvisit.cuh"

namespace hphi {

namespace {

struct FF {  // float-float accumulator (Knuth TwoSum + exact FMA product)
    float hi, lo;
};
__device__ __forceinline__ void ff_add_prod(FF &s, float a, float b) {
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

template <typename T, int CPL>
__device__ __forceinline__ void load_cols(const T *p, T (&v)[CPL]) {
    if constexpr (CPL == 1) {
        v[0] = __ldg(p);
    } else if constexpr (std::is_same<T, float>::value && CPL == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    } else if constexpr (std::is_same<T, float>::value && CPL == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < CPL; k += 2) {
            double2 t = __ldg(reinterpret_cast<const double2 *>(p + k));
            v[k] = t.x;
            v[k + 1] = t.y;
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void load_cols_rw(const T *p, T (&v)[CPL]) {  // may alias the output
    if constexpr (CPL == 1) {
        v[0] = *p;
    } else if constexpr (std::is_same<T, float>::value && CPL == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else if constexpr (std::is_same<T, float>::value && CPL == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < CPL; k += 2) {
            double2 t = *reinterpret_cast<const double2 *>(p + k);
            v[k] = t.x;
            v[k + 1] = t.y;
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void store_cols(T *p, const T (&v)[CPL]) {
    if constexpr (CPL == 1) {
        *p = v[0];
    } else if constexpr (std::is_same<T, float>::value && CPL == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else if constexpr (std::is_same<T, float>::value && CPL == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < CPL; k += 2) *reinterpret_cast<double2 *>(p + k) = make_double2(v[k], v[k + 1]);
    }
}

template <typename T, int CPL>
struct HvSink {
    const T *__restrict__ x;
    int64_t ldx;
    int col0;
    bool act;
    int64_t row;
    T acc[CPL];
    T xo[CPL];
    __device__ __forceinline__ void diag(int64_t r, T d) {
        row = r;
        if (act) {
            load_cols<T, CPL>(x + r * ldx + col0, xo);
#pragma unroll
            for (int k = 0; k < CPL; k++) acc[k] = d * xo[k];
        }
    }
    // all gathers of the chunk are issued before the first use
    __device__ __forceinline__ void add8(const int64_t (&t)[kChunk], const T (&c)[kChunk]) {
        if (!act) return;
        T xv[kChunk][CPL];
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            if (t[u] >= 0) {
                load_cols<T, CPL>(x + t[u] * ldx + col0, xv[u]);
            } else {
#pragma unroll
                for (int k = 0; k < CPL; k++) xv[u][k] = (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < kChunk; u++)
#pragma unroll
            for (int k = 0; k < CPL; k++) acc[k] = fma(c[u], xv[u][k], acc[k]);
    }
};

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
};

template <typename T, int G, int CPL>
__global__ void __launch_bounds__(kThreads) k_hv(const HvArgs<T> a) {
    extern __shared__ double red_sm[];  // [nwarps][3][G*CPL]
    __shared__ HBlock<T> hb;
    __shared__ T coef_sm[kMaxCoef];
    const HamDesc &D = *a.P.desc;
    for (int i = threadIdx.x; i < D.n_ncoef; i += blockDim.x) coef_sm[i] = (T)D.coef[i];

    const int gl = threadIdx.x % G, grp = threadIdx.x / G, ngrp = kThreads / G;
    const int col0 = gl * CPL;
    const bool act = col0 < a.ncol;
    T al[CPL], ga[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k++) {
        int c = col0 + k < a.ncol ? col0 + k : 0;
        al[k] = (T)(a.alpha_dev ? a.alpha_dev[c] : a.alpha[c]);
        ga[k] = (T)(a.gamma_dev ? a.gamma_dev[c] : a.gamma[c]);
    }
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0;
    const bool use_v = a.v != nullptr;
    const bool any_red = a.red[0] | a.red[1] | a.red[2];
    RedAcc<T> racc[3][CPL];

    for (int64_t h = blockIdx.x; h < a.P.nh; h += gridDim.x) {
        __syncthreads();  // the previous block's rows are done with hb
        setup_block<T>(a.P, h, hb);
        if (!hb.valid) continue;
        const uint32_t len = hb.len;
        for (uint32_t q = grp; q < len; q += ngrp) {
            HvSink<T, CPL> s;
            s.x = a.x;
            s.ldx = a.ldx;
            s.col0 = col0;
            s.act = act;
            visit_row<T>(a.P, hb, coef_sm, q, s);
            if (!act) continue;
            const int64_t row = s.row;
            T out[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) out[k] = al[k] * s.acc[k];
            if (use_beta) {
                T yo[CPL];
                load_cols_rw<T, CPL>(a.y + row * a.ldy + col0, yo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(be, yo[k], out[k]);
            }
            if (use_v) {
                T vo[CPL];
                load_cols_rw<T, CPL>(a.v + row * a.ldv + col0, vo);
#pragma unroll
                for (int k = 0; k < CPL; k++) out[k] = fma(ga[k], vo[k], out[k]);
            }
            store_cols<T, CPL>(a.y + row * a.ldy + col0, out);
            if (any_red) {
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    const int code = a.red[r];
                    if (code == R_NONE) continue;
#pragma unroll
                    for (int k = 0; k < CPL; k++) {
                        T u, w;
                        if (code == R_XHX) { u = s.xo[k]; w = s.acc[k]; }
                        else if (code == R_HXHX) { u = s.acc[k]; w = s.acc[k]; }
                        else if (code == R_XX) { u = s.xo[k]; w = s.xo[k]; }
                        else if (code == R_XO) { u = s.xo[k]; w = out[k]; }
                        else { u = out[k]; w = out[k]; }
                        racc[r][k].add(u, w);
                    }
                }
            }
        }
    }
    if (!any_red) return;
    // fixed-shape block reduction: lanes with the same column inside a warp,
    // then warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = kThreads / 32;
    constexpr int W = G * CPL;
#pragma unroll
    for (int r = 0; r < 3; r++) {
#pragma unroll
        for (int k = 0; k < CPL; k++) {
            double val = racc[r][k].value();
#pragma unroll
            for (int off = 16; off >= G; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
            if (lane < G) red_sm[(warp * 3 + r) * W + col0 + k] = val;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * W; t += blockDim.x) {
        int r = t / W, c = t % W;
        if (c >= a.ncol) continue;
        double s = 0.0;
        for (int w = 0; w < nwarp; w++) s += red_sm[(w * 3 + r) * W + c];
        a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol + c] = s;
    }
}

HvTables make_tables(const hphi_ham *ham, int real_dtype) {
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
    return P;
}

template <typename T, int G, int CPL>
int grid_for(hphi_ctx *ctx, int64_t nh, bool red) {
    static int occ[64] = {0};
    int dev = ctx->device;
    if (occ[dev] == 0) {
        int n = 0;
        size_t dyn = 3 * (kThreads / 32) * G * CPL * sizeof(double);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hv<T, G, CPL>, kThreads, dyn);
        occ[dev] = n > 0 ? n : 1;
    }
    int64_t g = (int64_t)occ[dev] * ctx->sm_count;
    if (g > nh) g = nh;
    if (g < 1) g = 1;
    (void)red;
    return (int)g;
}

template <typename T, int G, int CPL>
int launch_one(hphi_ctx *ctx, const HvArgs<T> &a, int64_t nh, int grid) {
    bool red = a.red[0] | a.red[1] | a.red[2];
    size_t dyn = red ? 3 * (kThreads / 32) * G * CPL * sizeof(double) : 0;
    int slot = prof_begin(ctx, PROF_HV);
    k_hv<T, G, CPL><<<grid, kThreads, dyn, ctx->stream>>>(a);
    prof_end(ctx, slot);
    (void)nh;
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

template <typename T>
int dispatch(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, bool pair_ok, bool quad_ok, int *grid_out) {
    bool red = a.red[0] | a.red[1] | a.red[2];
    int n = a.ncol;
    int grid;
#define HPHI_GO(G, CPL)                                      \
    do {                                                    \
        grid = grid_for<T, G, CPL>(ctx, ham->nh, red);      \
        *grid_out = grid;                                   \
        return launch_one<T, G, CPL>(ctx, a, ham->nh, grid); \
    } while (0)
    if (n == 1) HPHI_GO(1, 1);
    if (n == 2 && pair_ok) HPHI_GO(1, 2);
    if (n == 32 && quad_ok) {
        if (std::is_same<T, float>::value) HPHI_GO(8, 4);   // 4 rows per warp, 16-byte loads
        HPHI_GO(16, 2);                                     // 2 rows per warp, 16-byte loads
    }
    if (n <= 2) HPHI_GO(2, 1);
    if (n <= 4) HPHI_GO(4, 1);
    if (n <= 8) HPHI_GO(8, 1);
    if (n <= 16) HPHI_GO(16, 1);
    HPHI_GO(32, 1);
#undef HPHI_GO
}

template <typename T>
int launch_typed(hphi_ctx *ctx, const hphi_ham *ham, HvLaunch &L) {
    int c0 = 0;
    int64_t part_off = 0;
    L.nslice = 0;
    while (c0 < L.ncol) {
        int nc = L.ncol - c0 < 32 ? L.ncol - c0 : 32;
        HvArgs<T> a;
        a.P = make_tables(ham, L.dtype_real);
        a.x = (const T *)L.x + c0;
        a.ldx = L.ldx;
        a.y = (T *)L.y + c0;
        a.ldy = L.ldy;
        a.v = L.v ? (const T *)L.v + c0 : nullptr;
        a.ldv = L.ldv;
        a.ncol = nc;
        a.beta = L.beta;
        for (int c = 0; c < 32; c++) {
            a.alpha[c] = c < nc ? (L.alpha_h ? L.alpha_h[c0 + c] : L.alpha_s) : 0.0;
            a.gamma[c] = c < nc ? (L.gamma_h ? L.gamma_h[c0 + c] : L.gamma_s) : 0.0;
        }
        a.alpha_dev = L.coef_dev ? L.coef_dev + c0 : nullptr;
        a.gamma_dev = L.coef_dev ? L.coef_dev + L.ncol + c0 : nullptr;
        for (int r = 0; r < 3; r++) a.red[r] = L.red[r];
        a.partials = L.partials ? L.partials + part_off : nullptr;
        bool pair_ok = nc == 2 && (L.ldx % 2 == 0) && (L.ldy % 2 == 0) && (!L.v || L.ldv % 2 == 0) &&
                       ((uintptr_t)a.x % (2 * sizeof(T)) == 0) && ((uintptr_t)a.y % (2 * sizeof(T)) == 0) &&
                       (!a.v || (uintptr_t)a.v % (2 * sizeof(T)) == 0);
        // 32 columns with 16-byte aligned rows: several rows per warp, vector loads
        const size_t vb = 16;
        bool quad_ok = nc == 32 && ((L.ldx * sizeof(T)) % vb == 0) && ((L.ldy * sizeof(T)) % vb == 0) &&
                       (!L.v || (L.ldv * sizeof(T)) % vb == 0) && ((uintptr_t)a.x % vb == 0) &&
                       ((uintptr_t)a.y % vb == 0) && (!a.v || (uintptr_t)a.v % vb == 0);
        int grid = 0;
        int st = dispatch<T>(ctx, ham, a, pair_ok, quad_ok, &grid);
        if (st) return st;
        L.sgrid[L.nslice++] = grid;
        part_off += (int64_t)grid * 3 * nc;
        c0 += nc;
    }
    return HPHI_OK;
}

// out[r * ncol_total + c0 + c] = sum over blocks b (in order) of part[b][r][c]
__global__ void k_reduce_slice(const double *part, int grid, int nc, int c0, int ncol_total, double *out) {
    int t = threadIdx.x;
    if (t >= 3 * nc) return;
    int r = t / nc, c = t % nc;
    double s = 0.0;
    for (int b = 0; b < grid; b++) s += part[((int64_t)b * 3 + r) * nc + c];
    out[r * ncol_total + c0 + c] = s;
}

}  // namespace

size_t hv_partials_size(hphi_ctx *ctx, const hphi_ham *ham, int ncol) {
    // at most 2048 / kThreads resident blocks per SM, so no launch is larger
    int64_t g = (int64_t)ctx->sm_count * (2048 / kThreads);
    if (g > ham->nh) g = ham->nh;
    if (g < 1) g = 1;
    return (size_t)g * 3 * (size_t)ncol;
}

int reduce_hv(hphi_ctx *ctx, const HvLaunch &L, double *out_dev) {
    int64_t off = 0;
    int c0 = 0;
    for (int s = 0; s < L.nslice; s++) {
        int nc = L.ncol - c0 < 32 ? L.ncol - c0 : 32;
        k_reduce_slice<<<1, 96, 0, ctx->stream>>>(L.partials + off, L.sgrid[s], nc, c0, L.ncol, out_dev);
        HPHI_CUDA(ctx, cudaGetLastError());
        off += (int64_t)L.sgrid[s] * 3 * nc;
        c0 += nc;
    }
    return HPHI_OK;
}

int launch_hv(hphi_ctx *ctx, const hphi_ham *ham, HvLaunch &L) {
    if (L.dtype_real == HPHI_F64) return launch_typed<double>(ctx, ham, L);
    return launch_typed<float>(ctx, ham, L);
}

}  // namespace hphi
