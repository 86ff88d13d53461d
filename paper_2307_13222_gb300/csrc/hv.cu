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

#include "hvcommon.cuh"

namespace hphi {

namespace {

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
            // pair swap: the partner column is in this lane (CPL even) or in
            // lane gl ^ 1 of the same row group, which runs the same rows
            T hx[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) hx[k] = s.acc[k];
            if (a.swap) {
                if constexpr (CPL % 2 == 0) {
#pragma unroll
                    for (int k = 0; k < CPL; k++) hx[k] = s.acc[k ^ 1];
                } else if constexpr (G >= 2) {
                    const int lane = threadIdx.x & 31;
                    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane - gl);
                    hx[0] = __shfl_xor_sync(gmask, s.acc[0], 1);
                }
            }
            if (!act) continue;
            const int64_t row = s.row;
            T out[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) out[k] = al[k] * hx[k];
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

template <typename T, int G, int CPL>
int grid_for(hphi_ctx *ctx, int64_t nh, bool red) {
    const size_t dyn = 3 * (kThreads / 32) * G * CPL * sizeof(double);
    const int occ = dyn_occupancy(ctx, (const void *)k_hv<T, G, CPL>, kThreads, dyn);
    int64_t g = (int64_t)(occ > 0 ? occ : 1) * ctx->sm_count;
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
    if (L.swap && (L.ncol % 2 != 0)) return set_err(ctx, HPHI_E_INVAL, "pair swap needs an even column count");
    const bool same_ld = L.ldx == L.ldy && (!L.v || L.ldv == L.ldx);
    int red_mode = -1;
    if (!L.red[0] && !L.red[1] && !L.red[2]) red_mode = 0;
    else if (L.red[0] == R_XO && !L.red[1] && !L.red[2]) red_mode = 1;
    else if (L.red[0] == R_XHX && L.red[1] == R_HXHX && L.red[2] == R_XX) red_mode = 2;
    else if (L.red[0] == R_OO && !L.red[1] && !L.red[2]) red_mode = 3;
    constexpr int WIDE = std::is_same<T, float>::value ? 8 : 4;
    auto aligned = [](const void *p, size_t b) { return p == nullptr || (uintptr_t)p % b == 0; };
    int c0 = 0;
    int64_t part_off = 0;
    L.nslice = 0;
    while (c0 < L.ncol) {
        const int rem = L.ncol - c0;
        const T *xs = (const T *)L.x + c0;
        T *ys = (T *)L.y + c0;
        const T *vs = L.v ? (const T *)L.v + c0 : nullptr;
        // spin sector, one column: the staged kernels (variants 2 and 3), automatic there
        // (measured faster than the table-driven kernel on the 6x5 and 4x8 sectors)
        const bool one_col = same_ld && red_mode >= 0 && L.ldx == 1 && L.ncol == 1 && !L.swap &&
                             (double)ham->D < 4294967296.0;
        // the high-high pass plus the bond-major kernel (variant 4): spin sector, one column,
        // row offsets of 32 bits
        const bool seg = ham->tune_variant == 4 && ham->seg && ham->ph_ent && ham->host.n_ll <= 128 && one_col &&
                         (double)ham->D < 2147483648.0;
        const bool spin_staged = !seg &&
                                 (ham->tune_variant == 2 || ham->tune_variant == 3 || ham->tune_variant < 0) &&
                                 ham->model == HPHI_SPIN_HALF && ham->nlo <= 16 && ham->host.n_ll <= 128 && one_col;
        // Hubbard, one column: the bond-major kernel where its down-hop lists exist and the
        // D_dn-row block (x and accumulator) fits in shared memory next to the block set-up
        const bool hub_phased = (ham->tune_variant == 3 || ham->tune_variant < 0) && ham->model == HPHI_HUBBARD &&
                                ham->ph_ent && one_col &&
                                (double)ham->basis->sp[1].dim * 2.0 * sizeof(T) <= 200.0 * 1024.0;
        const bool staged = spin_staged || hub_phased || seg;
        // spin models: the on-the-fly-rank kernel for unit / pair / 32-wide rows
        int fG = 0, fcpl = 0;
        // variant -1 (automatic): on-the-fly ranks for 32-wide rows, lists for unit / pair rows
        const int variant = ham->tune_variant >= 0 ? ham->tune_variant : (L.ldx == 32 ? 1 : 0);
        const bool fly_ok = !staged && variant == 1 && ham->host.n_ll <= 128 &&
                            (ham->model == HPHI_SPIN_HALF_GC || (ham->model == HPHI_SPIN_HALF && ham->ja16));
        if (same_ld && red_mode >= 0 && fly_ok && (double)ham->D * (double)L.ldx < 4294967296.0) {
            if (L.ldx == 1) {
                fG = 1;
                fcpl = 1;
            } else if (L.ldx == 2 && rem >= 2 && aligned(xs, 2 * sizeof(T)) && aligned(ys, 2 * sizeof(T)) &&
                       aligned(vs, 2 * sizeof(T))) {
                fG = 1;
                fcpl = 2;
            } else if (L.ldx == 32 && c0 == 0 && L.ncol == 32 && aligned(xs, 16) && aligned(ys, 16) &&
                       aligned(vs, 16)) {
                fG = std::is_same<T, float>::value ? 8 : 16;
                fcpl = std::is_same<T, float>::value ? 4 : 2;
            }
        }
        // the lean kernel covers unit / pair / 32-wide rows; the rest goes generic
        int cpl = 0, ldc = -1;
        // the lean kernel addresses elements with 32-bit offsets
        const bool off32 = (double)ham->D * (double)L.ldx < 4294967296.0;
        // Hubbard: the generic kernel measured fastest; the lean one only on request
        const bool lean_ok = ham->model != HPHI_HUBBARD || ham->tune_variant == 0;
        if (same_ld && red_mode >= 0 && off32 && lean_ok && !fG && !staged) {
            const size_t vb = WIDE * sizeof(T) >= 16 ? 16 : WIDE * sizeof(T);
            if (L.ldx == 1) {
                cpl = 1;
                ldc = 1;
            } else if (L.ldx == 2 && rem >= 2 && aligned(xs, 2 * sizeof(T)) && aligned(ys, 2 * sizeof(T)) &&
                       aligned(vs, 2 * sizeof(T))) {
                cpl = 2;
                ldc = 2;
            } else if (L.ldx == 32 && rem >= WIDE && aligned(xs, vb) && aligned(ys, vb) && aligned(vs, vb)) {
                cpl = WIDE;
                ldc = 32;
            }
        }
        const int nc = staged ? 1 : (fG ? fG * fcpl : (cpl ? cpl : (rem < 32 ? rem : 32)));
        HvArgs<T> a;
        a.P = make_tables(ham, L.dtype_real);
        a.x = xs;
        a.ldx = L.ldx;
        a.y = ys;
        a.ldy = L.ldy;
        a.v = vs;
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
        a.swap = L.swap;
        a.tin = nullptr;
        if (L.swap && ((nc % 2) != 0 || (c0 % 2) != 0 || (fG == 1 && fcpl == 1) || (cpl == 1)))
            return set_err(ctx, HPHI_E_INVAL, "pair swap: column slice [%d, %d) splits a pair", c0, c0 + nc);
        int grid = 0, st;
        // the tiled two-pass block kernel (variant 5, automatic there): full space, 32
        // columns, 16-byte accesses (measured on the N=26 cTPQ block: 1.3x faster than the
        // single-pass kernels in FP32, 1.1x in FP64)
        bool tiled = false;
        {
            constexpr int prec = std::is_same<T, float>::value ? 0 : 1;
            if ((ham->tune_variant == 5 || ham->tune_variant < 0) && ham->model == HPHI_SPIN_HALF_GC && c0 == 0 &&
                L.ncol == 32 &&
                L.ldx == 32 && L.ldy == 32 && (!L.v || L.ldv == 32) && red_mode >= 0 && aligned(xs, 16) &&
                aligned(ys, 16) && aligned(vs, 16)) {
                if ((st = build_tile_tables(ctx, const_cast<hphi_ham *>(ham), prec))) return st;
                tiled = ham->tile[prec] != nullptr;
            }
        }
        if (tiled) {
            a.ncol = 32;
            for (int c = 0; c < 32; c++) {
                a.alpha[c] = L.alpha_h ? L.alpha_h[c] : L.alpha_s;
                a.gamma[c] = L.gamma_h ? L.gamma_h[c] : L.gamma_s;
            }
            st = launch_tile<T>(ctx, ham, a, red_mode, &grid);
            if (st) return st;
            L.sgrid[L.nslice] = grid;
            L.sc0[L.nslice] = 0;
            L.snc[L.nslice] = 32;
            L.nslice++;
            c0 = 32;
            continue;
        }
        if (staged) {
            set_traversal(ctx, ham, a.P, (double)sizeof(T));
            a.P.split = 1;
            // automatic: the bond-major kernel where its lists exist (measured 14-42 % faster than
            // the staged kernel on the 6x5 and 4x8 sectors, FP32 and FP64)
            const bool phased = hub_phased || ham->tune_variant == 3 ||
                                (ham->tune_variant < 0 && ham->ph_ent && ham->host.n_ll <= 128);
            st = seg ? launch_seg<T>(ctx, ham, a, red_mode, &grid)
                     : phased ? launch_phased<T>(ctx, ham, a, red_mode, &grid)
                              : launch_staged<T>(ctx, ham, a, red_mode, &grid);
        } else if (fG) {
            set_traversal(ctx, ham, a.P, (double)nc * sizeof(T) < 4.0 ? 4.0 : (double)nc * sizeof(T));
            a.P.split = ham->tune_split;
            st = launch_fly<T>(ctx, ham, a, fG, fcpl, red_mode, &grid);
            snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_hvo/k_hvc<%s,G%d,CPL%d,RED%d,coop%d>@" HPHI_SRC_TAG, tname<T>(),
                     fG, fcpl, red_mode, ham->tune_coop);
        } else if (cpl) {
            set_traversal(ctx, ham, a.P, (double)cpl * sizeof(T) < 4.0 ? 4.0 : (double)cpl * sizeof(T));
            a.P.split = ham->tune_split;
            st = launch_lean<T>(ctx, ham, a, cpl, ldc, red_mode, &grid);
            snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_hvl<%s,CPL%d,LDC%d,RED%d>@" HPHI_SRC_TAG, tname<T>(), cpl, ldc,
                     red_mode);
        } else {
            bool pair_ok = nc == 2 && (L.ldx % 2 == 0) && (L.ldy % 2 == 0) && (!L.v || L.ldv % 2 == 0) &&
                           aligned(xs, 2 * sizeof(T)) && aligned(ys, 2 * sizeof(T)) && aligned(vs, 2 * sizeof(T));
            const size_t vb = 16;
            bool quad_ok = nc == 32 && ((L.ldx * sizeof(T)) % vb == 0) && ((L.ldy * sizeof(T)) % vb == 0) &&
                           (!L.v || (L.ldv * sizeof(T)) % vb == 0) && aligned(xs, vb) && aligned(ys, vb) &&
                           aligned(vs, vb);
            st = dispatch<T>(ctx, ham, a, pair_ok, quad_ok, &grid);
            snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_hv<%s,NC%d>@" HPHI_SRC_TAG, tname<T>(), nc);
        }
        if (st) return st;
        L.sgrid[L.nslice] = grid;
        L.sc0[L.nslice] = c0;
        L.snc[L.nslice] = nc;
        L.nslice++;
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
    for (int s = 0; s < L.nslice; s++) {
        k_reduce_slice<<<1, 96, 0, ctx->stream>>>(L.partials + off, L.sgrid[s], L.snc[s], L.sc0[s], L.ncol, out_dev);
        HPHI_CUDA(ctx, cudaGetLastError());
        off += (int64_t)L.sgrid[s] * 3 * L.snc[s];
    }
    return HPHI_OK;
}

int launch_hv(hphi_ctx *ctx, const hphi_ham *ham, HvLaunch &L) {
    if (L.dtype_real == HPHI_F64) return launch_typed<double>(ctx, ham, L);
    return launch_typed<float>(ctx, ham, L);
}

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_ham_set_tuning(hphi_ham *ham, int knob, int value) {
    if (!ham) return HPHI_E_INVAL;
    switch (knob) {
    case HPHI_TUNE_INNER_BITS:
        if (value < -1 || value > 32) return HPHI_E_INVAL;
        ham->tune_inner = value;
        return HPHI_OK;
    case HPHI_TUNE_SPLIT:
        if (value < 1 || value > 8) return HPHI_E_INVAL;
        ham->tune_split = value;
        return HPHI_OK;
    case HPHI_TUNE_L2_HINTS:
        if (value != 0 && value != 1) return HPHI_E_INVAL;
        ham->tune_hints = value;
        return HPHI_OK;
    case HPHI_TUNE_VARIANT:
        if (value < -1 || value > 5) return HPHI_E_INVAL;
        ham->tune_variant = value;
        return HPHI_OK;
    case HPHI_TUNE_COOP:
        if (value < -1 || value > 5) return HPHI_E_INVAL;
        ham->tune_coop = value;
        return HPHI_OK;
    case HPHI_TUNE_STAGED_LISTS:
        if (value < -1 || value > 3) return HPHI_E_INVAL;
        ham->tune_staged_lists = value;
        return HPHI_OK;
    default:
        return HPHI_E_INVAL;
    }
}

extern "C" int hphi_ham_get_tuning(const hphi_ham *ham, int knob, int *value) {
    if (!ham || !value) return HPHI_E_INVAL;
    switch (knob) {
    case HPHI_TUNE_INNER_BITS: *value = ham->tune_inner; return HPHI_OK;
    case HPHI_TUNE_SPLIT: *value = ham->tune_split; return HPHI_OK;
    case HPHI_TUNE_L2_HINTS: *value = ham->tune_hints; return HPHI_OK;
    case HPHI_TUNE_VARIANT: *value = ham->tune_variant; return HPHI_OK;
    case HPHI_TUNE_COOP: *value = ham->tune_coop; return HPHI_OK;
    case HPHI_TUNE_STAGED_LISTS: *value = ham->tune_staged_lists; return HPHI_OK;
    default: return HPHI_E_INVAL;
    }
}
