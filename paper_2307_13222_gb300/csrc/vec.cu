// Vector kernels around H*x: dot / nrm2 / axpy / scal (the Krylov and TPQ
// bookkeeping of Sec. 1 and Sec. 3.5.1), start vectors, copies, and the
// fixed-order reduction of per-block partial sums.
//
// Layout: n rows of nr real values, row stride ld (elements).  A row is
// handled by TPR lanes (the smallest power of two >= nr, at most 32); lane t
// takes the real columns t, t + TPR, ...  Grids are fixed for a given (n, nr),
// so every reduction is summed in the same order on every call.
#include <math.h>

#include "hphi_internal.cuh"

namespace hphi {

namespace {

struct FFv {
    float hi, lo;
};

template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
    FFv s{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) {
        float p = a * b, pe = fmaf(a, b, -p);
        float t = s.hi + p, bp = t - s.hi;
        float e = (s.hi - (t - bp)) + (p - bp);
        s.hi = t;
        s.lo += e + pe;
    }
    __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};

constexpr int kVT = 256;  // threads per block of the vector kernels

inline int tpr_of(int nr) {
    int t = 1;
    while (t < nr && t < 32) t <<= 1;
    return t;
}

// S[c] = sum_r x[r][c] y[r][c];  X[c] = sum_r x[r][c] y[r][c^1]  (if cross).
// Lane `lane` of a row group owns columns lane + j*tpr, j < CPL; every
// thread runs the same number of row iterations; the block sum is taken in
// shared memory in a fixed order (group 0, 1, ...).
template <typename T, int CPL>
__global__ void __launch_bounds__(kVT) k_dot(int64_t n, int nr, int tpr, int cross, const T *__restrict__ x,
                                             int64_t ldx, const T *__restrict__ y, int64_t ldy, double *partials) {
    __shared__ double sm[2][kVT][CPL];
    const int lane = threadIdx.x % tpr, grp = threadIdx.x / tpr, ngrp = kVT / tpr;
    Acc<T> s[CPL], xs[CPL];
    for (int64_t r0 = blockIdx.x * (int64_t)ngrp; r0 < n; r0 += (int64_t)gridDim.x * ngrp) {
        const int64_t r = r0 + grp;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < CPL; j++) {
            const int c = lane + j * tpr;
            if (c < nr) {
                const T xv = x[r * ldx + c];
                s[j].add(xv, y[r * ldy + c]);
                if (cross) xs[j].add(xv, y[r * ldy + (c ^ 1)]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CPL; j++) {
        sm[0][threadIdx.x][j] = s[j].value();
        sm[1][threadIdx.x][j] = xs[j].value();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * nr; t += blockDim.x) {
        const int which = t / nr, c = t % nr, l = c % tpr, j = c / tpr;
        double acc = 0.0;
        for (int g = 0; g < ngrp; g++) acc += sm[which][g * tpr + l][j];
        partials[((int64_t)blockIdx.x * 2 + which) * nr + c] = acc;
    }
}

__global__ void k_reduce(const double *partials, int grid, int nval, double *out) {
    for (int v = threadIdx.x; v < nval; v += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < grid; b++) s += partials[(int64_t)b * nval + v];
        out[v] = s;
    }
}

// out[v] = sum_b partials[b][v], one warp per value: lane l sums b = l, l + 32,
// ... in order, then a fixed butterfly (deterministic).  For many values.
__global__ void k_reduce_wide(const double *partials, int grid, int nval, double *out) {
    const int v = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (v >= nval) return;
    double sum = 0.0;
    for (int b = lane; b < grid; b += 32) sum += partials[(int64_t)b * nval + v];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) out[v] = sum;
}

struct LCArgs {
    int64_t n;
    int nr, tpr, red;
    const void *x;
    int64_t ldx;
    const void *y;
    int64_t ldy;
    void *out;
    int64_t ldo;
    const double *coef_dev;  // device [3][nr] (a, b, g); overrides the arrays below
    double *partials;
    double a[256], b[256], g[256];
};

template <typename T, int CPL>
__global__ void __launch_bounds__(kVT) k_lincomb(const LCArgs A) {
    __shared__ double sm[kVT][CPL];
    __shared__ double cf[3][256];
    for (int t = threadIdx.x; t < A.nr; t += blockDim.x) {
        if (A.coef_dev) {
            cf[0][t] = A.coef_dev[t];
            cf[1][t] = A.coef_dev[A.nr + t];
            cf[2][t] = A.coef_dev[2 * A.nr + t];
        } else {
            cf[0][t] = A.a[t];
            cf[1][t] = A.b[t];
            cf[2][t] = A.g[t];
        }
    }
    __syncthreads();
    const T *x = (const T *)A.x;
    const T *y = (const T *)A.y;
    T *o = (T *)A.out;
    const int lane = threadIdx.x % A.tpr, grp = threadIdx.x / A.tpr, ngrp = kVT / A.tpr;
    Acc<T> s[CPL];
    // every thread runs the same number of iterations (uniform __syncwarp)
    for (int64_t r0 = blockIdx.x * (int64_t)ngrp; r0 < A.n; r0 += (int64_t)gridDim.x * ngrp) {
        const int64_t r = r0 + grp;
        const bool rv = r < A.n;
        T res[CPL];
#pragma unroll
        for (int j = 0; j < CPL; j++) {
            const int c = lane + j * A.tpr;
            if (rv && c < A.nr) {
                T v = (T)cf[0][c] * x[r * A.ldx + c];
                if (cf[1][c] != 0.0) v = fma((T)cf[1][c], x[r * A.ldx + (c ^ 1)], v);
                if (y && cf[2][c] != 0.0) v = fma((T)cf[2][c], y[r * A.ldy + c], v);
                res[j] = v;
            }
        }
        __syncwarp();  // all lanes have read x[c^1] before any writes (in-place complex scal)
#pragma unroll
        for (int j = 0; j < CPL; j++) {
            const int c = lane + j * A.tpr;
            if (rv && c < A.nr) {
                o[r * A.ldo + c] = res[j];
                if (A.red) s[j].add(res[j], res[j]);
            }
        }
        __syncwarp();
    }
    if (!A.red) return;
#pragma unroll
    for (int j = 0; j < CPL; j++) sm[threadIdx.x][j] = s[j].value();
    __syncthreads();
    for (int c = threadIdx.x; c < A.nr; c += blockDim.x) {
        const int l = c % A.tpr, j = c / A.tpr;
        double acc = 0.0;
        for (int g = 0; g < ngrp; g++) acc += sm[g * A.tpr + l][j];
        A.partials[(int64_t)blockIdx.x * A.nr + c] = acc;
    }
}

// Single contiguous column: out = a x + g y (+ sum out^2), 16-byte vector
// accesses, four in flight per thread.  Same arithmetic per element as
// k_lincomb (a x, then fma with g y); the pair term b does not exist for one
// column.  out may alias x or y (element-wise, read before written).
template <typename T>
__global__ void __launch_bounds__(kVT) k_lincomb1(int64_t n, const T *x, const T *y, T *o, const double *coef_dev,
                                                  double a0, double g0, int red, double *partials) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int V = 16 / sizeof(T), U = 4;
    const T a = (T)(coef_dev ? coef_dev[0] : a0);
    const T g = (T)(coef_dev ? coef_dev[2] : g0);
    const bool use_y = y != nullptr && g != (T)0;
    Acc<T> s;
    const int64_t nv = n / V, stride = (int64_t)gridDim.x * kVT;
    const VT *xv = (const VT *)x, *yv = (const VT *)y;
    VT *ov = (VT *)o;
    for (int64_t i0 = blockIdx.x * (int64_t)kVT + threadIdx.x; i0 < nv; i0 += stride * U) {
        VT xr[U], yr[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t i = i0 + u * stride;
            if (i < nv) {
                xr[u] = xv[i];
                if (use_y) yr[u] = yv[i];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t i = i0 + u * stride;
            if (i < nv) {
                T *xe = (T *)&xr[u], *ye = (T *)&yr[u];
                VT r;
                T *re = (T *)&r;
#pragma unroll
                for (int e = 0; e < V; e++) {
                    T v = a * xe[e];
                    if (use_y) v = fma(g, ye[e], v);
                    re[e] = v;
                    if (red) s.add(v, v);
                }
                ov[i] = r;
            }
        }
    }
    // tail (n not a multiple of the vector width)
    for (int64_t i = nv * V + blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += stride) {
        T v = a * x[i];
        if (use_y) v = fma(g, y[i], v);
        o[i] = v;
        if (red) s.add(v, v);
    }
    if (!red) return;
    __shared__ double sm[kVT];
    sm[threadIdx.x] = s.value();
    __syncthreads();
    for (int w = kVT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

// Contiguous rows of nr columns (ld = nr, nr dividing the vector stride): the
// data is one flat array and a thread's 16-byte vectors always hold the same
// columns, so the coefficients stay in registers and the column reductions in
// per-thread accumulators.  Per element the arithmetic of k_lincomb: a x_c,
// then fma with b x_{c^1} (the pair partner, inside the same vector), then
// fma with g y_c.  out may alias x or y.
template <typename T>
__global__ void __launch_bounds__(kVT) k_lincomb_rows(const LCArgs A) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int V = 16 / sizeof(T);
    __shared__ double sm[kVT][V];
    const int nr = A.nr;
    const int64_t tg = blockIdx.x * (int64_t)kVT + threadIdx.x, stride = (int64_t)gridDim.x * kVT;
    const int c0 = (int)((tg * V) % nr);
    T ca[V], cb[V], cg[V];
#pragma unroll
    for (int e = 0; e < V; e++) {
        const int c = c0 + e;
        ca[e] = (T)(A.coef_dev ? A.coef_dev[c] : A.a[c]);
        cb[e] = (T)(A.coef_dev ? A.coef_dev[nr + c] : A.b[c]);
        cg[e] = (T)(A.coef_dev ? A.coef_dev[2 * nr + c] : A.g[c]);
    }
    const VT *xv = (const VT *)A.x, *yv = (const VT *)A.y;
    VT *ov = (VT *)A.out;
    const int64_t nv = A.n * nr / V;
    Acc<T> s[V];
    for (int64_t i0 = tg; i0 < nv; i0 += stride * 2) {
        VT xr[2], yr[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int64_t i = i0 + u * stride;
            if (i < nv) {
                xr[u] = xv[i];
                if (yv) yr[u] = yv[i];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int64_t i = i0 + u * stride;
            if (i < nv) {
                const T *xe = (const T *)&xr[u], *ye = (const T *)&yr[u];
                VT r;
                T *re = (T *)&r;
#pragma unroll
                for (int e = 0; e < V; e++) {
                    T v = ca[e] * xe[e];
                    if (cb[e] != (T)0) v = fma(cb[e], xe[e ^ 1], v);
                    if (yv && cg[e] != (T)0) v = fma(cg[e], ye[e], v);
                    re[e] = v;
                    if (A.red) s[e].add(v, v);
                }
                ov[i] = r;
            }
        }
    }
    if (!A.red) return;
#pragma unroll
    for (int e = 0; e < V; e++) sm[threadIdx.x][e] = s[e].value();
    __syncthreads();
    for (int c = threadIdx.x; c < nr; c += kVT) {
        double acc = 0.0;
        for (int t = 0; t < kVT; t++) {
            const int ct = (int)(((blockIdx.x * (int64_t)kVT + t) * V) % nr);
            if (c >= ct && c < ct + V) acc += sm[t][c - ct];
        }
        A.partials[(int64_t)blockIdx.x * nr + c] = acc;
    }
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; r++) {
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

template <typename T>
__global__ void k_random(int64_t n, int nr, uint64_t seed, T *x, int64_t ldx) {
    const int64_t total = n * nr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)e, (uint32_t)((uint64_t)e >> 32), 0u, 0u};
        philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        uint64_t wa = ((uint64_t)c[1] << 32) | c[0], wb = ((uint64_t)c[3] << 32) | c[2];
        double ua = ((double)(wa >> 11) + 0.5) * 0x1.0p-53;
        double ub = ((double)(wb >> 11) + 0.5) * 0x1.0p-53;
        double z = sqrt(-2.0 * log(ua)) * cos(6.283185307179586 * ub);
        int64_t r = e / nr;
        int c0 = (int)(e - r * nr);
        x[r * ldx + c0] = (T)z;
    }
}

template <typename T>
__global__ void k_copy(int64_t n, int nr, const T *x, int64_t ldx, T *y, int64_t ldy) {
    const int64_t total = n * nr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / nr;
        int c = (int)(e - r * nr);
        y[r * ldy + c] = x[r * ldx + c];
    }
}

// FP64 data: c[j] partials = sum over this block's rows of V[j][r] * w[r], j in
// a chunk of 8 stored vectors (grid.y walks the chunks), one accumulator per
// thread and vector, so the FP64 pipe does one FMA per element.  V holds nv vectors of length n,
// vector j at V + j * n.  Fixed grid and order: deterministic.
template <typename T>
__global__ void __launch_bounds__(kVT) k_mdot(int64_t n, int nv, const T *__restrict__ V, const T *__restrict__ w,
                                              double *partials) {
    constexpr int J = 8;
    __shared__ double sm[kVT / 32][J];
    const int j0 = blockIdx.y * J;
    Acc<T> s[J];
    for (int64_t r = blockIdx.x * (int64_t)kVT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kVT) {
        const T wv = w[r];
#pragma unroll
        for (int j = 0; j < J; j++)
            if (j0 + j < nv) s[j].add(V[(int64_t)(j0 + j) * n + r], wv);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < J; j++) {
        double v = s[j].value();
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) sm[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < J && j0 + (int)threadIdx.x < nv) {
        double acc = 0.0;
        for (int w2 = 0; w2 < kVT / 32; w2++) acc += sm[w2][threadIdx.x];
        partials[(int64_t)blockIdx.x * nv + j0 + threadIdx.x] = acc;
    }
}

// Multi-vector kernels of the reorthogonalisation (V holds nv vectors of
// length n, vector j at V + j * n), tiled by rows: a thread
// holds kMR rows of a tile of kMT * kMR rows, so every pass reads each V_j and w
// once from memory.
constexpr int kMT = 256, kMR = 4;

// FP32 data: partials[block][j] = sum over the block's tiles of <V_j, w>.  Per
// tile, a lane forms its partial products for 32 vectors at a time (4 rows
// each); a transposing butterfly (31 shuffles) leaves in lane l the warp's sum
// for vector j0 + l, which lane l adds to the warp's FP64 slot.  The block then
// sums its warps in order (deterministic).
template <typename T>
__global__ void __launch_bounds__(kMT, 4) k_mdot_tiled(int64_t n, int nv, const T *__restrict__ V,
                                                    const T *__restrict__ w, double *partials) {
    extern __shared__ double acc_sm[];  // [kMT / 32][nv]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < (kMT / 32) * nv; j += kMT) acc_sm[j] = 0.0;
    __syncthreads();
    constexpr int64_t TILE = (int64_t)kMT * kMR;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * TILE + threadIdx.x;
        T wv[kMR];
#pragma unroll
        for (int i = 0; i < kMR; i++) wv[i] = r0 + i * kMT < n ? w[r0 + i * kMT] : (T)0;
        for (int j0 = 0; j0 < nv; j0 += 32) {
            T v[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
                v[j] = (T)0;
                if (j0 + j < nv) {
                    const T *vj = V + (int64_t)(j0 + j) * n;
#pragma unroll
                    for (int i = 0; i < kMR; i++)
                        if (r0 + i * kMT < n) v[j] = fma(vj[r0 + i * kMT], wv[i], v[j]);
                }
            }
            // transposing butterfly: after the step of width s, lane l keeps the
            // half of its values whose index offset matches bit s of l
#pragma unroll
            for (int s2 = 16; s2 >= 1; s2 >>= 1) {
                const bool upper = (lane & s2) != 0;
#pragma unroll
                for (int j = 0; j < s2; j++) {
                    const T send = upper ? v[j] : v[j + s2];
                    const T keep = upper ? v[j + s2] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s2);
                }
            }
            if (j0 + lane < nv) acc_sm[warp * nv + j0 + lane] += (double)v[0];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nv; j += kMT) {
        double sum = 0.0;
        for (int w2 = 0; w2 < kMT / 32; w2++) sum += acc_sm[w2 * nv + j];
        partials[(int64_t)blockIdx.x * nv + j] = sum;
    }
}

// w[r] -= sum_j c[j] V[j][r], the sum in T in order of j, kMR rows per thread
// so that 4 loads per vector are in flight.
template <typename T>
__global__ void __launch_bounds__(kMT) k_maxpy_tiled(int64_t n, int nv, const T *__restrict__ V,
                                                     const double *__restrict__ c, T *w) {
    extern __shared__ __align__(16) unsigned char cs_raw[];
    T *cs = (T *)cs_raw;  // [nv]
    for (int j = threadIdx.x; j < nv; j += kMT) cs[j] = (T)c[j];
    __syncthreads();
    constexpr int64_t TILE = (int64_t)kMT * kMR;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * TILE + threadIdx.x;
        T acc[kMR];
#pragma unroll
        for (int i = 0; i < kMR; i++) acc[i] = (T)0;
#pragma unroll 4
        for (int j = 0; j < nv; j++) {
            const T *vj = V + (int64_t)j * n;
            const T cj = cs[j];
#pragma unroll
            for (int i = 0; i < kMR; i++)
                if (r0 + i * kMT < n) acc[i] = fma(cj, vj[r0 + i * kMT], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < kMR; i++)
            if (r0 + i * kMT < n) w[r0 + i * kMT] -= acc[i];
    }
}

int vec_grid(hphi_ctx *ctx, int64_t n, int tpr) {
    int64_t rows_per_block = kVT / tpr;
    int64_t g = (n + rows_per_block - 1) / rows_per_block;
    int64_t cap = (int64_t)ctx->sm_count * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int reduce_partials(hphi_ctx *ctx, const double *partials, int grid, int nval, double *out_dev) {
    k_reduce<<<1, 256, 0, ctx->stream>>>(partials, grid, nval, out_dev);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int launch_dot(hphi_ctx *ctx, int real_dtype, int cplx, int64_t n, int nr, const void *x, int64_t ldx, const void *y,
               int64_t ldy, double *out_dev) {
    int tpr = tpr_of(nr);
    int grid = vec_grid(ctx, n, tpr);
    int st = ensure_partials(ctx, (size_t)grid * 2 * nr);
    if (st) return st;
    int slot = prof_begin(ctx, PROF_VEC);
    const int cpl = (nr + tpr - 1) / tpr;
#define HPHI_DOT(T, C)                                                                                         \
    k_dot<T, C><<<grid, kVT, 0, ctx->stream>>>(n, nr, tpr, cplx, (const T *)x, ldx, (const T *)y, ldy, \
                                               ctx->partials)
    if (real_dtype == HPHI_F64) {
        if (cpl <= 1) HPHI_DOT(double, 1);
        else if (cpl <= 2) HPHI_DOT(double, 2);
        else if (cpl <= 4) HPHI_DOT(double, 4);
        else HPHI_DOT(double, 8);
    } else {
        if (cpl <= 1) HPHI_DOT(float, 1);
        else if (cpl <= 2) HPHI_DOT(float, 2);
        else if (cpl <= 4) HPHI_DOT(float, 4);
        else HPHI_DOT(float, 8);
    }
#undef HPHI_DOT
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return reduce_partials(ctx, ctx->partials, grid, 2 * nr, out_dev);
}

int launch_lincomb(hphi_ctx *ctx, LinComb &L) {
    LCArgs A;
    A.n = L.n;
    A.nr = L.nr;
    A.tpr = tpr_of(L.nr);
    A.red = L.red_oo;
    A.x = L.x;
    A.ldx = L.ldx;
    A.y = L.y;
    A.ldy = L.ldy;
    A.out = L.out;
    A.ldo = L.ldo;
    A.coef_dev = L.coef_dev;
    A.partials = L.partials;
    L.grid = vec_grid(ctx, L.n, A.tpr);
    // one contiguous column with 16-byte aligned operands: the vector-width kernel
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (L.nr == 1 && L.ldx == 1 && (!L.y || L.ldy == 1) && L.ldo == 1 && al16(L.x) && al16(L.y) && al16(L.out) &&
        (L.coef_dev || !L.b_h || L.b_h[0] == 0.0)) {
        const int slot = prof_begin(ctx, PROF_VEC);
        const double a0 = L.a_h ? L.a_h[0] : 0.0, g0 = L.g_h ? L.g_h[0] : 0.0;
        if (L.real_dtype == HPHI_F64)
            k_lincomb1<double><<<L.grid, kVT, 0, ctx->stream>>>(L.n, (const double *)L.x, (const double *)L.y,
                                                                (double *)L.out, L.coef_dev, a0, g0, L.red_oo,
                                                                L.partials);
        else
            k_lincomb1<float><<<L.grid, kVT, 0, ctx->stream>>>(L.n, (const float *)L.x, (const float *)L.y,
                                                               (float *)L.out, L.coef_dev, a0, g0, L.red_oo,
                                                               L.partials);
        prof_end(ctx, slot);
        HPHI_CUDA(ctx, cudaGetLastError());
        return HPHI_OK;
    }
    for (int c = 0; c < 256; c++) {
        A.a[c] = (c < L.nr && L.a_h) ? L.a_h[c] : 0.0;
        A.b[c] = (c < L.nr && L.b_h) ? L.b_h[c] : 0.0;
        A.g[c] = (c < L.nr && L.g_h) ? L.g_h[c] : 0.0;
    }
    // contiguous rows of several columns with 16-byte aligned operands: the flat kernel
    {
        const int V = L.real_dtype == HPHI_F64 ? 2 : 4;
        const int64_t vstride = (int64_t)kVT * V;  // a multiple of the stride of every grid
        if (L.nr > 1 && L.nr <= 256 && L.nr % V == 0 && vstride % L.nr == 0 && L.ldx == L.nr &&
            (!L.y || L.ldy == L.nr) && L.ldo == L.nr && al16(L.x) && al16(L.y) && al16(L.out)) {
            const int slot = prof_begin(ctx, PROF_VEC);
            if (L.real_dtype == HPHI_F64) k_lincomb_rows<double><<<L.grid, kVT, 0, ctx->stream>>>(A);
            else k_lincomb_rows<float><<<L.grid, kVT, 0, ctx->stream>>>(A);
            prof_end(ctx, slot);
            HPHI_CUDA(ctx, cudaGetLastError());
            return HPHI_OK;
        }
    }
    int slot = prof_begin(ctx, PROF_VEC);
    const int cpl = (L.nr + A.tpr - 1) / A.tpr;
#define HPHI_LC(T, C) k_lincomb<T, C><<<L.grid, kVT, 0, ctx->stream>>>(A)
    if (L.real_dtype == HPHI_F64) {
        if (cpl <= 1) HPHI_LC(double, 1);
        else if (cpl <= 2) HPHI_LC(double, 2);
        else if (cpl <= 4) HPHI_LC(double, 4);
        else HPHI_LC(double, 8);
    } else {
        if (cpl <= 1) HPHI_LC(float, 1);
        else if (cpl <= 2) HPHI_LC(float, 2);
        else if (cpl <= 4) HPHI_LC(float, 4);
        else HPHI_LC(float, 8);
    }
#undef HPHI_LC
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int launch_mdot(hphi_ctx *ctx, int real_dtype, int64_t n, int nv, const void *V, const void *w, double *out_dev) {
    if (nv < 1 || nv > 1024) return set_err(ctx, HPHI_E_INVAL, "1 to 1024 stored vectors");
    int st;
    if (real_dtype == HPHI_F64) {
        // per-tile warp sums would cost more FP64 adds than the products themselves
        int64_t gx = (n + kVT - 1) / kVT;
        if (gx > (int64_t)ctx->sm_count * 4) gx = (int64_t)ctx->sm_count * 4;
        if (gx < 1) gx = 1;
        if ((st = ensure_partials(ctx, (size_t)gx * nv))) return st;
        const int slot = prof_begin(ctx, PROF_VEC);
        dim3 grid((unsigned)gx, (unsigned)((nv + 7) / 8));
        k_mdot<double><<<grid, kVT, 0, ctx->stream>>>(n, nv, (const double *)V, (const double *)w, ctx->partials);
        prof_end(ctx, slot);
        HPHI_CUDA(ctx, cudaGetLastError());
        return reduce_partials(ctx, ctx->partials, (int)gx, nv, out_dev);
    }
    const int64_t tile = (int64_t)kMT * kMR;
    int64_t g = (n + tile - 1) / tile;
    if (g > (int64_t)ctx->sm_count * 8) g = (int64_t)ctx->sm_count * 8;
    if (g < 1) g = 1;
    if ((st = ensure_partials(ctx, (size_t)g * nv))) return st;
    const size_t dyn = sizeof(double) * (kMT / 32) * nv;
    if (dyn > 48 * 1024 && dyn_occupancy(ctx, (const void *)k_mdot_tiled<float>, kMT, dyn) < 1)
        return set_err(ctx, HPHI_E_INVAL, "multi-vector dot: %d vectors need too much shared memory", nv);
    const int slot = prof_begin(ctx, PROF_VEC);
    k_mdot_tiled<float><<<(unsigned)g, kMT, dyn, ctx->stream>>>(n, nv, (const float *)V, (const float *)w,
                                                               ctx->partials);
    k_reduce_wide<<<(nv + 7) / 8, 256, 0, ctx->stream>>>(ctx->partials, (int)g, nv, out_dev);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int launch_maxpy(hphi_ctx *ctx, int real_dtype, int64_t n, int nv, const void *V, const double *c_dev, void *w) {
    if (nv < 1 || nv > 1024) return set_err(ctx, HPHI_E_INVAL, "1 to 1024 stored vectors");
    const int64_t tile = (int64_t)kMT * kMR;
    int64_t g = (n + tile - 1) / tile;
    if (g > (int64_t)ctx->sm_count * 8) g = (int64_t)ctx->sm_count * 8;
    if (g < 1) g = 1;
    const int slot = prof_begin(ctx, PROF_VEC);
    if (real_dtype == HPHI_F64)
        k_maxpy_tiled<double><<<(unsigned)g, kMT, sizeof(double) * nv, ctx->stream>>>(n, nv, (const double *)V, c_dev,
                                                                                      (double *)w);
    else
        k_maxpy_tiled<float><<<(unsigned)g, kMT, sizeof(float) * nv, ctx->stream>>>(n, nv, (const float *)V, c_dev,
                                                                                    (float *)w);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int launch_random(hphi_ctx *ctx, int real_dtype, int64_t n, int nr, uint64_t seed, void *x, int64_t ldx) {
    int64_t total = n * nr;
    int64_t g = (total + 255) / 256;
    if (g > (int64_t)ctx->sm_count * 16) g = (int64_t)ctx->sm_count * 16;
    if (g < 1) g = 1;
    if (real_dtype == HPHI_F64)
        k_random<double><<<(unsigned)g, 256, 0, ctx->stream>>>(n, nr, seed, (double *)x, ldx);
    else
        k_random<float><<<(unsigned)g, 256, 0, ctx->stream>>>(n, nr, seed, (float *)x, ldx);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int launch_copy(hphi_ctx *ctx, int real_dtype, int64_t n, int nr, const void *x, int64_t ldx, void *y, int64_t ldy) {
    int64_t total = n * nr;
    int64_t g = (total + 255) / 256;
    if (g > (int64_t)ctx->sm_count * 16) g = (int64_t)ctx->sm_count * 16;
    if (g < 1) g = 1;
    if (real_dtype == HPHI_F64)
        k_copy<double><<<(unsigned)g, 256, 0, ctx->stream>>>(n, nr, (const double *)x, ldx, (double *)y, ldy);
    else
        k_copy<float><<<(unsigned)g, 256, 0, ctx->stream>>>(n, nr, (const float *)x, ldx, (float *)y, ldy);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace hphi

// ---- dot product with file-scope scratch (no device allocation) ------------
// The partials of the block reduction and the reduced values live in a
// file-scope device array.  Host code cannot use the array's name as a device
// address, so every call looks the address up (cudaGetSymbolAddress, a
// host-side lookup that allocates nothing) with the target device current.
// Nothing is cached, so the address stays valid across cudaDeviceReset and
// concurrent first calls from several threads need no synchronisation.
namespace {

constexpr int kStaticReal = HPHI_DOT_STATIC_MAX_REAL;
constexpr int kStaticBlocks = HPHI_DOT_STATIC_MAX_BLOCKS;
constexpr size_t kStaticDoubles = HPHI_DOT_STATIC_SCRATCH_BYTES / sizeof(double);
static_assert(kStaticDoubles == 2 * kStaticBlocks * kStaticReal + 2 * kStaticReal, "scratch layout");

static __device__ __align__(256) double g_dot_scratch[kStaticDoubles];

// 1 if p is device (or managed) memory that `device` can address directly.
bool on_device(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" int hphi_dot_static(int device, void *stream, int dtype, int64_t n, int nvec, const void *x, int64_t ldx,
                               const void *y, int64_t ldy, double *out) {
    using namespace hphi;
    if (!out || n < 0 || nvec < 1 || !valid_dtype(dtype) || device < 0) return HPHI_E_INVAL;
    const int cpl = is_complex(dtype) ? 2 : 1, nr = nvec * cpl;
    if (nr > kStaticReal) return HPHI_E_INVAL;
    if (ldx < nvec || ldy < nvec || (n > 0 && (!x || !y))) return HPHI_E_INVAL;
    if (n == 0) {
        for (int k = 0; k < nr; k++) out[k] = 0.0;
        return HPHI_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return HPHI_E_CUDA;
    }
    if (device >= ndev) return HPHI_E_INVAL;
    // operands on another device (or in plain host memory) would be read
    // through their unified addresses: refuse them instead
    if (!on_device(x, device) || !on_device(y, device)) return HPHI_E_INVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return HPHI_E_CUDA;
    }
    int rc = HPHI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    do {
        if (cudaSetDevice(device) != cudaSuccess) {
            rc = HPHI_E_CUDA;
            break;
        }
        double *partials = nullptr;
        if (cudaGetSymbolAddress((void **)&partials, g_dot_scratch) != cudaSuccess || !partials) {
            rc = HPHI_E_CUDA;
            break;
        }
        double *result = partials + 2 * kStaticBlocks * kStaticReal;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            rc = HPHI_E_CUDA;
            break;
        }
        // the grid of hphi_dot (vec_grid: SMs x 8 blocks at most), so that both
        // entry points sum in the same order; devices with more than
        // kStaticBlocks / 8 SMs get the capped grid (equal to rounding then)
        const int tpr = tpr_of(nr);
        int64_t g = (n + (kVT / tpr) - 1) / (kVT / tpr);
        int64_t cap = (int64_t)sms * 8;
        if (cap > kStaticBlocks) cap = kStaticBlocks;
        if (g > cap) g = cap;
        const int grid = (int)(g < 1 ? 1 : g);
        const int cplane = (nr + tpr - 1) / tpr;
        const int rd = real_of(dtype);
        const int64_t lx = ldx * cpl, ly = ldy * cpl;
#define HPHI_SDOT(T, C)                                                                                    \
    k_dot<T, C><<<grid, kVT, 0, st>>>(n, nr, tpr, cpl == 2, (const T *)x, lx, (const T *)y, ly, partials)
        if (rd == HPHI_F64) {
            if (cplane <= 1) HPHI_SDOT(double, 1);
            else HPHI_SDOT(double, 2);
        } else {
            if (cplane <= 1) HPHI_SDOT(float, 1);
            else HPHI_SDOT(float, 2);
        }
#undef HPHI_SDOT
        k_reduce<<<1, 256, 0, st>>>(partials, grid, 2 * nr, result);
        if (cudaGetLastError() != cudaSuccess) {
            rc = HPHI_E_CUDA;
            break;
        }
        double host[2 * kStaticReal];
        if (cudaMemcpyAsync(host, result, sizeof(double) * 2 * nr, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = HPHI_E_CUDA;
            break;
        }
        const double *S = host, *X = host + nr;
        for (int q = 0; q < nvec; q++) {
            if (cpl == 1) {
                out[q] = S[q];
            } else {
                out[2 * q] = S[2 * q] + S[2 * q + 1];
                out[2 * q + 1] = X[2 * q] - X[2 * q + 1];
            }
        }
    } while (0);
    if (rc != HPHI_OK) cudaGetLastError();
    cudaSetDevice(prev);
    return rc;
}
