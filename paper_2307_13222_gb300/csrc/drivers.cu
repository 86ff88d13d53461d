// Drivers built on the H*x kernel: Lanczos ground state (the paper's
// ground-state method, Sec. 1 and Table 1) and one canonical-TPQ step
// (Sec. 3.5.1, U_c = sum_{n<=nmax} (-dtau H/2)^n / n!).
//
// Lanczos keeps the Krylov vectors unnormalised: v_k = w_k / beta_k with
// beta_k = |w_k| (beta_0 = |v0|, w_0 = v0).  One step is
//   u       = (1/beta_k) H w_k - (beta_k/beta_{k-1}) w_{k-1}     (fused H*x)
//   alpha_k = <w_k, u> / beta_k                                  (same pass)
//   w_{k+1} = u - (alpha_k/beta_k) w_k,  beta_{k+1}^2 = |w_{k+1}|^2
// All scalars of the recurrence stay on the device (a one-thread kernel
// derives the next coefficients from the reductions), so a run of steps needs
// no host round trip; the host reads alpha/beta only at convergence checks and
// solves the tridiagonal problem with the implicit QL method.
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "hphi_internal.cuh"

namespace hphi {

// Symmetric tridiagonal eigenproblem by the implicit QL iteration with
// Wilkinson shifts (Bowdler, Martin, Reinsch, Wilkinson, Numer. Math. 11
// (1968) 293).  d[0..n-1] diagonal -> eigenvalues; e[0..n-2] off-diagonal
// (destroyed); z (n*n, row-major, may be null) -> eigenvectors in columns.
int tridiag_ql(int n, double *d, double *e, double *z) {
    if (n <= 0) return HPHI_OK;
    std::vector<double> ee(n, 0.0);
    for (int i = 0; i + 1 < n; i++) ee[i] = e[i];
    if (z)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) z[i * n + j] = i == j ? 1.0 : 0.0;
    for (int l = 0; l < n; l++) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; m++) {
                double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(ee[m]) <= DBL_EPSILON * dd) break;
            }
            if (m == l) break;
            if (++iter > 200) return HPHI_E_NUMERIC;
            double g = (d[l + 1] - d[l]) / (2.0 * ee[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + ee[l] / (g + (g >= 0.0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            bool early = false;
            for (int i = m - 1; i >= l; i--) {
                double f = s * ee[i], b = c * ee[i];
                r = hypot(f, g);
                ee[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    ee[m] = 0.0;
                    early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                if (z) {
                    for (int k = 0; k < n; k++) {
                        double t = z[k * n + i + 1];
                        z[k * n + i + 1] = s * z[k * n + i] + c * t;
                        z[k * n + i] = c * z[k * n + i] - s * t;
                    }
                }
            }
            if (early) continue;
            d[l] -= p;
            ee[l] = g;
            ee[m] = 0.0;
        }
    }
    return HPHI_OK;
}

// Solves (T - s I) x = r in place (r -> x) for the symmetric tridiagonal T with
// diagonal a[0..n-1] and off-diagonal b[1..n-1], by Gaussian elimination with
// partial pivoting (U keeps two super-diagonals); a zero pivot becomes `tiny`.
static void tridiag_shift_solve(int n, const double *a, const double *b, double s, double tiny, double *r) {
    std::vector<double> u0(n), u1(n), u2(n), rhs(n);
    double cd = a[0] - s, ce = n > 1 ? b[1] : 0.0, cf = 0.0, cr = r[0];
    for (int i = 0; i < n; i++) {
        if (i == n - 1) {
            u0[i] = cd != 0.0 ? cd : tiny;
            u1[i] = u2[i] = 0.0;
            rhs[i] = cr;
            break;
        }
        const double g = b[i + 1], hd = a[i + 1] - s, hk = i + 2 < n ? b[i + 2] : 0.0, hr = r[i + 1];
        if (fabs(cd) >= fabs(g)) {  // pivot on the current row
            if (cd == 0.0) cd = tiny;
            const double m = g / cd;
            u0[i] = cd;
            u1[i] = ce;
            u2[i] = cf;
            rhs[i] = cr;
            cd = hd - m * ce;
            ce = hk - m * cf;
            cr = hr - m * cr;
        } else {  // pivot on the next row
            const double m = cd / g;
            u0[i] = g;
            u1[i] = hd;
            u2[i] = hk;
            rhs[i] = hr;
            cd = ce - m * hd;
            ce = cf - m * hk;
            cr = cr - m * hr;
        }
        cf = 0.0;
    }
    for (int i = n - 1; i >= 0; i--) {
        double v = rhs[i];
        if (i + 1 < n) v -= u1[i] * r[i + 1];
        if (i + 2 < n) v -= u2[i] * r[i + 2];
        r[i] = v / u0[i];
    }
}

// Number of eigenvalues of T (diagonal a, off-diagonal b[1..n-1]) below x, from
// the signs of the LDL^T pivots (Sturm sequence); a zero pivot becomes -tiny.
static int sturm_below(int n, const double *a, const double *b, double x, double tiny) {
    int c = 0;
    double d = a[0] - x;
    if (d == 0.0) d = -tiny;
    c += d < 0.0;
    for (int i = 1; i < n; i++) {
        d = a[i] - x - b[i] * b[i] / d;
        if (d == 0.0) d = -tiny;
        c += d < 0.0;
    }
    return c;
}

// Lowest eigenvalue of T_m and the last component of its normalised
// eigenvector: what a convergence check needs, at O(m) cost.  With a warm
// start (*warm finite: e.g. the lowest Ritz value of an earlier T_j, an upper
// bound of this one) Rayleigh-quotient iteration converges in a few O(m)
// solves; its answer is accepted only if the Sturm count shows it is the
// lowest eigenvalue, otherwise (or without a warm start) bisection on the
// Sturm count decides.  *warm receives the result.  The full eigenvector is
// formed only at the end of a run.
int lowest_ritz_warm(int m, const double *alpha, const double *beta2, double *warm, double *theta, double *ylast) {
    std::vector<double> b(m + 1, 0.0), y(m);
    double lo = alpha[0], scale = 0.0;
    for (int j = 1; j < m; j++) b[j] = sqrt(beta2[j]);
    for (int j = 0; j < m; j++) {
        const double r = (j > 0 ? b[j] : 0.0) + (j + 1 < m ? b[j + 1] : 0.0);
        lo = alpha[j] - r < lo ? alpha[j] - r : lo;  // Gershgorin lower bound
        scale = fabs(alpha[j]) + r > scale ? fabs(alpha[j]) + r : scale;
    }
    if (!isfinite(scale)) return HPHI_E_NUMERIC;
    if (scale == 0.0) scale = 1.0;
    const double tiny = DBL_MIN * 4.0, pivot_floor = DBL_EPSILON * scale;
    auto normalise = [&]() -> bool {
        double nn = 0.0;
        for (int j = 0; j < m; j++) nn += y[j] * y[j];
        nn = sqrt(nn);
        if (!(nn > 0.0) || !isfinite(nn)) return false;
        for (int j = 0; j < m; j++) y[j] /= nn;
        return true;
    };
    auto rayleigh = [&]() {
        double s = 0.0;
        for (int j = 0; j < m; j++) {
            double ty = alpha[j] * y[j];
            if (j > 0) ty += b[j] * y[j - 1];
            if (j + 1 < m) ty += b[j + 1] * y[j + 1];
            s += y[j] * ty;
        }
        return s;
    };
    double t = 0.0;
    bool ok = false;
    if (warm && isfinite(*warm) && m > 1) {
        double sig = *warm;
        for (int j = 0; j < m; j++) y[j] = 1.0 / sqrt((double)m);
        for (int it = 0; it < 8; it++) {
            tridiag_shift_solve(m, alpha, b.data(), sig, pivot_floor, y.data());
            if (!normalise()) break;
            const double s2 = rayleigh();
            const bool done = fabs(s2 - sig) <= 4.0 * DBL_EPSILON * scale;
            sig = s2;
            if (done) {
                ok = sturm_below(m, alpha, b.data(), sig + 16.0 * DBL_EPSILON * scale, tiny) == 1;
                break;
            }
        }
        t = sig;
    }
    if (!ok) {
        double hi = alpha[0];  // the lowest eigenvalue is at most the Rayleigh quotient of e_1
        for (int it = 0; it < 200 && hi - lo > 2.0 * DBL_EPSILON * (fabs(lo) + fabs(hi)); it++) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_below(m, alpha, b.data(), mid, tiny) >= 1) hi = mid;
            else lo = mid;
        }
        t = 0.5 * (lo + hi);
        for (int j = 0; j < m; j++) y[j] = 1.0 / sqrt((double)m);
    }
    for (int it = 0; it < (ok ? 1 : 3); it++) {
        tridiag_shift_solve(m, alpha, b.data(), t, pivot_floor, y.data());
        if (!normalise()) return HPHI_E_NUMERIC;
    }
    *theta = t;
    *ylast = fabs(y[m - 1]);
    if (warm) *warm = t;
    return HPHI_OK;
}

int lowest_ritz(int m, const double *alpha, const double *beta2, double *theta, double *ylast) {
    return lowest_ritz_warm(m, alpha, beta2, nullptr, theta, ylast);
}

namespace {

enum LzMode { LZ_INIT = 0, LZ_PREP_A = 1, LZ_ALPHA = 2, LZ_BETA = 3 };

// one thread: scalar bookkeeping of the device-side recurrence
__global__ void k_lz(int mode, int k, const double *red, double *alpha, double *beta2, double *coefA, double *coefB,
                     int *flag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    // *flag records the first step (k + 1) whose scalars were not finite; -1
    // marks a start vector of zero norm
    if (mode == LZ_INIT) {
        beta2[0] = red[0];
        if (!(red[0] > 0.0) || !isfinite(red[0])) *flag = -1;
    } else if (mode == LZ_PREP_A) {
        double bk = sqrt(beta2[k]);
        coefA[0] = 1.0 / bk;
        coefA[1] = k > 0 ? -bk / sqrt(beta2[k - 1]) : 0.0;
    } else if (mode == LZ_ALPHA) {
        double bk = sqrt(beta2[k]);
        double a = red[0] / bk;
        alpha[k] = a;
        coefB[0] = -a / bk;  // coefficient of w_k
        coefB[1] = 0.0;
        coefB[2] = 1.0;      // coefficient of u
        if (!isfinite(a) && *flag == 0) *flag = k + 1;
    } else {
        beta2[k + 1] = red[0];
        if ((!(red[0] >= 0.0) || !isfinite(red[0])) && *flag == 0) *flag = k + 1;
    }
}

// scalar bookkeeping of the reorthogonalising recurrence (normalised vectors)
enum RzMode { RZ_INIT = 0, RZ_PREP = 1, RZ_ALPHA = 2, RZ_BETA = 3 };

__global__ void k_rz(int mode, int k, const double *red, double *alpha, double *beta2, double *coef, int *flag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == RZ_INIT) {
        beta2[0] = red[0];
        if (!(red[0] > 0.0) || !isfinite(red[0])) *flag = -1;
        coef[0] = 1.0 / sqrt(red[0]);  // scale of v_0
        coef[1] = 0.0;
        coef[2] = 0.0;
    } else if (mode == RZ_PREP) {
        coef[0] = 1.0;                               // alpha of H*x
        coef[1] = k > 0 ? -sqrt(beta2[k]) : 0.0;     // gamma: -beta_k v_{k-1}
    } else if (mode == RZ_ALPHA) {
        alpha[k] = red[0];
        coef[0] = -red[0];  // u -= alpha_k v_k
        coef[1] = 0.0;
        coef[2] = 1.0;
        if (!isfinite(red[0]) && *flag == 0) *flag = k + 1;
    } else {
        beta2[k + 1] = red[0];
        coef[0] = 1.0 / sqrt(red[0]);  // v_{k+1} = u / beta_{k+1}
        coef[1] = 0.0;
        coef[2] = 0.0;
        if ((!(red[0] >= 0.0) || !isfinite(red[0])) && *flag == 0) *flag = k + 1;
    }
}

}  // namespace

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_tridiag_eigen(int n, const double *a, const double *b, double *evals, double *evecs) {
    if (n < 1 || !a || !evals || (n > 1 && !b)) return HPHI_E_INVAL;
    std::vector<double> d(a, a + n), e(n, 0.0);
    for (int i = 0; i + 1 < n; i++) e[i] = b[i + 1];
    std::vector<double> z(evecs ? (size_t)n * n : 0);
    int st = tridiag_ql(n, d.data(), e.data(), evecs ? z.data() : nullptr);
    if (st) return st;
    // ascending order of eigenvalues (columns follow)
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) { return d[p] < d[q]; });
    for (int j = 0; j < n; j++) {
        evals[j] = d[idx[j]];
        if (evecs) {
            double sg = z[idx[j]] < 0.0 ? -1.0 : 1.0;  // first component non-negative
            for (int i = 0; i < n; i++) evecs[(size_t)i * n + j] = sg * z[(size_t)i * n + idx[j]];
        }
    }
    return HPHI_OK;
}

// x (FP32) -> w (FP64), exact
__global__ void k_widen(int64_t n, const float *__restrict__ x, double *__restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (double)x[i];
}

// Rayleigh quotient <x|H x> / <x|x> of a device vector in FP64 arithmetic.
// An FP32 vector is widened to FP64 first, so the product and both
// reductions run in double precision: for the ground-state vector of an
// FP32-storage Lanczos run this is the FP64 refinement of the energy (its
// error is quadratic in the vector's error, where the Ritz value of the FP32
// recurrence carries the FP32 rounding of alpha and beta linearly).
// Buffers (D doubles, two for FP32 input) are allocated for the call; when
// they do not fit, *rq is NaN and the call still succeeds.
static int rayleigh_fp64(hphi_ctx *ctx, const hphi_ham *ham, int dt, const void *x, double *rq) {
    *rq = std::nan("");
    const int64_t D = ham->D;
    double *buf = nullptr;
    const size_t nd = (dt == HPHI_F64 ? 1 : 2) * (size_t)D;
    if (cudaMalloc((void **)&buf, nd * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return HPHI_OK;
    }
    const double *x64 = (const double *)x;
    if (dt == HPHI_F32) {
        double *w = buf + D;
        const int64_t g = (D + 255) / 256 < (int64_t)ctx->sm_count * 16 ? (D + 255) / 256 : (int64_t)ctx->sm_count * 16;
        k_widen<<<(int)(g < 1 ? 1 : g), 256, 0, ctx->stream>>>(D, (const float *)x, w);
        x64 = w;
    }
    int st = ensure_partials(ctx, hv_partials_size(ctx, ham, 1));
    double *red = ctx->dscal + 3016;
    if (!st) {
        HvLaunch R{};
        R.dtype_real = HPHI_F64;
        R.ncol = 1;
        R.x = x64;
        R.ldx = 1;
        R.y = buf;
        R.ldy = 1;
        R.alpha_s = 1.0;
        R.red[0] = R_XHX;
        R.red[1] = R_HXHX;
        R.red[2] = R_XX;
        R.partials = ctx->partials;
        st = launch_hv(ctx, ham, R);
        if (!st) st = reduce_hv(ctx, R, red);
    }
    double r[3] = {0.0, 0.0, 0.0};
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(r, red, sizeof(r), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_err(ctx, e, "Rayleigh quotient");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (!st && r[2] > 0.0) *rq = r[0] / r[2];
    return st;
}

// Lanczos with full reorthogonalisation: every normalised Krylov vector is kept
// and each new direction is projected out of all of them twice (classical
// Gram-Schmidt, twice is enough), with FP64 projection coefficients.
static int lanczos_reorth(hphi_ctx *ctx, const hphi_ham *ham, const hphi_lanczos_opts *opts, const void *v0,
                          void *gs_out, double *alpha_host, double *beta_host, hphi_lanczos_result *res) {
    const int dt = opts->dtype, M = opts->max_steps;
    const int check = opts->check_every < 1 ? 1 : opts->check_every;
    const int64_t D = ham->D;
    const size_t es = real_size(dt), vb = (size_t)D * es;
    int st;
    if ((st = ensure_vecs(ctx, vb))) return st;
    size_t np = hv_partials_size(ctx, ham, 1);
    if (np < (size_t)ctx->sm_count * 8 * 2) np = (size_t)ctx->sm_count * 8 * 2;
    if ((st = ensure_partials(ctx, np))) return st;
    char *Vb = nullptr;
    double *sc = nullptr;
    cudaError_t e = cudaMalloc((void **)&Vb, vb * ((size_t)M + 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, HPHI_E_NOMEM, "reorthogonalisation needs %zu bytes for %d Krylov vectors",
                       vb * ((size_t)M + 1), M + 1);
    }
    e = cudaMalloc((void **)&sc, sizeof(double) * (4 * (size_t)M + 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(Vb);
        return set_err(ctx, HPHI_E_NOMEM, "reorthogonalisation scalars");
    }
    double *alpha_d = sc, *beta2_d = sc + M + 1, *cbuf = sc + 2 * (size_t)M + 4;  // cbuf: M + 1 entries
    double *coefA = ctx->dscal + 3000, *coefB = ctx->dscal + 3008, *red = ctx->dscal + 3016;
    auto V = [&](int j) -> void * { return Vb + (size_t)j * vb; };
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(Vb);
        cudaFree(sc);
        return code;
    };
    void *u = ctx->vec[0];
    std::vector<double> alpha_h(M + 1, 0.0), beta2_h(M + 2, 0.0), y;
    int steps = 0, conv = 0, brk = 0;
    double theta = 0.0, resid_est = -1.0, warm = std::nan("");
    auto lincomb = [&](const void *x, const void *yv, void *out, const double *cdev, int red_oo) -> int {
        LinComb B{};
        B.real_dtype = dt;
        B.n = D;
        B.nr = 1;
        B.x = x;
        B.ldx = 1;
        B.y = yv;
        B.ldy = 1;
        B.out = out;
        B.ldo = 1;
        B.coef_dev = cdev;
        B.red_oo = red_oo;
        B.partials = ctx->partials;
        int s2 = launch_lincomb(ctx, B);
        if (!s2 && red_oo) s2 = reduce_partials(ctx, ctx->partials, B.grid, 1, red);
        return s2;
    };
    HPHI_CUDA(ctx, cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->stream));
    if ((st = launch_copy(ctx, dt, D, 1, v0, 1, V(0), 1))) return fail(st);
    if ((st = launch_dot(ctx, dt, 0, D, 1, V(0), 1, V(0), 1, red))) return fail(st);
    k_rz<<<1, 32, 0, ctx->stream>>>(RZ_INIT, 0, red, alpha_d, beta2_d, coefB, ctx->dflag);
    if ((st = lincomb(V(0), nullptr, V(0), coefB, 0))) return fail(st);
    for (int k = 0; k < M; k++) {
        k_rz<<<1, 32, 0, ctx->stream>>>(RZ_PREP, k, red, alpha_d, beta2_d, coefA, ctx->dflag);
        HvLaunch A{};
        A.dtype_real = dt;
        A.ncol = 1;
        A.x = V(k);
        A.ldx = 1;
        A.y = u;
        A.ldy = 1;
        A.v = k > 0 ? V(k - 1) : nullptr;
        A.ldv = 1;
        A.coef_dev = coefA;
        A.red[0] = R_XO;
        A.partials = ctx->partials;
        if ((st = launch_hv(ctx, ham, A)) || (st = reduce_hv(ctx, A, red))) return fail(st);
        k_rz<<<1, 32, 0, ctx->stream>>>(RZ_ALPHA, k, red, alpha_d, beta2_d, coefB, ctx->dflag);
        if ((st = lincomb(V(k), u, u, coefB, 0))) return fail(st);
        for (int pass = 0; pass < 2; pass++) {
            if ((st = launch_mdot(ctx, dt, D, k + 1, Vb, u, cbuf)) ||
                (st = launch_maxpy(ctx, dt, D, k + 1, Vb, cbuf, u)))
                return fail(st);
        }
        if ((st = launch_dot(ctx, dt, 0, D, 1, u, 1, u, 1, red))) return fail(st);
        k_rz<<<1, 32, 0, ctx->stream>>>(RZ_BETA, k, red, alpha_d, beta2_d, coefB, ctx->dflag);
        if ((st = lincomb(u, nullptr, V(k + 1), coefB, 0))) return fail(st);
        HPHI_CUDA(ctx, cudaGetLastError());
        steps = k + 1;
        if ((k + 1) % check == 0 || k + 1 == M) {
            int flag = 0;
            HPHI_CUDA(ctx, cudaMemcpyAsync(alpha_h.data(), alpha_d, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaMemcpyAsync(beta2_h.data(), beta2_d, sizeof(double) * (k + 2), cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            if (flag == -1) return fail(set_err(ctx, HPHI_E_INVAL, "Lanczos: start vector has zero norm"));
            int mstop = k + 1;
            double tn = 0.0;
            for (int j = 0; j <= k; j++) {
                double r = fabs(alpha_h[j]) + (j > 0 ? sqrt(beta2_h[j]) : 0.0) + sqrt(beta2_h[j + 1]);
                tn = r > tn ? r : tn;
                if (sqrt(beta2_h[j + 1]) <= 64.0 * DBL_EPSILON * tn) {
                    mstop = j + 1;
                    brk = 1;
                    break;
                }
            }
            if (flag > 0 && !(brk && mstop <= flag - 1))
                return fail(set_err(ctx, HPHI_E_NUMERIC, "Lanczos: non-finite scalars at step %d", flag - 1));
            double yl = 0.0;
            if ((st = lowest_ritz_warm(mstop, alpha_h.data(), beta2_h.data(), &warm, &theta, &yl)))
                return fail(set_err(ctx, st, "tridiagonal eigensolver failed"));
            resid_est = sqrt(beta2_h[mstop]) * yl;
            steps = mstop;
            if (brk) break;
            if (opts->tol > 0.0 && mstop >= 2 && resid_est <= opts->tol * (fabs(theta) > 1.0 ? fabs(theta) : 1.0)) {
                conv = 1;
                break;
            }
        }
    }
    const int m = steps;
    res->e0 = theta;
    res->resid_est = resid_est;
    res->resid = -1.0;
    res->steps = m;
    res->breakdown = brk;
    if (alpha_host)
        for (int j = 0; j < M; j++) alpha_host[j] = j < m ? alpha_h[j] : 0.0;
    if (beta_host)
        for (int j = 0; j <= M; j++) beta_host[j] = (j >= 1 && j <= m) ? sqrt(beta2_h[j]) : 0.0;
    if (gs_out) {
        {
            std::vector<double> a(alpha_h.begin(), alpha_h.begin() + m), b(m, 0.0), ev(m), Z((size_t)m * m);
            for (int j = 1; j < m; j++) b[j] = sqrt(beta2_h[j]);
            if ((st = hphi_tridiag_eigen(m, a.data(), b.data(), ev.data(), Z.data())))
                return fail(set_err(ctx, st, "tridiagonal eigensolver failed"));
            y.assign(m, 0.0);
            for (int i = 0; i < m; i++) y[i] = Z[(size_t)i * m];
        }
        // x = sum_j y_j v_j, as gs -= sum_j (-y_j) v_j from zero
        std::vector<double> ny(m);
        for (int j = 0; j < m; j++) ny[j] = -y[j];
        HPHI_CUDA(ctx, cudaMemcpyAsync(cbuf, ny.data(), sizeof(double) * m, cudaMemcpyHostToDevice, ctx->stream));
        HPHI_CUDA(ctx, cudaMemsetAsync(gs_out, 0, vb, ctx->stream));
        if ((st = launch_maxpy(ctx, dt, D, m, Vb, cbuf, gs_out))) return fail(st);
        double nrm = 0.0;
        if ((st = hphi_nrm2(ctx, dt, D, 1, gs_out, 1, &nrm))) return fail(st);
        if (!(nrm > 0.0)) return fail(set_err(ctx, HPHI_E_NUMERIC, "ground-state vector has zero norm"));
        double inv = 1.0 / nrm;
        if ((st = hphi_scal(ctx, dt, D, 1, &inv, gs_out, 1))) return fail(st);
        HvLaunch R{};
        R.dtype_real = dt;
        R.ncol = 1;
        R.x = gs_out;
        R.ldx = 1;
        R.y = u;
        R.ldy = 1;
        R.v = gs_out;
        R.ldv = 1;
        R.alpha_s = 1.0;
        R.gamma_s = -theta;
        R.red[0] = R_OO;
        R.partials = ctx->partials;
        if ((st = launch_hv(ctx, ham, R)) || (st = reduce_hv(ctx, R, red))) return fail(st);
        double rr = 0.0;
        HPHI_CUDA(ctx, cudaMemcpyAsync(&rr, red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        res->resid = sqrt(rr);
    }
    fail(HPHI_OK);  // frees the stored Krylov vectors
    res->e0_rq = std::nan("");
    if (gs_out && (st = rayleigh_fp64(ctx, ham, dt, gs_out, &res->e0_rq))) return st;
    if (opts->tol > 0.0 && !conv && !brk)
        return set_err(ctx, HPHI_E_NOTCONV, "Lanczos: tolerance not reached in %d steps", m);
    return HPHI_OK;
}

extern "C" int hphi_lanczos(hphi_ctx *ctx, const hphi_ham *ham, const hphi_lanczos_opts *opts, const void *v0,
                            void *gs_out, double *alpha_host, double *beta_host, hphi_lanczos_result *res) {
    if (!ctx || !ham || !opts || !v0 || !res) return HPHI_E_INVAL;
    ctx->err.clear();
    const int dt = opts->dtype;
    if (dt != HPHI_F64 && dt != HPHI_F32) return set_err(ctx, HPHI_E_INVAL, "Lanczos dtype must be F64 or F32");
    const int M = opts->max_steps;
    if (M < 1 || M > 100000) return set_err(ctx, HPHI_E_INVAL, "max_steps must be in [1, 100000]");
    const int check = opts->check_every < 1 ? 1 : opts->check_every;
    const int64_t D = ham->D;
    const size_t es = real_size(dt);
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    if (opts->reorth != 0 && opts->reorth != 1) return set_err(ctx, HPHI_E_INVAL, "reorth must be 0 or 1");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    if (opts->reorth) return lanczos_reorth(ctx, ham, opts, v0, gs_out, alpha_host, beta_host, res);
    int st;
    if ((st = ensure_vecs(ctx, (size_t)D * es))) return st;
    size_t np = hv_partials_size(ctx, ham, 1);
    if (np < (size_t)ctx->sm_count * 8 * 2) np = (size_t)ctx->sm_count * 8 * 2;
    if ((st = ensure_partials(ctx, np))) return st;
    double *ab = nullptr;
    HPHI_CUDA(ctx, cudaMalloc(&ab, sizeof(double) * (2 * (size_t)M + 4)));
    double *alpha_d = ab, *beta2_d = ab + M + 1;
    double *coefA = ctx->dscal + 3000, *coefB = ctx->dscal + 3008, *red = ctx->dscal + 3016;
    void *prev = ctx->vec[0], *cur = ctx->vec[1], *u = ctx->vec[2];
    std::vector<double> alpha_h(M + 1, 0.0), beta2_h(M + 2, 0.0), y;
    int steps = 0, conv = 0, brk = 0;
    double theta = 0.0, resid_est = -1.0;
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ab);
        return code;
    };
    HPHI_CUDA(ctx, cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->stream));
    if ((st = launch_copy(ctx, dt, D, 1, v0, 1, cur, 1))) return fail(st);
    if ((st = launch_dot(ctx, dt, 0, D, 1, cur, 1, cur, 1, red))) return fail(st);
    k_lz<<<1, 32, 0, ctx->stream>>>(LZ_INIT, 0, red, alpha_d, beta2_d, coefA, coefB, ctx->dflag);

    // convergence check: lowest Ritz value and the residual estimate (warm-started
    // from the previous check's value, an upper bound of the new one)
    double warm = std::nan("");
    auto solve_T = [&](int m) -> int {
        double yl = 0.0;
        int s2 = lowest_ritz_warm(m, alpha_h.data(), beta2_h.data(), &warm, &theta, &yl);
        if (s2) return s2;
        resid_est = sqrt(beta2_h[m]) * yl;
        return HPHI_OK;
    };
    // the Ritz vector of T_m (for the ground-state pass)
    auto full_y = [&](int m) -> int {
        std::vector<double> a(alpha_h.begin(), alpha_h.begin() + m), b(m, 0.0), ev(m), Z((size_t)m * m);
        for (int j = 1; j < m; j++) b[j] = sqrt(beta2_h[j]);
        int s2 = hphi_tridiag_eigen(m, a.data(), b.data(), ev.data(), Z.data());
        if (s2) return s2;
        theta = ev[0];
        y.assign(m, 0.0);
        for (int i = 0; i < m; i++) y[i] = Z[(size_t)i * m];
        return HPHI_OK;
    };

    for (int k = 0; k < M; k++) {
        k_lz<<<1, 32, 0, ctx->stream>>>(LZ_PREP_A, k, red, alpha_d, beta2_d, coefA, coefB, ctx->dflag);
        HvLaunch A{};
        A.dtype_real = dt;
        A.ncol = 1;
        A.x = cur;
        A.ldx = 1;
        A.y = u;
        A.ldy = 1;
        A.v = k > 0 ? prev : nullptr;
        A.ldv = 1;
        A.beta = 0.0;
        A.coef_dev = coefA;
        A.red[0] = R_XO;
        A.partials = ctx->partials;
        if ((st = launch_hv(ctx, ham, A)) || (st = reduce_hv(ctx, A, red))) return fail(st);
        k_lz<<<1, 32, 0, ctx->stream>>>(LZ_ALPHA, k, red, alpha_d, beta2_d, coefA, coefB, ctx->dflag);
        LinComb B{};
        B.real_dtype = dt;
        B.n = D;
        B.nr = 1;
        B.x = cur;
        B.ldx = 1;
        B.y = u;
        B.ldy = 1;
        B.out = u;
        B.ldo = 1;
        B.coef_dev = coefB;
        B.red_oo = 1;
        B.partials = ctx->partials;
        if ((st = launch_lincomb(ctx, B)) || (st = reduce_partials(ctx, ctx->partials, B.grid, 1, red)))
            return fail(st);
        k_lz<<<1, 32, 0, ctx->stream>>>(LZ_BETA, k, red, alpha_d, beta2_d, coefA, coefB, ctx->dflag);
        HPHI_CUDA(ctx, cudaGetLastError());
        void *t = prev;
        prev = cur;
        cur = u;
        u = t;
        steps = k + 1;
        if ((k + 1) % check == 0 || k + 1 == M) {
            int flag = 0;
            HPHI_CUDA(ctx, cudaMemcpyAsync(alpha_h.data(), alpha_d, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaMemcpyAsync(beta2_h.data(), beta2_d, sizeof(double) * (k + 2), cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            if (flag == -1) return fail(set_err(ctx, HPHI_E_INVAL, "Lanczos: start vector has zero norm"));
            // the first step at which beta vanished (an invariant subspace)
            int mstop = k + 1;
            double tn = 0.0;
            for (int j = 0; j <= k; j++) {
                double r = fabs(alpha_h[j]) + (j > 0 ? sqrt(beta2_h[j]) : 0.0) + sqrt(beta2_h[j + 1]);
                tn = r > tn ? r : tn;
                if (sqrt(beta2_h[j + 1]) <= 64.0 * DBL_EPSILON * tn) {
                    mstop = j + 1;
                    brk = 1;
                    break;
                }
            }
            // steps after a vanished beta divide by it; only a non-finite value
            // before the breakdown is an error
            if (flag > 0 && !(brk && mstop <= flag - 1))
                return fail(set_err(ctx, HPHI_E_NUMERIC, "Lanczos: non-finite scalars at step %d", flag - 1));
            if ((st = solve_T(mstop))) return fail(set_err(ctx, st, "tridiagonal eigensolver failed"));
            steps = mstop;
            if (brk) break;
            if (opts->tol > 0.0 && mstop >= 2 && resid_est <= opts->tol * (fabs(theta) > 1.0 ? fabs(theta) : 1.0)) {
                conv = 1;
                break;
            }
        }
    }
    const int m = steps;
    res->e0 = theta;
    res->resid_est = resid_est;
    res->resid = -1.0;
    res->steps = m;
    res->breakdown = brk;
    if (alpha_host)
        for (int j = 0; j < M; j++) alpha_host[j] = j < m ? alpha_h[j] : 0.0;
    if (beta_host)
        for (int j = 0; j <= M; j++) beta_host[j] = (j >= 1 && j <= m) ? sqrt(beta2_h[j]) : 0.0;

    if (gs_out) {
        if ((st = full_y(m))) return fail(set_err(ctx, st, "tridiagonal eigensolver failed"));
        // second pass: regenerate w_k with the stored alpha/beta (the same
        // kernels on the same inputs reproduce the first pass bit for bit) and
        // accumulate x = sum_k y_k v_k = sum_k (y_k / beta_k) w_k
        HPHI_CUDA(ctx, cudaMemsetAsync(gs_out, 0, (size_t)D * es, ctx->stream));
        prev = ctx->vec[0];
        cur = ctx->vec[1];
        u = ctx->vec[2];
        if ((st = launch_copy(ctx, dt, D, 1, v0, 1, cur, 1))) return fail(st);
        for (int k = 0; k < m; k++) {
            double bk = sqrt(beta2_h[k]);
            LinComb G{};
            double ga = y[k] / bk, one = 1.0, zero = 0.0;
            G.real_dtype = dt;
            G.n = D;
            G.nr = 1;
            G.x = cur;
            G.ldx = 1;
            G.y = gs_out;
            G.ldy = 1;
            G.out = gs_out;
            G.ldo = 1;
            G.a_h = &ga;
            G.b_h = &zero;
            G.g_h = &one;
            if ((st = launch_lincomb(ctx, G))) return fail(st);
            if (k + 1 == m) break;
            HvLaunch A{};
            A.dtype_real = dt;
            A.ncol = 1;
            A.x = cur;
            A.ldx = 1;
            A.y = u;
            A.ldy = 1;
            A.v = k > 0 ? prev : nullptr;
            A.ldv = 1;
            A.alpha_s = 1.0 / bk;
            A.gamma_s = k > 0 ? -bk / sqrt(beta2_h[k - 1]) : 0.0;
            if ((st = launch_hv(ctx, ham, A))) return fail(st);
            LinComb B{};
            double ca = -alpha_h[k] / bk;
            B.real_dtype = dt;
            B.n = D;
            B.nr = 1;
            B.x = cur;
            B.ldx = 1;
            B.y = u;
            B.ldy = 1;
            B.out = u;
            B.ldo = 1;
            B.a_h = &ca;
            B.b_h = &zero;
            B.g_h = &one;
            if ((st = launch_lincomb(ctx, B))) return fail(st);
            void *t = prev;
            prev = cur;
            cur = u;
            u = t;
        }
        double nrm = 0.0;
        if ((st = hphi_nrm2(ctx, dt, D, 1, gs_out, 1, &nrm))) return fail(st);
        if (!(nrm > 0.0)) return fail(set_err(ctx, HPHI_E_NUMERIC, "ground-state vector has zero norm"));
        double inv = 1.0 / nrm;
        if ((st = hphi_scal(ctx, dt, D, 1, &inv, gs_out, 1))) return fail(st);
        // explicit residual |H x - theta x|
        HvLaunch R{};
        R.dtype_real = dt;
        R.ncol = 1;
        R.x = gs_out;
        R.ldx = 1;
        R.y = ctx->vec[0];
        R.ldy = 1;
        R.v = gs_out;
        R.ldv = 1;
        R.alpha_s = 1.0;
        R.gamma_s = -theta;
        R.red[0] = R_OO;
        R.partials = ctx->partials;
        if ((st = launch_hv(ctx, ham, R)) || (st = reduce_hv(ctx, R, red))) return fail(st);
        double rr = 0.0;
        HPHI_CUDA(ctx, cudaMemcpyAsync(&rr, red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        res->resid = sqrt(rr);
    }
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ab);
    res->e0_rq = std::nan("");
    if (gs_out && (st = rayleigh_fp64(ctx, ham, dt, gs_out, &res->e0_rq))) return st;
    if (opts->tol > 0.0 && !conv && !brk)
        return set_err(ctx, HPHI_E_NOTCONV, "Lanczos: tolerance not reached in %d steps", m);
    return HPHI_OK;
}

// Microcanonical TPQ (Sec. 3.5.1): U_m = 1 - (dtau / 2) H with dtau = 2 / (l N_s),
// i.e. the cTPQ step with nmax = 1, plus beta_k = k dtau / (1 - u_k / l) from
// u_k = e / N_s of the state the step starts from.
extern "C" int hphi_mtpq_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv,
                              double l, int n_sites, int k, double *norm2_inout, double *e_out, double *h2_out,
                              double *logd_out, double *beta_out) {
    if (!ctx || !ham) return HPHI_E_INVAL;
    if (!(l > 0.0) || !isfinite(l) || n_sites < 1 || k < 0)
        return set_err(ctx, HPHI_E_INVAL, "mTPQ needs l > 0, n_sites >= 1 and k >= 0");
    const double dtau = 2.0 / (l * (double)n_sites);
    const int st = hphi_tpq_step(ctx, ham, dtype, nvec, V, ldv, dtau, 1, norm2_inout, e_out, h2_out, logd_out);
    if (st == HPHI_OK && beta_out) {
        // beta_k = k dtau / (1 - u_k / l), u_k the energy per site of Phi_k (Sec. 3.5.1)
        for (int q = 0; q < nvec; q++) beta_out[q] = (double)k * dtau / (1.0 - e_out[q] / (double)n_sites / l);
    }
    return st;
}

extern "C" int hphi_tpq_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv,
                             double dtau, int nmax, double *norm2, double *e_out, double *h2_out, double *logd_out) {
    if (!ctx || !ham || !V || !norm2 || !e_out || !h2_out || !logd_out) return HPHI_E_INVAL;
    ctx->err.clear();
    if (!valid_dtype(dtype)) return set_err(ctx, HPHI_E_INVAL, "unknown dtype %d", dtype);
    if (nmax < 1 || nmax > 64) return set_err(ctx, HPHI_E_INVAL, "nmax must be in [1, 64]");
    const int cpl = is_complex(dtype) ? 2 : 1, nr = nvec * cpl;
    if (nvec < 1 || nr > kMaxCols) return set_err(ctx, HPHI_E_INVAL, "1 <= real columns <= %d", kMaxCols);
    if (ldv < nvec) return set_err(ctx, HPHI_E_INVAL, "ldv < nvec");
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int rd = real_of(dtype);
    const int64_t D = ham->D;
    const int64_t ld = ldv * cpl;
    const size_t es = real_size(rd);
    int st;
    if ((st = ensure_vecs(ctx, (size_t)D * nr * es))) return st;
    size_t np = hv_partials_size(ctx, ham, nr);
    if ((st = ensure_partials(ctx, np))) return st;
    // |V|^2 where not supplied
    bool need = false;
    for (int q = 0; q < nvec; q++) need = need || !(norm2[q] > 0.0);
    if (need) {
        std::vector<double> nn(nvec);
        if ((st = hphi_nrm2(ctx, dtype, D, nvec, V, ldv, nn.data()))) return st;
        for (int q = 0; q < nvec; q++)
            if (!(norm2[q] > 0.0)) norm2[q] = nn[q] * nn[q];
    }
    std::vector<double> sig(nr), al(nr), ga(nr);
    for (int q = 0; q < nvec; q++) {
        if (!(norm2[q] > 0.0) || !isfinite(norm2[q]))
            return set_err(ctx, HPHI_E_NUMERIC, "column %d has a non-positive norm", q);
        for (int c = 0; c < cpl; c++) sig[q * cpl + c] = 1.0 / sqrt(norm2[q]);
    }
    void *W[2] = {ctx->vec[0], ctx->vec[1]};
    double *red = ctx->dscal + 2048;  // [3][nr]
    std::vector<double> first(3 * nr), last(nr);
    const void *x = V;
    int64_t ldx = ld;
    for (int j = nmax; j >= 1; j--) {
        const double cj = (-0.5 * dtau) / (double)j;
        const bool out_v = (j == 1 && nmax > 1);
        void *out = out_v ? V : W[j & 1];
        int64_t ldo = out_v ? ld : nr;
        for (int c = 0; c < nr; c++) {
            al[c] = j == nmax ? cj * sig[c] : cj;
            ga[c] = sig[c];
        }
        HvLaunch L{};
        L.dtype_real = rd;
        L.ncol = nr;
        L.x = x;
        L.ldx = ldx;
        L.y = out;
        L.ldy = ldo;
        L.v = V;
        L.ldv = ld;
        L.alpha_h = al.data();
        L.gamma_h = ga.data();
        L.partials = ctx->partials;
        if (j == nmax) {
            L.red[0] = R_XHX;
            L.red[1] = R_HXHX;
            L.red[2] = R_XX;
        } else if (j == 1) {
            L.red[0] = R_OO;
        }
        if ((st = launch_hv(ctx, ham, L))) return st;
        if (j == nmax) {
            if ((st = reduce_hv(ctx, L, red))) return st;
            HPHI_CUDA(ctx, cudaMemcpyAsync(first.data(), red, sizeof(double) * 3 * nr, cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
        if (j == 1 && nmax > 1) {
            if ((st = reduce_hv(ctx, L, red))) return st;
            HPHI_CUDA(ctx, cudaMemcpyAsync(last.data(), red, sizeof(double) * nr, cudaMemcpyDeviceToHost,
                                           ctx->stream));
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
        x = out;
        ldx = ldo;
    }
    if (nmax == 1) {
        // the single stage wrote W[1]; copy it into V and take its norms
        if ((st = launch_copy(ctx, rd, D, nr, W[1], nr, V, ld))) return st;
        if ((st = launch_dot(ctx, rd, 0, D, nr, V, ld, V, ld, red))) return st;
        HPHI_CUDA(ctx, cudaMemcpyAsync(last.data(), red, sizeof(double) * nr, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    for (int q = 0; q < nvec; q++) {
        double xhx = 0, hxhx = 0, xx = 0, oo = 0;
        for (int c = 0; c < cpl; c++) {
            xhx += first[0 * nr + q * cpl + c];
            hxhx += first[1 * nr + q * cpl + c];
            xx += first[2 * nr + q * cpl + c];
            oo += last[q * cpl + c];
        }
        if (!(xx > 0.0) || !(oo > 0.0) || !isfinite(oo))
            return set_err(ctx, HPHI_E_NUMERIC, "TPQ column %d: non-finite or zero norm", q);
        e_out[q] = xhx / xx;
        h2_out[q] = hxhx / xx;
        double s2 = 1.0 / norm2[q];
        logd_out[q] = log(oo) - log(s2 * xx);
        norm2[q] = oo;
    }
    return HPHI_OK;
}
