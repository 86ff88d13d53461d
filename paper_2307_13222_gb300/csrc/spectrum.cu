// Dynamical correlation functions (Sec. 3.2):
//   D(z) = <Phi_ex| (z I - H)^{-1} |Phi_ex>,  Phi_ex = O |Phi_0>,
// with the structure-factor excitation O = sum_l A_l S^z_l (A_l = e^{i q l}).
//
// hphi_apply_sz_sum builds Phi_ex: O is diagonal in the S^z basis, so one
// pass over the rows multiplies x by f(s) = sum_l A_l S^z_l(s).  f splits into
// a part of the block's high string and a part of the row's low string
// (spin: high/low halves of the spin string; Hubbard: up/down strings), each
// a sum of byte-table lookups held in shared memory.
//
// hphi_shifted_krylov evaluates D for many shifts z_j from one Krylov run per
// right-hand side.  Each real column b runs the Lanczos recurrence with
// unnormalised vectors (as the ground-state driver does); for real H and
// real b the m-step Galerkin solution of (z - H) x = b is the iterate of the
// shifted COCG method the paper's CG option uses, and both D_m(z) and its
// residual norm follow from alpha/beta alone:
//   D_m(z) = |b|^2 / (z - a_0 - b_1^2 / (z - a_1 - ... - b_{m-1}^2 / (z - a_{m-1}))),
//   |b - (z - H) x_m| / |b| = prod_{k=1..m} b_k / |u_k(z)|,
//   u_1 = z - a_0,  u_k = z - a_{k-1} - b_{k-1}^2 / u_{k-1}
// (u_k = det(z - T_k) / det(z - T_{k-1}); the last component of
// (z - T_m)^{-1} e_1 is prod b / det).  The columns share every kernel
// launch: one block H*x of ncol columns and one vector pass per step.
#include <float.h>
#include <math.h>

#include <complex>
#include <vector>

#include "hphi_internal.cuh"

namespace hphi {

namespace {

constexpr int kSzGroups = 4;  // byte groups of one string (<= 32 bits)

struct SzArgs {
    int model;
    int n;          // spin sector: up spins
    int nlo;        // bits of the low string
    int64_t nh;     // blocks
    const uint64_t *jb;
    const uint32_t *loff;
    const uint32_t *lstate;
    const uint32_t *st_up, *st_dn;
    int64_t ddn;
    int ghi, glo;   // byte groups of the high / low string
    // per-bit weights of the high and low strings (re, im) and the constant
    double whi[2][32], wlo[2][32];
    double c_re, c_im;
    const void *x;
    int64_t ldx;
    void *y;
    int64_t ldy;
};

template <typename T>
__global__ void __launch_bounds__(256) k_szsum(const SzArgs a) {
    __shared__ double th[kSzGroups][256][2];
    __shared__ double tl[kSzGroups][256][2];
    for (int e = threadIdx.x; e < kSzGroups * 256; e += blockDim.x) {
        const int g = e >> 8, b = e & 255;
        double hr = 0.0, hi = 0.0, lr = 0.0, li = 0.0;
        for (int k = 0; k < 8; k++) {
            if (!((b >> k) & 1)) continue;
            const int bit = 8 * g + k;
            if (bit < 32) {
                hr += a.whi[0][bit];
                hi += a.whi[1][bit];
                lr += a.wlo[0][bit];
                li += a.wlo[1][bit];
            }
        }
        th[g][b][0] = hr;
        th[g][b][1] = hi;
        tl[g][b][0] = lr;
        tl[g][b][1] = li;
    }
    __syncthreads();
    const T *x = (const T *)a.x;
    T *y = (T *)a.y;
    for (int64_t h = blockIdx.x; h < a.nh; h += gridDim.x) {
        uint64_t base;
        uint32_t len, cp0 = 0;
        uint32_t hs;
        if (a.model == kSpin) {
            base = a.jb[h];
            if (base == ~0ull) continue;
            const int c = a.n - __popcll((unsigned long long)h);
            cp0 = a.loff[c];
            len = a.loff[c + 1] - cp0;
            hs = (uint32_t)h;
        } else if (a.model == kSpinGC) {
            base = (uint64_t)h << a.nlo;
            len = 1u << a.nlo;
            hs = (uint32_t)h;
        } else {
            base = (uint64_t)h * (uint64_t)a.ddn;
            len = (uint32_t)a.ddn;
            hs = a.st_up[h];
        }
        double fr = a.c_re, fi = a.c_im;
        for (int g = 0; g < a.ghi; g++) {
            const uint32_t b = (hs >> (8 * g)) & 255u;
            fr += th[g][b][0];
            fi += th[g][b][1];
        }
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) {
            uint32_t l;
            if (a.model == kSpin) l = a.lstate[cp0 + q];
            else if (a.model == kSpinGC) l = q;
            else l = a.st_dn[q];
            double gr = fr, gi = fi;
            for (int g = 0; g < a.glo; g++) {
                const uint32_t b = (l >> (8 * g)) & 255u;
                gr += tl[g][b][0];
                gi += tl[g][b][1];
            }
            const uint64_t r = base + q;
            const double xv = (double)x[r * a.ldx];
            y[r * a.ldy] = (T)(gr * xv);
            y[r * a.ldy + 1] = (T)(gi * xv);
        }
    }
}

// Scalar bookkeeping of ncol independent Lanczos recurrences (one thread per
// column).  Unnormalised vectors w_k, beta_k = |w_k|:
//   u = (1/beta_k) H w_k - (beta_k/beta_{k-1}) w_{k-1},  alpha_k = <w_k, u>/beta_k,
//   w_{k+1} = u - (alpha_k/beta_k) w_k,  beta_{k+1}^2 = |w_{k+1}|^2.
// A column stops (its coefficients become 0, so its vectors become 0) when
// beta_{k+1} <= 64 eps max_j(|alpha_j| + beta_j + beta_{j+1}) (an invariant
// subspace), or when a scalar is not finite (flagged); nstep[c] records its
// number of steps.
enum KzMode { KZ_INIT = 0, KZ_PREP = 1, KZ_ALPHA = 2, KZ_BETA = 3 };

__global__ void k_kz(int mode, int k, int ncol, const double *red, double *alpha, double *beta2, double *coefA,
                     double *coefB, int *active, int *nstep, double *tn, int *flag) {
    const int c = threadIdx.x;
    if (c >= ncol) return;
    if (mode == KZ_INIT) {
        const double b2 = red[c];
        beta2[c] = b2;
        tn[c] = 0.0;
        nstep[c] = 0;
        active[c] = (b2 > 0.0 && isfinite(b2)) ? 1 : 0;
        if (!isfinite(b2)) atomicCAS(flag, 0, 1);
        return;
    }
    const bool on = active[c] != 0;
    if (mode == KZ_PREP) {
        const double bk = on ? sqrt(beta2[(size_t)k * ncol + c]) : 0.0;
        coefA[c] = on ? 1.0 / bk : 0.0;
        coefA[ncol + c] = (on && k > 0) ? -bk / sqrt(beta2[(size_t)(k - 1) * ncol + c]) : 0.0;
    } else if (mode == KZ_ALPHA) {
        double a = 0.0;
        if (on) {
            const double bk = sqrt(beta2[(size_t)k * ncol + c]);
            a = red[c] / bk;
            coefB[c] = -a / bk;  // coefficient of w_k
            coefB[2 * ncol + c] = 1.0;
            if (!isfinite(a)) atomicCAS(flag, 0, k + 2);
        } else {
            coefB[c] = 0.0;
            coefB[2 * ncol + c] = 0.0;
        }
        coefB[ncol + c] = 0.0;
        alpha[(size_t)k * ncol + c] = a;
    } else {
        if (!on) {
            beta2[(size_t)(k + 1) * ncol + c] = 0.0;
            return;
        }
        const double b2 = red[c];
        beta2[(size_t)(k + 1) * ncol + c] = b2;
        const double bk = sqrt(beta2[(size_t)k * ncol + c]), bn = sqrt(b2 > 0.0 ? b2 : 0.0);
        const double r = fabs(alpha[(size_t)k * ncol + c]) + (k > 0 ? bk : 0.0) + bn;
        const double t = r > tn[c] ? r : tn[c];
        tn[c] = t;
        nstep[c] = k + 1;
        if (!isfinite(b2)) {
            atomicCAS(flag, 0, k + 2);
            active[c] = 0;
        } else if (bn <= 64.0 * DBL_EPSILON * t) {
            active[c] = 0;
        }
    }
}

// Residual recurrence state of one (column, shift) pair on the host.
struct ShiftState {
    std::complex<double> u;  // u_k(z)
    double rho;              // prod b_j / |u_j|
};

}  // namespace

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_apply_sz_sum(hphi_ctx *ctx, const hphi_basis *basis, int dtype, const void *x, int64_t ldx,
                                 void *y, int64_t ldy, const double *a_host) {
    if (!ctx || !basis || !x || !y || !a_host) return HPHI_E_INVAL;
    ctx->err.clear();
    if (dtype != HPHI_F64 && dtype != HPHI_F32) return set_err(ctx, HPHI_E_INVAL, "dtype must be F64 or F32");
    if (ldx < 1 || ldy < 2) return set_err(ctx, HPHI_E_INVAL, "ldx >= 1 and ldy >= 2 required");
    if (basis->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "basis belongs to another device");
    const size_t es = real_size(dtype);
    const int64_t D = basis->D;
    {
        const char *x0 = (const char *)x, *x1 = x0 + ((D - 1) * ldx + 1) * es;
        const char *y0 = (const char *)y, *y1 = y0 + ((D - 1) * ldy + 2) * es;
        if (x0 < y1 && y0 < x1) return set_err(ctx, HPHI_E_INVAL, "x and y overlap");
    }
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int N = basis->N;
    SzArgs a{};
    a.model = basis->model;
    a.x = x;
    a.ldx = ldx;
    a.y = y;
    a.ldy = ldy;
    // S^z_l = n_l - 1/2 (spin), (n_{l up} - n_{l dn}) / 2 (Hubbard)
    if (basis->model == HPHI_HUBBARD) {
        const Species &u = basis->sp[0], &d = basis->sp[1];
        a.nh = u.dim;
        a.ddn = d.dim;
        a.st_up = u.states;
        a.st_dn = d.states;
        a.ghi = a.glo = (N + 7) / 8;
        for (int l = 0; l < N; l++) {
            a.whi[0][l] = 0.5 * a_host[2 * l];
            a.whi[1][l] = 0.5 * a_host[2 * l + 1];
            a.wlo[0][l] = -0.5 * a_host[2 * l];
            a.wlo[1][l] = -0.5 * a_host[2 * l + 1];
        }
    } else {
        const Species &s = basis->sp[0];
        a.nlo = s.nlo;
        a.nh = (int64_t)1 << s.nhi;
        a.n = basis->nup;
        a.jb = s.jb;
        a.loff = s.loff;
        a.lstate = s.lstate;
        a.glo = (s.nlo + 7) / 8;
        a.ghi = (s.nhi + 7) / 8;
        for (int l = 0; l < N; l++) {
            const int hi = l >= s.nlo;
            const int bit = hi ? l - s.nlo : l;
            (hi ? a.whi : a.wlo)[0][bit] = a_host[2 * l];
            (hi ? a.whi : a.wlo)[1][bit] = a_host[2 * l + 1];
            a.c_re -= 0.5 * a_host[2 * l];
            a.c_im -= 0.5 * a_host[2 * l + 1];
        }
    }
    int64_t grid = a.nh < (int64_t)ctx->sm_count * 8 ? a.nh : (int64_t)ctx->sm_count * 8;
    if (grid < 1) grid = 1;
    const int slot = prof_begin(ctx, PROF_VEC);
    if (dtype == HPHI_F64) k_szsum<double><<<(int)grid, 256, 0, ctx->stream>>>(a);
    else k_szsum<float><<<(int)grid, 256, 0, ctx->stream>>>(a);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

extern "C" int hphi_shifted_krylov(hphi_ctx *ctx, const hphi_ham *ham, const hphi_krylov_opts *opts, int ncol,
                                   const void *b, int64_t ldb, int nz, const double *z_host, double *g_host,
                                   double *resid_host, double *alpha_host, double *beta_host,
                                   hphi_krylov_result *res) {
    if (!ctx || !ham || !opts || !b || !z_host || !g_host || !res) return HPHI_E_INVAL;
    ctx->err.clear();
    const int dt = opts->dtype;
    if (dt != HPHI_F64 && dt != HPHI_F32) return set_err(ctx, HPHI_E_INVAL, "dtype must be F64 or F32");
    const int M = opts->max_steps;
    if (M < 1 || M > 100000) return set_err(ctx, HPHI_E_INVAL, "max_steps must be in [1, 100000]");
    if (ncol < 1 || ncol > 64) return set_err(ctx, HPHI_E_INVAL, "1 <= ncol <= 64 right-hand sides");
    if (ldb < ncol) return set_err(ctx, HPHI_E_INVAL, "ldb < ncol");
    if (nz < 1) return set_err(ctx, HPHI_E_INVAL, "nz >= 1 shifts required");
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    const int check = opts->check_every < 1 ? 1 : opts->check_every;
    const int64_t D = ham->D;
    const size_t es = real_size(dt);
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    // the Krylov block is [D][w]: more than two columns are padded with zero
    // columns (inactive from the start) to the 32-wide row layout of the
    // block H*x kernels
    const int w = ncol <= 2 ? ncol : (ncol <= 32 ? 32 : 64);
    int st;
    if ((st = ensure_vecs(ctx, (size_t)D * w * es))) return st;
    size_t np = hv_partials_size(ctx, ham, w);
    const size_t nl = (size_t)ctx->sm_count * 8 * (size_t)w * 2;
    if (np < nl) np = nl;
    if ((st = ensure_partials(ctx, np))) return st;
    // device scalars: alpha [M][ncol], beta2 [M+1][ncol], coefA [2 ncol], coefB [3 ncol],
    // red [3 ncol], tn [ncol]; ints: active, nstep [ncol], flag
    const size_t nd = (size_t)M * w + (size_t)(M + 1) * w + 9 * (size_t)w;
    double *sc = nullptr;
    int *iv = nullptr;
    if (cudaMalloc(&sc, nd * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&iv, (2 * (size_t)w + 1) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sc);
        return set_err(ctx, HPHI_E_NOMEM, "Krylov scalars");
    }
    double *alpha_d = sc, *beta2_d = alpha_d + (size_t)M * w, *coefA = beta2_d + (size_t)(M + 1) * w;
    double *coefB = coefA + 2 * w, *red = coefB + 3 * w, *tn = red + 3 * w;
    int *active = iv, *nstep = iv + w, *flag = iv + 2 * w;
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(sc);
        cudaFree(iv);
        return code;
    };
    void *prev = ctx->vec[0], *cur = ctx->vec[1], *u = ctx->vec[2];
    HPHI_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    if (w > ncol) HPHI_CUDA(ctx, cudaMemsetAsync(cur, 0, (size_t)D * w * es, ctx->stream));
    if ((st = launch_copy(ctx, dt, D, ncol, b, ldb, cur, w))) return fail(st);
    if ((st = launch_dot(ctx, dt, 0, D, w, cur, w, cur, w, red))) return fail(st);
    const int kt = w <= 32 ? 32 : 64;
    k_kz<<<1, kt, 0, ctx->stream>>>(KZ_INIT, 0, w, red, alpha_d, beta2_d, coefA, coefB, active, nstep, tn, flag);

    std::vector<double> ah((size_t)M * w), b2h((size_t)(M + 1) * w);
    std::vector<int> nsh(w), acth(w);
    std::vector<ShiftState> ss((size_t)ncol * nz);
    std::vector<int> done_to(ncol, 0);  // steps folded into ss
    for (auto &s : ss) s = ShiftState{std::complex<double>(0.0, 0.0), 1.0};
    int steps = 0, conv = 0;
    double max_resid = 0.0;
    for (int k = 0; k < M; k++) {
        k_kz<<<1, kt, 0, ctx->stream>>>(KZ_PREP, k, w, red, alpha_d, beta2_d, coefA, coefB, active, nstep, tn,
                                        flag);
        HvLaunch A{};
        A.dtype_real = dt;
        A.ncol = w;
        A.x = cur;
        A.ldx = w;
        A.y = u;
        A.ldy = w;
        A.v = k > 0 ? prev : nullptr;
        A.ldv = w;
        A.coef_dev = coefA;
        A.red[0] = R_XO;
        A.partials = ctx->partials;
        if ((st = launch_hv(ctx, ham, A)) || (st = reduce_hv(ctx, A, red))) return fail(st);
        k_kz<<<1, kt, 0, ctx->stream>>>(KZ_ALPHA, k, w, red, alpha_d, beta2_d, coefA, coefB, active, nstep, tn,
                                        flag);
        LinComb B{};
        B.real_dtype = dt;
        B.n = D;
        B.nr = w;
        B.x = cur;
        B.ldx = w;
        B.y = u;
        B.ldy = w;
        B.out = u;
        B.ldo = w;
        B.coef_dev = coefB;
        B.red_oo = 1;
        B.partials = ctx->partials;
        if ((st = launch_lincomb(ctx, B)) || (st = reduce_partials(ctx, ctx->partials, B.grid, w, red)))
            return fail(st);
        k_kz<<<1, kt, 0, ctx->stream>>>(KZ_BETA, k, w, red, alpha_d, beta2_d, coefA, coefB, active, nstep, tn,
                                        flag);
        HPHI_CUDA(ctx, cudaGetLastError());
        void *t = prev;
        prev = cur;
        cur = u;
        u = t;
        steps = k + 1;
        if ((k + 1) % check != 0 && k + 1 != M) continue;
        int fl = 0;
        HPHI_CUDA(ctx, cudaMemcpyAsync(ah.data(), alpha_d, sizeof(double) * (size_t)(k + 1) * w,
                                       cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(b2h.data(), beta2_d, sizeof(double) * (size_t)(k + 2) * w,
                                       cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(nsh.data(), nstep, sizeof(int) * w, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(acth.data(), active, sizeof(int) * w, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (fl == 1) return fail(set_err(ctx, HPHI_E_NUMERIC, "Krylov: right-hand side norm is not finite"));
        if (fl > 1) return fail(set_err(ctx, HPHI_E_NUMERIC, "Krylov: non-finite scalars at step %d", fl - 2));
        // fold the new steps of every column into the residual recurrences
        max_resid = 0.0;
        bool all = true;
        for (int c = 0; c < ncol; c++) {
            const int m = nsh[c];
            for (int j = done_to[c]; j < m; j++) {
                const double aj = ah[(size_t)j * w + c];
                const double bj1 = sqrt(b2h[(size_t)(j + 1) * w + c] > 0.0 ? b2h[(size_t)(j + 1) * w + c] : 0.0);
                const double bj2 = j > 0 ? b2h[(size_t)j * w + c] : 0.0;
                for (int q = 0; q < nz; q++) {
                    ShiftState &s = ss[(size_t)c * nz + q];
                    const std::complex<double> z(z_host[2 * q], z_host[2 * q + 1]);
                    s.u = j == 0 ? z - aj : z - aj - bj2 / s.u;
                    s.rho = s.rho * bj1 / std::abs(s.u);
                }
            }
            done_to[c] = m;
            if (b2h[c] <= 0.0) continue;  // zero right-hand side
            for (int q = 0; q < nz; q++) {
                const double r = acth[c] ? ss[(size_t)c * nz + q].rho : 0.0;
                max_resid = r > max_resid ? r : max_resid;
                if (acth[c] && !(r <= opts->tol)) all = false;
            }
        }
        bool any_active = false;
        for (int c = 0; c < ncol; c++) any_active = any_active || acth[c];
        if (!any_active || (opts->tol > 0.0 && all)) {
            conv = 1;
            break;
        }
    }
    // continued fractions over each column's own steps
    for (int c = 0; c < ncol; c++) {
        const int m = nsh[c];
        const double n2 = b2h[c];
        for (int q = 0; q < nz; q++) {
            const std::complex<double> z(z_host[2 * q], z_host[2 * q + 1]);
            std::complex<double> g(0.0, 0.0);
            if (n2 > 0.0 && m > 0) {
                std::complex<double> f = z - ah[(size_t)(m - 1) * w + c];
                for (int j = m - 2; j >= 0; j--) f = z - ah[(size_t)j * w + c] - b2h[(size_t)(j + 1) * w + c] / f;
                g = n2 / f;
            }
            g_host[2 * ((size_t)c * nz + q)] = g.real();
            g_host[2 * ((size_t)c * nz + q) + 1] = g.imag();
            if (resid_host) resid_host[(size_t)c * nz + q] = (n2 > 0.0 && acth[c]) ? ss[(size_t)c * nz + q].rho : 0.0;
        }
        if (alpha_host)
            for (int j = 0; j < M; j++) alpha_host[(size_t)c * M + j] = j < m ? ah[(size_t)j * w + c] : 0.0;
        if (beta_host)
            for (int j = 0; j <= M; j++)
                beta_host[(size_t)c * (M + 1) + j] = j <= m ? sqrt(b2h[(size_t)j * w + c] > 0.0 ? b2h[(size_t)j * w + c] : 0.0) : 0.0;
    }
    res->steps = steps;
    res->converged = conv;
    res->max_resid = max_resid;
    fail(HPHI_OK);
    if (opts->tol > 0.0 && !conv) return set_err(ctx, HPHI_E_NOTCONV, "shifted Krylov: tolerance not reached in %d steps", steps);
    return HPHI_OK;
}
