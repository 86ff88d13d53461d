// Real-time evolution (Sec. 3.4): one step
//   Phi(t + dt) = sum_{n<=nmax} (-i dt H)^n / n! Phi(t)
// by Horner stages W <- Phi + (-i dt / j) H W, j = nmax .. 1, one fused H*x
// launch per stage.  A complex column is a pair of real columns (re, im);
// since H is real, (-i c) H (a + i b) = c H b - i c H a: the launch takes the
// partner column of H W ("pair swap") with alpha = +c for the real and -c for
// the imaginary column, and adds Phi through its gamma term.  The first stage
// also reduces <Phi, H Phi>, |H Phi|^2 and |Phi|^2; the last one |Phi(t+dt)|^2.
#include <math.h>

#include <vector>

#include "hphi_internal.cuh"

using namespace hphi;

extern "C" int hphi_time_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv,
                              double dt, int nmax, double *norm2_out, double *e_out, double *h2_out,
                              double *norm2_new_out) {
    if (!ctx || !ham || !V || !norm2_out || !e_out || !h2_out || !norm2_new_out) return HPHI_E_INVAL;
    ctx->err.clear();
    if (dtype != HPHI_C128 && dtype != HPHI_C64) return set_err(ctx, HPHI_E_INVAL, "dtype must be C128 or C64");
    if (nmax < 1 || nmax > 64) return set_err(ctx, HPHI_E_INVAL, "nmax must be in [1, 64]");
    const int nr = 2 * nvec;
    if (nvec < 1 || nr > kMaxCols) return set_err(ctx, HPHI_E_INVAL, "1 <= complex columns <= %d", kMaxCols / 2);
    if (ldv < nvec) return set_err(ctx, HPHI_E_INVAL, "ldv < nvec");
    if (!isfinite(dt)) return set_err(ctx, HPHI_E_INVAL, "dt is not finite");
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int rd = real_of(dtype);
    const int64_t D = ham->D, ld = 2 * ldv;
    const size_t es = real_size(rd);
    int st;
    if ((st = ensure_vecs(ctx, (size_t)D * nr * es))) return st;
    if ((st = ensure_partials(ctx, hv_partials_size(ctx, ham, nr)))) return st;
    void *W[2] = {ctx->vec[0], ctx->vec[1]};
    double *red = ctx->dscal + 2048;  // [3][nr]
    std::vector<double> al(nr), ga(nr, 1.0), first(3 * (size_t)nr), last(nr);
    const void *x = V;
    int64_t ldx = ld;
    for (int j = nmax; j >= 1; j--) {
        const double cj = dt / (double)j;
        // the last stage writes Phi(t + dt) into V, unless it also reads V as x
        const bool out_v = j == 1 && nmax > 1;
        void *out = out_v ? V : W[j & 1];
        const int64_t ldo = out_v ? ld : nr;
        for (int q = 0; q < nvec; q++) {
            al[2 * q] = cj;       // Re out = Re Phi + c Im(H W)
            al[2 * q + 1] = -cj;  // Im out = Im Phi - c Re(H W)
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
        L.swap = 1;
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
        const double xhx = first[2 * q] + first[2 * q + 1];
        const double hxhx = first[nr + 2 * q] + first[nr + 2 * q + 1];
        const double xx = first[2 * (size_t)nr + 2 * q] + first[2 * (size_t)nr + 2 * q + 1];
        const double oo = last[2 * q] + last[2 * q + 1];
        if (!isfinite(xx) || !isfinite(oo) || !isfinite(xhx))
            return set_err(ctx, HPHI_E_NUMERIC, "time step column %d: non-finite values", q);
        norm2_out[q] = xx;
        e_out[q] = xx > 0.0 ? xhx / xx : 0.0;
        h2_out[q] = xx > 0.0 ? hxhx / xx : 0.0;
        norm2_new_out[q] = oo;
    }
    return HPHI_OK;
}
