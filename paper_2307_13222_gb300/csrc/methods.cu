// Method arithmetic on top of the drivers, behind the C ABI:
//   hphi_tpq_bootstrap  E(T), C(T) and their standard deviations from TPQ
//                       samples by the paper's bootstrap (Sec. 3.5.1);
//   hphi_szz_spectrum   the spin structure factor S^zz(q, omega) of Sec. 3.2:
//                       excitations of every wave number, one shifted-Krylov
//                       run, D_q = D_a + D_b and -Im D.
#include <math.h>

#include <vector>

#include "hphi_internal.cuh"

namespace hphi {

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the host: ten rounds
// of two 32x32->64 multiplications (0xD2511F53, 0xCD9E8D57), key bumped by
// the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.
void philox10_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = 0xD2511F53ull * c[0], p1 = 0xCD9E8D57ull * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)p1;
        c[2] = n2;
        c[3] = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// sample index of resampling slot e: floor(U n), U the 53-bit uniform of
// output words 0 and 1 of stream element e
int32_t philox_pick(uint64_t e, uint64_t seed, int n) {
    uint32_t c[4] = {(uint32_t)e, (uint32_t)(e >> 32), 0u, 0u};
    philox10_host(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t w = ((uint64_t)c[1] << 32) | c[0];
    const double u = ((double)(w >> 11) + 0.5) * 0x1.0p-53;
    int64_t k = (int64_t)floor(u * (double)n);
    if (k > n - 1) k = n - 1;
    return (int32_t)k;
}

}  // namespace

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_tpq_bootstrap(int n_samples, int n_temps, const double *e, const double *h2,
                                  const double *log_norm, const double *beta, int P, int M, const int32_t *picks,
                                  uint64_t seed, double *e_mean, double *e_sd, double *c_mean, double *c_sd) {
    if (n_samples < 1 || n_temps < 1 || P < 1 || M < 1) return HPHI_E_INVAL;
    if (!e || !h2 || !log_norm || !e_mean || !e_sd || (!c_mean != !c_sd)) return HPHI_E_INVAL;
    std::vector<int32_t> R((size_t)M * P);
    for (int64_t s = 0; s < (int64_t)M * P; s++) {
        R[s] = picks ? picks[s] : philox_pick((uint64_t)s, seed, n_samples);
        if (R[s] < 0 || R[s] >= n_samples) return HPHI_E_INVAL;
    }
    std::vector<double> w(n_samples), em(M), cm(M);
    for (int k = 0; k < n_temps; k++) {
        // norms relative to sample 0's (the paper's W(beta_k))
        for (int n = 0; n < n_samples; n++) {
            w[n] = exp(log_norm[(size_t)n * n_temps + k] - log_norm[k]);
            if (!isfinite(w[n])) return HPHI_E_NUMERIC;
        }
        const double b2 = beta ? beta[k] * beta[k] : 1.0;
        for (int m = 0; m < M; m++) {
            double z = 0.0, a1 = 0.0, a2 = 0.0;
            for (int p = 0; p < P; p++) {
                const int n = R[(size_t)m * P + p];
                z += w[n];
                a1 += w[n] * e[(size_t)n * n_temps + k];
                a2 += w[n] * h2[(size_t)n * n_temps + k];
            }
            if (!(z > 0.0) || !isfinite(z)) return HPHI_E_NUMERIC;
            const double h = a1 / z, hh = a2 / z;
            em[m] = h;
            cm[m] = b2 * (hh - h * h);
        }
        auto mean_sd = [&](const std::vector<double> &x, double *mu, double *sd) {
            double s = 0.0;
            for (int m = 0; m < M; m++) s += x[m];
            const double mean = s / M;
            double q = 0.0;
            for (int m = 0; m < M; m++) q += (x[m] - mean) * (x[m] - mean);
            *mu = mean;
            *sd = M > 1 ? sqrt(q / (M - 1)) : 0.0;
        };
        mean_sd(em, &e_mean[k], &e_sd[k]);
        if (c_mean) mean_sd(cm, &c_mean[k], &c_sd[k]);
    }
    return HPHI_OK;
}

extern "C" int hphi_szz_spectrum(hphi_ctx *ctx, const hphi_ham *ham, const hphi_krylov_opts *opts, const void *gs,
                                 int nq, const double *q_host, int nz, const double *z_host, double *s_host,
                                 double *d_host, double *resid_host, hphi_krylov_result *result) {
    if (!ctx || !ham || !opts || !gs || !q_host || !z_host || !s_host || !result) return HPHI_E_INVAL;
    ctx->err.clear();
    const int dt = opts->dtype;
    if (dt != HPHI_F64 && dt != HPHI_F32) return set_err(ctx, HPHI_E_INVAL, "dtype must be F64 or F32");
    if (nq < 1 || nz < 1) return set_err(ctx, HPHI_E_INVAL, "nq >= 1 and nz >= 1 required");
    const hphi_basis *basis = ham->basis;
    const int L = basis->N;
    // columns of each wave number: Re always, Im unless sin(q l) vanishes on every site
    std::vector<int> two(nq), col(nq + 1, 0);
    for (int k = 0; k < nq; k++) {
        double mx = 0.0;
        for (int l = 0; l < L; l++) mx = fmax(mx, fabs(sin(q_host[k] * l)));
        two[k] = mx > 1e-12;
        col[k + 1] = col[k] + (two[k] ? 2 : 1);
    }
    const int ncol = col[nq];
    if (ncol > 64) return set_err(ctx, HPHI_E_INVAL, "%d excitation columns (at most 64)", ncol);
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t D = ham->D, ld = ncol + 1;
    void *blk = nullptr;
    if (cudaMalloc(&blk, (size_t)D * ld * real_size(dt)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, HPHI_E_NOMEM, "excitation block");
    }
    // Phi_q into columns col[q] (Re) and col[q] + 1 (Im); a real-only q's
    // (zero) Im column is overwritten by the next q's Re, or lands in the
    // spare last column
    std::vector<double> a(2 * (size_t)L);
    int st = HPHI_OK;
    for (int k = 0; k < nq && !st; k++) {
        for (int l = 0; l < L; l++) {
            a[2 * l] = cos(q_host[k] * l);
            a[2 * l + 1] = two[k] ? sin(q_host[k] * l) : 0.0;
        }
        st = hphi_apply_sz_sum(ctx, basis, dt, gs, 1, (char *)blk + (size_t)col[k] * real_size(dt), ld, a.data());
    }
    std::vector<double> g(2 * (size_t)ncol * nz), res((size_t)ncol * nz);
    if (!st || st == HPHI_E_NOTCONV) {
        if (!st) st = hphi_shifted_krylov(ctx, ham, opts, ncol, blk, ld, nz, z_host, g.data(), res.data(), nullptr,
                                          nullptr, result);
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(blk);
    if (st != HPHI_OK && st != HPHI_E_NOTCONV) return st;
    for (int k = 0; k < nq; k++) {
        for (int j = 0; j < nz; j++) {
            const size_t a0 = (size_t)col[k] * nz + j, a1 = a0 + nz;
            double re = g[2 * a0], im = g[2 * a0 + 1], r = res[a0];
            if (two[k]) {
                re += g[2 * a1];
                im += g[2 * a1 + 1];
                r = fmax(r, res[a1]);
            }
            s_host[(size_t)k * nz + j] = -im;
            if (d_host) {
                d_host[2 * ((size_t)k * nz + j)] = re;
                d_host[2 * ((size_t)k * nz + j) + 1] = im;
            }
            if (resid_host) resid_host[(size_t)k * nz + j] = r;
        }
    }
    return st;
}
