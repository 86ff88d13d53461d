// LOBPCG (Sec. 3.3): the lowest m eigenpairs of H from block H*V products.
//
// The iterate keeps three blocks of m columns, the residuals R, the Ritz
// vectors Phi and the search directions P, with their images H R, H Phi, H P
// (only H R is a new product per iteration).  Each iteration solves the
// Rayleigh-Ritz problem on V = [R, Phi, P]:
//   A = V^T H V,  G = V^T V,  A c = lambda G c,
// and updates Phi = V c, H Phi = (H V) c, P = [R, 0, P] c, H P = [H R, 0, H P] c
// with the m lowest lambda.  On the device: the block H*V kernels, a Gram
// kernel (V^T W, fixed-order partial sums) and a block-combination kernel.
// On the host (dimension <= 3m): G is diagonalised and directions with
// eigenvalues below 1e-12 of the largest are dropped (the basis
// B = U_k Lambda_k^{-1/2} makes the reduced problem standard, which also
// guards against the loss of linear independence near convergence), then
// B^T A B is diagonalised, both by the cyclic Jacobi method.  FP64.  No
// preconditioner (T = identity).
#include <float.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "hphi_internal.cuh"

namespace hphi {
namespace {

constexpr int kMaxBlk = 3;    // sub-blocks of V
constexpr int kMaxM = 32;     // columns per sub-block
constexpr int kGT = 256;      // threads of the Gram kernel
constexpr int kTile = 16;     // rows per shared tile

struct Blocks {
    const double *p[kMaxBlk];  // sub-block j: [D][m], leading dimension m
    int nb;                    // sub-blocks
};

// partial[g][i][j] = sum over this block's rows of V[r][i] W[r][j]
__global__ void __launch_bounds__(kGT) k_gram(int64_t D, int m, Blocks V, Blocks W, double *partial) {
    __shared__ double vs[kTile][kMaxBlk * kMaxM];
    __shared__ double ws[kTile][kMaxBlk * kMaxM];
    const int na = V.nb * m, nbw = W.nb * m, ne = na * nbw;
    constexpr int kPer = (kMaxBlk * kMaxM * kMaxBlk * kMaxM + kGT - 1) / kGT;  // entries per thread
    double acc[kPer];
#pragma unroll
    for (int e = 0; e < kPer; e++) acc[e] = 0.0;
    const int64_t per = (D + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = r0 + per < D ? r0 + per : D;
    for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
        const int nt = (int)(r1 - t0 < kTile ? r1 - t0 : kTile);
        for (int e = threadIdx.x; e < nt * na; e += blockDim.x) {
            const int t = e / na, i = e % na;
            vs[t][i] = V.p[i / m][(t0 + t) * m + (i % m)];
        }
        for (int e = threadIdx.x; e < nt * nbw; e += blockDim.x) {
            const int t = e / nbw, j = e % nbw;
            ws[t][j] = W.p[j / m][(t0 + t) * m + (j % m)];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int e = threadIdx.x + k * kGT;
            if (e < ne) {
                const int i = e / nbw, j = e % nbw;
                double a = acc[k];
                for (int t = 0; t < nt; t++) a = fma(vs[t][i], ws[t][j], a);
                acc[k] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        const int e = threadIdx.x + k * kGT;
        if (e < ne) partial[(int64_t)blockIdx.x * ne + e] = acc[k];
    }
}

// Y[r][j] = sum_i X[r][i] C[i][j], X = [X_0, X_1, X_2] (sub-blocks [D][m]), C [nx][m]
__global__ void __launch_bounds__(256) k_combine(int64_t D, int m, Blocks X, const double *C, double *Y) {
    __shared__ double cs[kMaxBlk * kMaxM * kMaxM];
    const int nx = X.nb * m;
    for (int e = threadIdx.x; e < nx * m; e += blockDim.x) cs[e] = C[e];
    __syncthreads();
    const int rows = blockDim.x / m;  // rows per pass (m divides 256 is not required: extra threads idle)
    const int j = threadIdx.x % m, rl = threadIdx.x / m;
    if (rl >= rows) return;
    for (int64_t r = (int64_t)blockIdx.x * rows + rl; r < D; r += (int64_t)gridDim.x * rows) {
        double y = 0.0;
        for (int b = 0; b < X.nb; b++) {
            const double *x = X.p[b] + r * m;
            for (int i = 0; i < m; i++) y = fma(x[i], cs[(b * m + i) * m + j], y);
        }
        Y[r * m + j] = y;
    }
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row-major,
// destroyed): eigenvalues w (ascending), eigenvectors in the columns of V.
void jacobi_eig(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                const double a = A[(size_t)i * n + j];
                tot += a * a;
                if (i != j) off += a * a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {  // A <- J^T A J
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    std::vector<double> V2((size_t)n * n);
    w.resize(n);
    for (int c = 0; c < n; c++) {
        w[c] = A[(size_t)idx[c] * n + idx[c]];
        for (int r = 0; r < n; r++) V2[(size_t)r * n + c] = V[(size_t)r * n + idx[c]];
    }
    V.swap(V2);
}

}  // namespace
}  // namespace hphi

using namespace hphi;

extern "C" int hphi_lobpcg(hphi_ctx *ctx, const hphi_ham *ham, int m, void *X, int max_iter, double tol,
                           double *evals, double *resid, int *iters) {
    if (!ctx || !ham || !X || !evals || !resid || !iters) return HPHI_E_INVAL;
    ctx->err.clear();
    if (m < 1 || m > kMaxM) return set_err(ctx, HPHI_E_INVAL, "block size m must be in [1, %d]", kMaxM);
    if (max_iter < 1) return set_err(ctx, HPHI_E_INVAL, "max_iter >= 1");
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    const int64_t D = ham->D;
    if (D < 3 * (int64_t)m) return set_err(ctx, HPHI_E_INVAL, "dimension below 3 m");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t blk = (size_t)D * m;
    double *mem = nullptr;
    // H Phi, R, H R, P, H P and the four updated blocks (Phi is the caller's X)
    if (cudaMalloc(&mem, sizeof(double) * blk * 9) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, HPHI_E_NOMEM, "LOBPCG blocks (%zu bytes)", sizeof(double) * blk * 9);
    }
    double *Phi = (double *)X, *HPhi = mem, *R = mem + blk, *HR = mem + 2 * blk, *P = mem + 3 * blk,
           *HP = mem + 4 * blk, *nPhi = mem + 5 * blk, *nHPhi = mem + 6 * blk, *nP = mem + 7 * blk,
           *nHP = mem + 8 * blk;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->sm_count * 2, (D + kTile - 1) / kTile));
    const int nmax = kMaxBlk * m;
    int st = ensure_partials(ctx, (size_t)G * nmax * nmax + (size_t)ctx->sm_count * 8 * m * 2);
    if (!st) st = ensure_dscal(ctx, 2 * (size_t)nmax * nmax + 64);
    double *Cd = nullptr;
    if (!st && cudaMalloc(&Cd, sizeof(double) * (size_t)nmax * m) != cudaSuccess) {
        cudaGetLastError();
        st = set_err(ctx, HPHI_E_NOMEM, "LOBPCG coefficients");
    }
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(mem);
        cudaFree(Cd);
        return code;
    };
    if (st) return fail(st);
    double *red = ctx->dscal;
    auto hv = [&](const double *x, double *y) -> int {
        HvLaunch L{};
        L.dtype_real = HPHI_F64;
        L.ncol = m;
        L.x = x;
        L.ldx = m;
        L.y = y;
        L.ldy = m;
        L.alpha_s = 1.0;
        L.partials = ctx->partials;
        return launch_hv(ctx, ham, L);
    };
    // host Gram matrix V^T W of sub-block lists
    auto gram = [&](Blocks V, Blocks W, std::vector<double> &out) -> int {
        const int na = V.nb * m, nbw = W.nb * m;
        k_gram<<<G, kGT, 0, ctx->stream>>>(D, m, V, W, ctx->partials);
        HPHI_CUDA(ctx, cudaGetLastError());
        int s2 = reduce_partials(ctx, ctx->partials, G, na * nbw, red);
        if (s2) return s2;
        out.resize((size_t)na * nbw);
        HPHI_CUDA(ctx, cudaMemcpyAsync(out.data(), red, sizeof(double) * na * nbw, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return HPHI_OK;
    };
    auto combine = [&](Blocks Xb, const std::vector<double> &C, double *Y) -> int {
        HPHI_CUDA(ctx, cudaMemcpyAsync(Cd, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice, ctx->stream));
        const int rows = 256 / m;
        int64_t g = (D + rows - 1) / rows;
        if (g > (int64_t)ctx->sm_count * 16) g = (int64_t)ctx->sm_count * 16;
        k_combine<<<(int)g, 256, 0, ctx->stream>>>(D, m, Xb, Cd, Y);
        HPHI_CUDA(ctx, cudaGetLastError());
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // C staged from host memory
        return HPHI_OK;
    };
    // Rayleigh-Ritz on sub-blocks V (with images HV): the m lowest Ritz pairs as
    // coefficients c [nv][m] and values theta
    auto rayleigh_ritz = [&](Blocks Vb, Blocks HVb, std::vector<double> &c, std::vector<double> &theta) -> int {
        const int nv = Vb.nb * m;
        std::vector<double> Gm, Am;
        int s2 = gram(Vb, Vb, Gm);
        if (!s2) s2 = gram(Vb, HVb, Am);
        if (s2) return s2;
        for (int i = 0; i < nv; i++)
            for (int j = i + 1; j < nv; j++) {
                const double g = 0.5 * (Gm[(size_t)i * nv + j] + Gm[(size_t)j * nv + i]);
                const double a = 0.5 * (Am[(size_t)i * nv + j] + Am[(size_t)j * nv + i]);
                Gm[(size_t)i * nv + j] = Gm[(size_t)j * nv + i] = g;
                Am[(size_t)i * nv + j] = Am[(size_t)j * nv + i] = a;
            }
        std::vector<double> gw, U, Gc = Gm;
        jacobi_eig(nv, Gc, gw, U);
        const double gmax = gw[nv - 1];
        if (!(gmax > 0.0) || !isfinite(gmax)) return HPHI_E_NUMERIC;
        std::vector<int> keep;
        for (int i = 0; i < nv; i++)
            if (gw[i] > 1e-12 * gmax) keep.push_back(i);
        const int k = (int)keep.size();
        if (k < m) return HPHI_E_NUMERIC;
        std::vector<double> B((size_t)nv * k);  // B = U_k Lambda_k^{-1/2}
        for (int r = 0; r < nv; r++)
            for (int c2 = 0; c2 < k; c2++) B[(size_t)r * k + c2] = U[(size_t)r * nv + keep[c2]] / sqrt(gw[keep[c2]]);
        std::vector<double> T((size_t)nv * k, 0.0), Cm((size_t)k * k, 0.0);  // T = A B, C = B^T A B
        for (int r = 0; r < nv; r++)
            for (int q = 0; q < nv; q++) {
                const double a = Am[(size_t)r * nv + q];
                if (a == 0.0) continue;
                for (int c2 = 0; c2 < k; c2++) T[(size_t)r * k + c2] += a * B[(size_t)q * k + c2];
            }
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) {
                double s = 0.0;
                for (int r = 0; r < nv; r++) s += B[(size_t)r * k + i] * T[(size_t)r * k + j];
                Cm[(size_t)i * k + j] = s;
            }
        for (int i = 0; i < k; i++)
            for (int j = i + 1; j < k; j++) Cm[(size_t)i * k + j] = Cm[(size_t)j * k + i] = 0.5 * (Cm[(size_t)i * k + j] + Cm[(size_t)j * k + i]);
        std::vector<double> cw, W;
        jacobi_eig(k, Cm, cw, W);
        theta.assign(cw.begin(), cw.begin() + m);
        c.assign((size_t)nv * m, 0.0);  // c = B W[:, :m]
        for (int r = 0; r < nv; r++)
            for (int j = 0; j < m; j++) {
                double s = 0.0;
                for (int i = 0; i < k; i++) s += B[(size_t)r * k + i] * W[(size_t)i * k + j];
                c[(size_t)r * m + j] = s;
            }
        return HPHI_OK;
    };
    // normalise the columns of a block (and of its image with the same factors)
    auto col_norms = [&](const double *Z, std::vector<double> &nrm) -> int {
        nrm.resize(m);
        int s2 = hphi_nrm2(ctx, HPHI_F64, D, m, Z, m, nrm.data());
        return s2;
    };
    auto scale_cols = [&](double *Z, const std::vector<double> &f) -> int {
        return hphi_scal(ctx, HPHI_F64, D, m, f.data(), Z, m);
    };
    // start: Rayleigh-Ritz on the start block alone
    std::vector<double> E(m), c, th, nr;
    if ((st = hv(Phi, HPhi))) return fail(st);
    {
        Blocks Vb{{Phi, nullptr, nullptr}, 1}, Hb{{HPhi, nullptr, nullptr}, 1};
        if ((st = rayleigh_ritz(Vb, Hb, c, th))) return fail(set_err(ctx, st, "LOBPCG: start block is degenerate"));
        if ((st = combine(Vb, c, nPhi)) || (st = combine(Hb, c, nHPhi))) return fail(st);
        HPHI_CUDA(ctx, cudaMemcpyAsync(Phi, nPhi, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(HPhi, nHPhi, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        E = th;
    }
    bool have_p = false, conv = false;
    int it = 0;
    std::vector<double> rn(m, 0.0);
    for (it = 0; it < max_iter; it++) {
        // R = H Phi - Phi diag(E), with its column norms
        {
            LinComb Lc{};
            std::vector<double> a(m), g(m, 1.0), zero(m, 0.0);
            for (int j = 0; j < m; j++) a[j] = -E[j];
            Lc.real_dtype = HPHI_F64;
            Lc.n = D;
            Lc.nr = m;
            Lc.x = Phi;
            Lc.ldx = m;
            Lc.y = HPhi;
            Lc.ldy = m;
            Lc.out = R;
            Lc.ldo = m;
            Lc.a_h = a.data();
            Lc.b_h = zero.data();
            Lc.g_h = g.data();
            if ((st = launch_lincomb(ctx, Lc))) return fail(st);
        }
        if ((st = col_norms(R, rn))) return fail(st);
        bool all = true;
        for (int j = 0; j < m; j++) all = all && rn[j] <= tol * (fabs(E[j]) > 1.0 ? fabs(E[j]) : 1.0);
        if (all) {
            conv = true;
            break;
        }
        // normalised residual directions (a converged column becomes zero)
        std::vector<double> f(m);
        for (int j = 0; j < m; j++) f[j] = rn[j] > 1e-300 ? 1.0 / rn[j] : 0.0;
        if ((st = scale_cols(R, f)) || (st = hv(R, HR))) return fail(st);
        Blocks Vb{{R, Phi, P}, have_p ? 3 : 2}, Hb{{HR, HPhi, HP}, have_p ? 3 : 2};
        if ((st = rayleigh_ritz(Vb, Hb, c, th))) return fail(set_err(ctx, st, "LOBPCG: Rayleigh-Ritz failed"));
        const int nv = Vb.nb * m;
        if ((st = combine(Vb, c, nPhi)) || (st = combine(Hb, c, nHPhi))) return fail(st);
        // P = [R, 0, P] c (the Phi rows of c dropped)
        std::vector<double> cp = c;
        for (int r = m; r < 2 * m; r++)
            for (int j = 0; j < m; j++) cp[(size_t)r * m + j] = 0.0;
        if ((st = combine(Vb, cp, nP)) || (st = combine(Hb, cp, nHP))) return fail(st);
        (void)nv;
        HPHI_CUDA(ctx, cudaMemcpyAsync(Phi, nPhi, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(HPhi, nHPhi, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(P, nP, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(HP, nHP, sizeof(double) * blk, cudaMemcpyDeviceToDevice, ctx->stream));
        // normalise P (and H P with the same factors) for the next Gram matrices
        std::vector<double> pn;
        if ((st = col_norms(P, pn))) return fail(st);
        for (int j = 0; j < m; j++) f[j] = pn[j] > 1e-300 ? 1.0 / pn[j] : 0.0;
        if ((st = scale_cols(P, f)) || (st = scale_cols(HP, f))) return fail(st);
        have_p = true;
        E = th;
    }
    for (int j = 0; j < m; j++) {
        evals[j] = E[j];
        resid[j] = rn[j];
    }
    *iters = it;
    fail(HPHI_OK);
    if (!conv) return set_err(ctx, HPHI_E_NOTCONV, "LOBPCG: tolerance not reached in %d iterations", max_iter);
    return HPHI_OK;
}
