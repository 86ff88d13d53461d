// Basis enumeration and two-table (Lin) ranking on the device.
//
// For a species of N sites with n set bits, the string s splits into a low
// half l (N_lo = N - floor(N/2) bits) and a high half h (floor(N/2) bits):
//   ja[l]  = rank of l among the N_lo-bit strings of the same popcount, in
//            ascending order (computed with the combinatorial number system
//            sum_k C(p_k, k) over the set-bit positions p_1 < p_2 < ...);
//   jb[h]  = number of sector states whose high half is below h (exclusive
//            prefix sum of C(N_lo, n - popcount(h))), or ~0 when no state of
//            the sector has high half h;
//   rank(s) = ja[l] + jb[h]  (H. Q. Lin, Phys. Rev. B 42, 6561 (1990)).
// The paper leaves the encoding to its version-1 predecessor; the sector
// itself is the S^z / particle-number sector of Sec. 3.5.1 and Table 1.
#include <stdio.h>

#include "hphi_internal.cuh"

namespace hphi {

namespace {

__constant__ uint64_t c_binom[41][41];
bool g_binom_ready[64] = {false};

uint64_t host_binom(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

int ensure_binom(hphi_ctx *ctx) {
    if (g_binom_ready[ctx->device]) return HPHI_OK;
    uint64_t t[41][41];
    for (int a = 0; a <= 40; a++)
        for (int b = 0; b <= 40; b++) t[a][b] = host_binom(a, b);
    HPHI_CUDA(ctx, cudaMemcpyToSymbol(c_binom, t, sizeof(t)));
    g_binom_ready[ctx->device] = true;
    return HPHI_OK;
}

__global__ void k_ja(uint32_t *ja, int nlo) {
    uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= (1u << nlo)) return;
    uint64_t r = 0;
    int k = 0;
    for (int p = 0; p < nlo; p++) {
        if ((l >> p) & 1u) {
            k++;
            r += c_binom[p][k];
        }
    }
    ja[l] = (uint32_t)r;
}

__global__ void k_lstate(const uint32_t *ja, const uint32_t *loff, uint32_t *lstate, int nlo) {
    uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= (1u << nlo)) return;
    lstate[loff[__popc(l)] + ja[l]] = l;
}

// One block: exclusive prefix over h of the number of sector states with high
// half h.  Thread t scans a contiguous chunk; chunk totals are scanned in
// order by thread 0.
__global__ void k_jb(uint64_t *jb, uint64_t *jbp, int nlo, int nhi, int n) {
    __shared__ uint64_t tot[1024];
    const uint64_t H = 1ull << nhi;
    const uint64_t chunk = (H + blockDim.x - 1) / blockDim.x;
    const uint64_t h0 = threadIdx.x * chunk;
    uint64_t s = 0;
    for (uint64_t h = h0; h < h0 + chunk && h < H; h++) {
        int need = n - __popcll(h);
        if (need >= 0 && need <= nlo) s += c_binom[nlo][need];
    }
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            uint64_t v = tot[t];
            tot[t] = run;
            run += v;
        }
        jbp[H] = run;
    }
    __syncthreads();
    uint64_t run = tot[threadIdx.x];
    for (uint64_t h = h0; h < h0 + chunk && h < H; h++) {
        int need = n - __popcll(h);
        bool valid = need >= 0 && need <= nlo;
        jbp[h] = run;
        jb[h] = valid ? run : ~0ull;
        if (valid) run += c_binom[nlo][need];
    }
}

__global__ void k_states(const uint64_t *jb, const uint32_t *loff, const uint32_t *lstate, uint32_t *states,
                         int nlo, int nhi, int n) {
    const uint64_t H = 1ull << nhi;
    for (uint64_t h = blockIdx.x; h < H; h += gridDim.x) {
        uint64_t base = jb[h];
        if (base == ~0ull) continue;
        int p = n - __popcll(h);
        uint32_t c0 = loff[p], len = loff[p + 1] - loff[p];
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x)
            states[base + q] = (uint32_t)((h << nlo) | lstate[c0 + q]);
    }
}

// rank of (su, sd) rows; -1 outside the sector
struct SpDev {
    const uint32_t *ja;
    const uint64_t *jb;
    int nlo, n, N;
};

__device__ __forceinline__ int64_t sp_rank(const SpDev &s, uint64_t x) {
    if (s.N < 64 && (x >> s.N) != 0) return -1;
    if (__popcll(x) != s.n) return -1;
    uint64_t b = s.jb[x >> s.nlo];
    if (b == ~0ull) return -1;
    return (int64_t)(b + s.ja[x & ((1ull << s.nlo) - 1)]);
}

__global__ void k_rank(int model, SpDev up, SpDev dn, int64_t ddn, int N, const uint64_t *su, const uint64_t *sd,
                       int64_t n, int64_t *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        if (model == HPHI_SPIN_HALF_GC) {
            r = (N < 64 && (su[k] >> N) != 0) ? -1 : (int64_t)su[k];
        } else if (model == HPHI_SPIN_HALF) {
            r = sp_rank(up, su[k]);
        } else {
            int64_t a = sp_rank(up, su[k]), b = sp_rank(dn, sd[k]);
            r = (a < 0 || b < 0) ? -1 : a * ddn + b;
        }
        out[k] = r;
    }
}

// row -> state: binary search of the block by the monotone prefix jbp
__device__ __forceinline__ uint64_t sp_state(const uint64_t *jbp, const uint32_t *loff, const uint32_t *lstate,
                                             int nlo, int nhi, int n, uint64_t r) {
    uint64_t lo = 0, hi = (1ull << nhi);  // find largest h with jbp[h] <= r
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (jbp[mid] <= r) lo = mid;
        else hi = mid;
    }
    uint64_t h = lo;
    int p = n - __popcll(h);
    return (h << nlo) | lstate[loff[p] + (uint32_t)(r - jbp[h])];
}

struct SpState {
    const uint64_t *jbp;
    const uint32_t *loff, *lstate;
    int nlo, nhi, n;
};

__global__ void k_unrank(int model, SpState up, SpState dn, int64_t ddn, int64_t row0, int64_t n, uint64_t *su,
                         uint64_t *sd) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = (uint64_t)(row0 + k);
        if (model == HPHI_SPIN_HALF_GC) {
            su[k] = r;
            if (sd) sd[k] = 0;
        } else if (model == HPHI_SPIN_HALF) {
            su[k] = sp_state(up.jbp, up.loff, up.lstate, up.nlo, up.nhi, up.n, r);
            if (sd) sd[k] = 0;
        } else {
            uint64_t a = r / (uint64_t)ddn, b = r % (uint64_t)ddn;
            su[k] = sp_state(up.jbp, up.loff, up.lstate, up.nlo, up.nhi, up.n, a);
            if (sd) sd[k] = sp_state(dn.jbp, dn.loff, dn.lstate, dn.nlo, dn.nhi, dn.n, b);
        }
    }
}

}  // namespace

void free_species(Species &sp) {
    cudaFree(sp.ja);
    cudaFree(sp.jb);
    cudaFree(sp.jbp);
    cudaFree(sp.loff);
    cudaFree(sp.lstate);
    cudaFree(sp.states);
    sp = Species();
}

int build_species(hphi_ctx *ctx, Species &sp, int N, int n, bool want_states) {
    int st = ensure_binom(ctx);
    if (st) return st;
    sp.N = N;
    sp.n = n;
    sp.nlo = N - N / 2;
    sp.nhi = N / 2;
    sp.dim = (int64_t)host_binom(N, n);
    const uint64_t L = 1ull << sp.nlo, H = 1ull << sp.nhi;
    sp.loff_h.assign(sp.nlo + 2, 0);
    for (int p = 0; p <= sp.nlo; p++) sp.loff_h[p + 1] = sp.loff_h[p] + (uint32_t)host_binom(sp.nlo, p);
    auto alloc = [&](void **p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, HPHI_E_NOMEM, "basis tables: cudaMalloc(%zu) failed", bytes);
        }
        return HPHI_OK;
    };
    if ((st = alloc((void **)&sp.ja, L * 4)) || (st = alloc((void **)&sp.lstate, L * 4)) ||
        (st = alloc((void **)&sp.loff, (sp.nlo + 2) * 4)) || (st = alloc((void **)&sp.jb, H * 8)) ||
        (st = alloc((void **)&sp.jbp, (H + 1) * 8))) {
        free_species(sp);
        return st;
    }
    HPHI_CUDA(ctx, cudaMemcpyAsync(sp.loff, sp.loff_h.data(), (sp.nlo + 2) * 4, cudaMemcpyHostToDevice,
                                   ctx->stream));
    int tb = 256;
    k_ja<<<(unsigned)((L + tb - 1) / tb), tb, 0, ctx->stream>>>(sp.ja, sp.nlo);
    k_lstate<<<(unsigned)((L + tb - 1) / tb), tb, 0, ctx->stream>>>(sp.ja, sp.loff, sp.lstate, sp.nlo);
    k_jb<<<1, 1024, 0, ctx->stream>>>(sp.jb, sp.jbp, sp.nlo, sp.nhi, n);
    HPHI_CUDA(ctx, cudaGetLastError());
    if (want_states) {
        if ((st = alloc((void **)&sp.states, (size_t)sp.dim * 4))) {
            free_species(sp);
            return st;
        }
        unsigned g = (unsigned)(H < 4096 ? H : 4096);
        k_states<<<g, 256, 0, ctx->stream>>>(sp.jb, sp.loff, sp.lstate, sp.states, sp.nlo, sp.nhi, n);
        HPHI_CUDA(ctx, cudaGetLastError());
    }
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HPHI_OK;
}

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_build_basis(hphi_ctx *ctx, int model, int n_sites, int n_up, int n_dn, hphi_basis **out) {
    if (!ctx || !out) return HPHI_E_INVAL;
    *out = nullptr;
    ctx->err.clear();
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    int N = n_sites;
    if (model == HPHI_SPIN_HALF) {
        if (N < 2 || N > 40 || n_up < 0 || n_up > N)
            return set_err(ctx, HPHI_E_INVAL, "SPIN_HALF needs 2 <= n_sites <= 40 and 0 <= n_up <= n_sites");
    } else if (model == HPHI_SPIN_HALF_GC) {
        if (N < 2 || N > 36) return set_err(ctx, HPHI_E_INVAL, "SPIN_HALF_GC needs 2 <= n_sites <= 36");
    } else if (model == HPHI_HUBBARD) {
        if (N < 2 || N > 32 || n_up < 0 || n_up > N || n_dn < 0 || n_dn > N)
            return set_err(ctx, HPHI_E_INVAL, "HUBBARD needs 2 <= n_sites <= 32 and 0 <= n_up, n_dn <= n_sites");
        if (host_binom(N, n_up) >= (1ull << 31) || host_binom(N, n_dn) >= (1ull << 31))
            return set_err(ctx, HPHI_E_INVAL, "HUBBARD species dimension must be below 2^31");
    } else {
        return set_err(ctx, HPHI_E_INVAL, "unknown model %d", model);
    }
    hphi_basis *b = new (std::nothrow) hphi_basis();
    if (!b) return set_err(ctx, HPHI_E_NOMEM, "host allocation failed");
    b->model = model;
    b->N = N;
    b->nup = n_up;
    b->ndn = n_dn;
    b->device = ctx->device;
    int st = HPHI_OK;
    if (model == HPHI_SPIN_HALF) {
        st = build_species(ctx, b->sp[0], N, n_up, false);
        b->D = b->sp[0].dim;
    } else if (model == HPHI_SPIN_HALF_GC) {
        b->D = (int64_t)1 << N;
        b->sp[0].N = N;
        b->sp[0].nlo = N - N / 2;
        b->sp[0].nhi = N / 2;
        b->sp[0].dim = b->D;
    } else {
        st = build_species(ctx, b->sp[0], N, n_up, true);
        if (!st) st = build_species(ctx, b->sp[1], N, n_dn, true);
        b->D = b->sp[0].dim * b->sp[1].dim;
    }
    if (st) {
        free_species(b->sp[0]);
        free_species(b->sp[1]);
        delete b;
        return st;
    }
    *out = b;
    return HPHI_OK;
}

extern "C" void hphi_basis_destroy(hphi_basis *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    free_species(b->sp[0]);
    free_species(b->sp[1]);
    delete b;
}

extern "C" int64_t hphi_basis_dim(const hphi_basis *b) { return b ? b->D : -1; }

extern "C" int hphi_basis_table_sizes(const hphi_basis *b, int species, int64_t *n_ja, int64_t *n_jb) {
    if (!b || !n_ja || !n_jb || species < 0 || species > 1) return HPHI_E_INVAL;
    if (b->model == HPHI_SPIN_HALF_GC || (species == 1 && b->model != HPHI_HUBBARD)) {
        *n_ja = *n_jb = 0;
        return HPHI_OK;
    }
    *n_ja = (int64_t)1 << b->sp[species].nlo;
    *n_jb = (int64_t)1 << b->sp[species].nhi;
    return HPHI_OK;
}

extern "C" int hphi_basis_export(hphi_ctx *ctx, const hphi_basis *b, int species, uint32_t *ja_host,
                                 uint64_t *jb_host) {
    if (!ctx || !b || species < 0 || species > 1) return HPHI_E_INVAL;
    ctx->err.clear();
    const Species &sp = b->sp[species];
    if (!sp.ja) return set_err(ctx, HPHI_E_INVAL, "this basis has no tables for species %d", species);
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    if (ja_host)
        HPHI_CUDA(ctx, cudaMemcpyAsync(ja_host, sp.ja, (1ull << sp.nlo) * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (jb_host)
        HPHI_CUDA(ctx, cudaMemcpyAsync(jb_host, sp.jb, (1ull << sp.nhi) * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HPHI_OK;
}

extern "C" int hphi_basis_rank(hphi_ctx *ctx, const hphi_basis *b, const uint64_t *su, const uint64_t *sd,
                               int64_t n, int64_t *row) {
    if (!ctx || !b || (n > 0 && (!su || !row))) return HPHI_E_INVAL;
    ctx->err.clear();
    if (b->model == HPHI_HUBBARD && n > 0 && !sd) return set_err(ctx, HPHI_E_INVAL, "HUBBARD needs sd");
    if (n <= 0) return HPHI_OK;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    SpDev up{b->sp[0].ja, b->sp[0].jb, b->sp[0].nlo, b->sp[0].n, b->N};
    SpDev dn{b->sp[1].ja, b->sp[1].jb, b->sp[1].nlo, b->sp[1].n, b->N};
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_rank<<<(unsigned)g, 256, 0, ctx->stream>>>(b->model, up, dn, b->sp[1].dim, b->N, su, sd, n, row);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

extern "C" int hphi_basis_states(hphi_ctx *ctx, const hphi_basis *b, int64_t row0, int64_t n, uint64_t *su,
                                 uint64_t *sd) {
    if (!ctx || !b || (n > 0 && !su)) return HPHI_E_INVAL;
    ctx->err.clear();
    if (row0 < 0 || n < 0 || row0 + n > b->D) return set_err(ctx, HPHI_E_INVAL, "row range outside [0, D)");
    if (b->model == HPHI_HUBBARD && n > 0 && !sd) return set_err(ctx, HPHI_E_INVAL, "HUBBARD needs sd");
    if (n == 0) return HPHI_OK;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    SpState up{b->sp[0].jbp, b->sp[0].loff, b->sp[0].lstate, b->sp[0].nlo, b->sp[0].nhi, b->sp[0].n};
    SpState dn{b->sp[1].jbp, b->sp[1].loff, b->sp[1].lstate, b->sp[1].nlo, b->sp[1].nhi, b->sp[1].n};
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_unrank<<<(unsigned)g, 256, 0, ctx->stream>>>(b->model, up, dn, b->sp[1].dim, row0, n, su, sd);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}
