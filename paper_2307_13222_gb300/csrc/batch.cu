// Many small eigenproblems at once: the Lanczos method (Sec. 1) for a batch of
// independent Hamiltonians, one thread block per problem.
//
// A problem small enough for one SM (D up to ~10^5-10^6) gains nothing from
// the grid-wide H*x kernels: their launches, reductions and host round trips
// dominate.  Here one thread block runs the whole recurrence of its problem,
//   u = H w_k / beta_k - (beta_k / beta_{k-1}) w_{k-1},  alpha_k = <w_k, u> / beta_k,
//   w_{k+1} = u - (alpha_k / beta_k) w_k,  beta_{k+1}^2 = |w_{k+1}|^2,
// with block-level reductions in a fixed order, for a chunk of steps per
// launch.  Rows are evaluated directly from the plain term list: the row's
// basis state, every bond / hop / U / V term, the target state's Lin rank
// (ja[low] + jb[high], per species for Hubbard) and the gathered x value.
// Between chunks the host evaluates the stopping rule of hphi_lanczos at every
// step of the chunk (so the stop step is the one a check after every step
// would give), retires finished problems and may add new ones: the same chunk
// launch is the continuous-batching step of a serving loop.  A second kernel
// regenerates the Krylov vectors (same arithmetic, so bit-identical) and
// accumulates the ground-state vector.  FP64 throughout.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "batch.cuh"

namespace hphi {

namespace {

constexpr int kBT = kBatchThreads;
constexpr int kMaxBTerms = kBatchMaxTerms;
constexpr size_t kSmemBudget = kBatchSmemBudget;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum over the thread block in a fixed order; every thread gets the total.
__device__ double block_sum(double v, double *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sm[32] = t;
    }
    __syncthreads();
    const double t = sm[32];
    __syncthreads();
    return t;
}

__device__ __forceinline__ int64_t lin_rank(const uint32_t *ja, const uint64_t *jb, int nlo, uint64_t s) {
    return (int64_t)((uint64_t)ja[s & ((1ull << nlo) - 1ull)] + jb[s >> nlo]);
}

// Off-diagonal term in the form the row loop uses.
struct OffTerm {
    uint64_t mask;     // the two flipped bits
    uint64_t between;  // hops: bits strictly between the two sites
    int s;             // 0: spin bond / up hop, 1: down hop
    double c;          // element: Jxy / 2 (spin), -t (hop, times the fermion sign)
};

// Rank tables and state lists as the row loop sees them (shared or global).
struct RowTables {
    const uint32_t *ja_u, *ja_d, *st_u, *st_d;
    const uint64_t *jb_u, *jb_d;
};

// H_rr from the plain term list (computed once per problem).
__device__ double diag_of(const BProb &P, const DTerm *T, int64_t r) {
    double d = 0.0;
    if (P.model != kHubbard) {
        const uint64_t s = P.model == kSpin ? (uint64_t)P.rowstate[r] : (uint64_t)r;
        for (int k = 0; k < P.nterms; k++) {
            const uint64_t bi = (s >> T[k].i) & 1ull, bj = (s >> T[k].j) & 1ull;
            d += (bi == bj ? 0.25 : -0.25) * T[k].a;
        }
    } else {
        const int64_t iu = r / P.ddn, id = r - iu * P.ddn;
        const uint64_t su = P.st_u[iu], sd = P.st_d[id];
        for (int k = 0; k < P.nterms; k++) {
            const DTerm &t = T[k];
            if (t.kind == DT_U) {
                d += t.a * (double)(((su & sd) >> t.i) & 1ull);
            } else if (t.kind == DT_V) {
                const double ni = (double)(((su >> t.i) & 1ull) + ((sd >> t.i) & 1ull));
                const double nj = (double)(((su >> t.j) & 1ull) + ((sd >> t.j) & 1ull));
                d += t.a * ni * nj;
            }
        }
    }
    return d;
}

// (H x)[r] = H_rr x_r + sum over the off-diagonal terms that connect r.
__device__ __forceinline__ double h_row(const BProb &P, const RowTables &R, const OffTerm *O, int no, int64_t r,
                                        const double *x) {
    double acc = P.diag[r] * x[r];
    if (P.model != kHubbard) {
        const uint64_t s = P.model == kSpin ? (uint64_t)P.rowstate[r] : (uint64_t)r;
        for (int k = 0; k < no; k++) {
            const uint64_t m = O[k].mask, sm = s & m;
            if (sm != 0 && sm != m) {
                const uint64_t s2 = s ^ m;
                const int64_t r2 = P.model == kSpin ? lin_rank(R.ja_u, R.jb_u, P.nlo_u, s2) : (int64_t)s2;
                acc = fma(O[k].c, x[r2], acc);
            }
        }
    } else {
        const int64_t iu = r / P.ddn, id = r - iu * P.ddn;
        const uint64_t su = R.st_u[iu], sd = R.st_d[id];
        for (int k = 0; k < no; k++) {
            const OffTerm &t = O[k];
            const uint64_t s = t.s ? sd : su, sm = s & t.mask;
            if (sm != 0 && sm != t.mask) {
                const uint64_t s2 = s ^ t.mask;
                const double c = (__popcll((unsigned long long)(s & t.between)) & 1) ? -t.c : t.c;
                const int64_t r2 = t.s ? iu * P.ddn + lin_rank(R.ja_d, R.jb_d, P.nlo_d, s2)
                                       : lin_rank(R.ja_u, R.jb_u, P.nlo_u, s2) * P.ddn + id;
                acc = fma(c, x[r2], acc);
            }
        }
    }
    return acc;
}

// Per-block set-up shared by both kernels: off-diagonal terms and the tables
// in shared memory where they fit.  Returns the number of off-diagonal terms.
__device__ int setup_rows(const BProb &P, const DTerm *T, OffTerm *O, unsigned char *dyn, double **xs,
                          RowTables *R) {
    __shared__ int no_sh;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < P.nterms; k++) {
            const DTerm &t = T[k];
            const bool off = (t.kind == DT_SPIN && t.b != 0.0) || (t.kind == DT_HOP && t.a != 0.0);
            if (!off) continue;
            const int lo = t.i < t.j ? t.i : t.j, hi = t.i < t.j ? t.j : t.i;
            O[n].mask = (1ull << t.i) | (1ull << t.j);
            O[n].between = ((1ull << hi) - 1ull) & ~((2ull << lo) - 1ull);
            O[n].s = t.kind == DT_HOP ? t.s : 0;
            O[n].c = t.kind == DT_SPIN ? 0.5 * t.b : -t.a;
            n++;
        }
        no_sh = n;
    }
    // shared layout: x [D] (if staged), then the tables
    size_t off = 0;
    *xs = nullptr;
    if (P.stage_x) {
        *xs = (double *)dyn;
        off = ((size_t)P.D * 8 + 15) & ~(size_t)15;
    }
    R->ja_u = P.ja_u;
    R->jb_u = P.jb_u;
    R->ja_d = P.ja_d;
    R->jb_d = P.jb_d;
    R->st_u = P.st_u;
    R->st_d = P.st_d;
    if (P.stage_tab && P.model != kSpinGC) {
        const int nsp = P.model == kHubbard ? 2 : 1;
        for (int sp = 0; sp < nsp; sp++) {
            const int nlo = sp ? P.nlo_d : P.nlo_u;
            const int nhi = P.nbits[sp] - nlo;
            const uint32_t *ja = sp ? P.ja_d : P.ja_u;
            const uint64_t *jb = sp ? P.jb_d : P.jb_u;
            uint64_t *jbs = (uint64_t *)(dyn + off);
            off += ((size_t)8 << nhi);
            uint32_t *jas = (uint32_t *)(dyn + off);
            off += (((size_t)4 << nlo) + 15) & ~(size_t)15;
            for (int64_t i = threadIdx.x; i < ((int64_t)1 << nhi); i += blockDim.x) jbs[i] = jb[i];
            for (int64_t i = threadIdx.x; i < ((int64_t)1 << nlo); i += blockDim.x) jas[i] = ja[i];
            if (sp) {
                R->ja_d = jas;
                R->jb_d = jbs;
            } else {
                R->ja_u = jas;
                R->jb_u = jbs;
            }
        }
        if (P.model == kHubbard) {
            uint32_t *su = (uint32_t *)(dyn + off);
            off += (((size_t)4 * (P.D / P.ddn)) + 15) & ~(size_t)15;
            uint32_t *sd = (uint32_t *)(dyn + off);
            for (int64_t i = threadIdx.x; i < P.D / P.ddn; i += blockDim.x) su[i] = P.st_u[i];
            for (int64_t i = threadIdx.x; i < P.ddn; i += blockDim.x) sd[i] = P.st_d[i];
            R->st_u = su;
            R->st_d = sd;
        }
    }
    __syncthreads();
    return no_sh;
}

// One Lanczos step of the block's problem; the vectors rotate through three
// buffers: w_k = buf[k % 3], w_{k-1} = buf[(k + 2) % 3], u and w_{k+1} =
// buf[(k + 1) % 3].  With use_given, alpha_k is the stored value (the
// ground-state pass) and no reductions are taken.
__device__ void lz_step(const BProb &P, const RowTables &R, const OffTerm *O, int no, double *xs, int k,
                        double ak_given, bool use_given, double *sm, double *a_out, double *b2_out) {
    const int64_t D = P.D;
    const double *wc = P.w + (int64_t)(k % 3) * D;
    const double *wp = P.w + (int64_t)((k + 2) % 3) * D;
    double *wu = P.w + (int64_t)((k + 1) % 3) * D;
    const double *x = wc;
    if (xs) {
        for (int64_t r = threadIdx.x; r < D; r += blockDim.x) xs[r] = wc[r];
        __syncthreads();
        x = xs;
    }
    const double bk = sqrt(P.beta2[(int64_t)k * P.stride]);
    const double ibk = 1.0 / bk;
    const double ck = k > 0 ? bk / sqrt(P.beta2[(int64_t)(k - 1) * P.stride]) : 0.0;
    double dot = 0.0;
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
        double u = h_row(P, R, O, no, r, x) * ibk;
        if (k > 0) u = fma(-ck, wp[r], u);
        wu[r] = u;
        dot = fma(x[r], u, dot);
    }
    const double a = use_given ? ak_given : block_sum(dot, sm) * ibk;
    const double f = a * ibk;
    double nn = 0.0;
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
        const double v = fma(-f, x[r], wu[r]);
        wu[r] = v;
        nn = fma(v, v, nn);
    }
    *a_out = a;
    *b2_out = use_given ? 0.0 : block_sum(nn, sm);
    if (use_given) __syncthreads();  // w_{k+1} complete (and xs free) before the next step
}

__global__ void __launch_bounds__(kBT) k_lzb(const BProb *probs) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ DTerm T[kMaxBTerms];
    __shared__ OffTerm O[kMaxBTerms];
    __shared__ double sm[33];
    __shared__ int stop;
    const BProb P = probs[blockIdx.x];
    if (P.nsteps <= 0) return;
    for (int i = threadIdx.x; i < P.nterms; i += blockDim.x) T[i] = P.terms[i];
    if (threadIdx.x == 0) stop = P.state[0] != 0;
    __syncthreads();
    const int64_t D = P.D;
    if (!stop) {
        double *xs;
        RowTables R;
        const int no = setup_rows(P, T, O, dyn, &xs, &R);
        for (int s = 0; s < P.nsteps; s++) {
            const int k = P.k0 + s;
            if (k == 0) {
                double nn = 0.0;
                for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
                    const double v = P.v0[r * P.v0_stride];
                    P.w[r] = v;
                    P.diag[r] = diag_of(P, T, r);
                    nn = fma(v, v, nn);
                }
                const double b2 = block_sum(nn, sm);
                if (threadIdx.x == 0) {
                    P.beta2[0] = b2;  // k = 0: row 0 of the step-major array
                    P.scal[0] = 0.0;
                    if (!(b2 > 0.0) || !isfinite(b2)) {
                        P.state[0] = 3;
                        P.state[1] = 0;
                        stop = 1;
                    }
                }
                __syncthreads();
                if (stop) break;
            }
            double a, b2;
            lz_step(P, R, O, no, xs, k, 0.0, false, sm, &a, &b2);
            if (threadIdx.x == 0) {
                P.alpha[(int64_t)k * P.stride] = a;
                P.beta2[(int64_t)(k + 1) * P.stride] = b2;
                if (P.stage) {
                    P.stage[1 + 2 * s] = a;
                    P.stage[2 + 2 * s] = b2;
                }
                P.state[1] = k + 1;
                const double bk = sqrt(P.beta2[(int64_t)k * P.stride]), bn = sqrt(b2 > 0.0 ? b2 : 0.0);
                const double r = fabs(a) + (k > 0 ? bk : 0.0) + bn;
                const double tn = r > P.scal[0] ? r : P.scal[0];
                P.scal[0] = tn;
                if (!isfinite(a) || !isfinite(b2)) {
                    P.state[0] = 2;
                    stop = 1;
                } else if (bn <= 64.0 * DBL_EPSILON * tn) {
                    P.state[0] = 1;
                    stop = 1;
                }
            }
            __syncthreads();
            if (stop) break;
        }
    }
    if (P.stage && threadIdx.x == 0) {
        P.stage[0] = P.beta2[(int64_t)P.k0 * P.stride];
        P.stage[1 + 2 * P.nsteps] = (double)P.state[0];
        P.stage[2 + 2 * P.nsteps] = (double)P.state[1];
    }
}

// Ground-state pass: regenerate w_k with the stored alpha / beta and
// accumulate gs = sum_k (y_k / beta_k) w_k; normalise; |H gs - theta gs|.
__global__ void __launch_bounds__(kBT) k_gsb(const BProb *probs) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ DTerm T[kMaxBTerms];
    __shared__ OffTerm O[kMaxBTerms];
    __shared__ double sm[33];
    const BProb P = probs[blockIdx.x];
    if (P.m <= 0 || !P.gs) return;
    for (int i = threadIdx.x; i < P.nterms; i += blockDim.x) T[i] = P.terms[i];
    __syncthreads();
    double *xs;
    RowTables R;
    const int no = setup_rows(P, T, O, dyn, &xs, &R);
    const int64_t D = P.D;
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
        P.w[r] = P.v0[r * P.v0_stride];
        P.gs[r] = 0.0;
    }
    __syncthreads();
    for (int k = 0; k < P.m; k++) {
        const double *wc = P.w + (int64_t)(k % 3) * D;
        const double c = P.y[k] / sqrt(P.beta2[(int64_t)k * P.stride]);
        for (int64_t r = threadIdx.x; r < D; r += blockDim.x) P.gs[r] = fma(c, wc[r], P.gs[r]);
        if (k + 1 == P.m) break;
        double a, b2;
        lz_step(P, R, O, no, xs, k, P.alpha[(int64_t)k * P.stride], true, sm, &a, &b2);
    }
    double nn = 0.0;
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) nn = fma(P.gs[r], P.gs[r], nn);
    const double inv = 1.0 / sqrt(block_sum(nn, sm));
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) P.gs[r] *= inv;
    __syncthreads();
    const double *g = P.gs;
    if (xs) {
        for (int64_t r = threadIdx.x; r < D; r += blockDim.x) xs[r] = P.gs[r];
        __syncthreads();
        g = xs;
    }
    double rr = 0.0;
    for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
        const double v = h_row(P, R, O, no, r, g) - P.theta * g[r];
        rr = fma(v, v, rr);
    }
    rr = block_sum(rr, sm);
    if (threadIdx.x == 0) P.resid[0] = sqrt(rr);
}

// Row -> state of an S^z sector.
__global__ void k_rowstate(const uint64_t *jb, const uint32_t *loff, const uint32_t *lstate, int nlo, int n,
                           int64_t nh, uint32_t *out) {
    for (int64_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const uint64_t base = jb[h];
        if (base == ~0ull) continue;
        const int c = n - __popcll((unsigned long long)h);
        const uint32_t c0 = loff[c], len = loff[c + 1] - c0;
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x)
            out[base + q] = (uint32_t)(((uint64_t)h << nlo) | lstate[c0 + q]);
    }
}

}  // namespace

int ensure_rowstate(hphi_ctx *ctx, hphi_ham *ham) {
    if (ham->model != HPHI_SPIN_HALF || ham->rowstate) return HPHI_OK;
    const Species &sp = ham->basis->sp[0];
    if (sp.N > 32) return set_err(ctx, HPHI_E_INVAL, "small-problem solver: at most 32 sites");
    cudaError_t e = cudaMalloc(&ham->rowstate, sizeof(uint32_t) * (size_t)ham->D);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ham->rowstate = nullptr;
        return set_err(ctx, HPHI_E_NOMEM, "row states (%lld rows)", (long long)ham->D);
    }
    const int64_t nh = (int64_t)1 << sp.nhi;
    const int grid = (int)(nh < 4096 ? nh : 4096);
    k_rowstate<<<grid, 256, 0, ctx->stream>>>(sp.jb, sp.loff, sp.lstate, sp.nlo, sp.n, nh, ham->rowstate);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}


size_t batch_fill(const hphi_ham *h, BProb &P) {
    const hphi_basis *b = h->basis;
    P.model = h->model;
    P.nterms = (int)h->dterms.size();
    P.D = h->D;
    P.nlo_u = b->sp[0].nlo;
    P.nbits[0] = P.nbits[1] = b->N;
    P.ja_u = b->sp[0].ja;
    P.jb_u = b->sp[0].jb;
    if (h->model == HPHI_HUBBARD) {
        P.nlo_d = b->sp[1].nlo;
        P.ja_d = b->sp[1].ja;
        P.jb_d = b->sp[1].jb;
        P.st_u = b->sp[0].states;
        P.st_d = b->sp[1].states;
        P.ddn = b->sp[1].dim;
    }
    P.rowstate = h->rowstate;
    P.terms = h->dterms_d;
    P.v0_stride = 1;
    // shared memory: x of the step if it fits, then the rank tables / state lists
    const size_t xb = ((size_t)h->D * 8 + 15) & ~(size_t)15;
    size_t tb = 0;
    if (h->model != HPHI_SPIN_HALF_GC) {
        const int nsp = h->model == HPHI_HUBBARD ? 2 : 1;
        for (int sp = 0; sp < nsp; sp++)
            tb += ((size_t)8 << (b->N - b->sp[sp].nlo)) + ((((size_t)4 << b->sp[sp].nlo) + 15) & ~(size_t)15);
        if (h->model == HPHI_HUBBARD) tb += ((4 * (size_t)b->sp[0].dim + 15) & ~(size_t)15) + 4 * (size_t)b->sp[1].dim;
    }
    P.stage_x = xb <= kSmemBudget;
    P.stage_tab = (P.stage_x ? xb : 0) + tb <= kSmemBudget;
    return (P.stage_x ? xb : 0) + (P.stage_tab ? tb : 0);
}

int batch_launch_steps(hphi_ctx *ctx, const BProb *dprob, int n, size_t dyn) {
    // the dynamic shared-memory limits of both kernels, raised once per device under a lock
    if (dyn_occupancy(ctx, (const void *)k_lzb, kBT, dyn) < 1 || dyn_occupancy(ctx, (const void *)k_gsb, kBT, dyn) < 1)
        return set_err(ctx, HPHI_E_INVAL, "batched Lanczos: %zu bytes of shared memory per problem do not fit", dyn);
    if (n <= 0) return HPHI_OK;
    const int slot = prof_begin(ctx, PROF_HV);
    k_lzb<<<n, kBT, dyn, ctx->stream>>>(dprob);
    prof_end(ctx, slot);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

int batch_launch_gs(hphi_ctx *ctx, const BProb *dprob, int n, size_t dyn) {
    if (n <= 0) return HPHI_OK;
    const int st = batch_launch_steps(ctx, dprob, 0, dyn);  // sets the shared-memory attribute once
    if (st) return st;
    k_gsb<<<n, kBT, dyn, ctx->stream>>>(dprob);
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_lanczos_batch(hphi_ctx *ctx, int nprob, hphi_ham *const *hams, const void *const *v0,
                                  void *const *gs_out, const hphi_lanczos_opts *opts, hphi_lanczos_result *results,
                                  int *status) {
    if (!ctx || nprob < 0 || (nprob > 0 && (!hams || !v0 || !results || !status)) || !opts) return HPHI_E_INVAL;
    ctx->err.clear();
    if (nprob == 0) return HPHI_OK;
    if (opts->dtype != HPHI_F64) return set_err(ctx, HPHI_E_INVAL, "batched Lanczos: FP64 vectors only");
    if (opts->reorth) return set_err(ctx, HPHI_E_INVAL, "batched Lanczos: no reorthogonalisation");
    const int M = opts->max_steps;
    if (M < 1 || M > 100000) return set_err(ctx, HPHI_E_INVAL, "max_steps must be in [1, 100000]");
    if (nprob > 65535) return set_err(ctx, HPHI_E_INVAL, "at most 65535 problems per call");
    const int chunk = opts->check_every < 1 ? 1 : opts->check_every;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    size_t nvec = 0;
    for (int p = 0; p < nprob; p++) {
        hphi_ham *h = hams[p];
        if (!h || !v0[p]) return set_err(ctx, HPHI_E_INVAL, "problem %d: null Hamiltonian or start vector", p);
        if (h->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "problem %d: another device", p);
        if ((int)h->dterms.size() > kMaxBTerms)
            return set_err(ctx, HPHI_E_INVAL, "problem %d: more than %d terms", p, kMaxBTerms);
        if (h->D > ((int64_t)1 << 31)) return set_err(ctx, HPHI_E_INVAL, "problem %d: dimension above 2^31", p);
        int st = ensure_rowstate(ctx, h);
        if (st) return st;
        nvec += 4 * (size_t)h->D;
    }
    // workspace: vectors, then alpha [M][nprob], beta^2 [M+1][nprob], per problem
    // (running max, residual, Ritz vector [M])
    const size_t n_ab = (size_t)M * nprob + (size_t)(M + 1) * nprob, n_pp = (size_t)nprob * (M + 2);
    double *ws = nullptr;
    int *iws = nullptr;
    BProb *dprob = nullptr;
    if (cudaMalloc(&ws, (nvec + n_ab + n_pp) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&iws, 2 * (size_t)nprob * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&dprob, (size_t)nprob * sizeof(BProb)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ws);
        cudaFree(iws);
        return set_err(ctx, HPHI_E_NOMEM, "batched Lanczos workspace");
    }
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ws);
        cudaFree(iws);
        cudaFree(dprob);
        return code;
    };
    double *alpha_all = ws + nvec, *beta2_all = alpha_all + (size_t)M * nprob, *pp = beta2_all + (size_t)(M + 1) * nprob;
    std::vector<BProb> hp(nprob);
    size_t off = 0, dyn_bytes = 0;
    for (int p = 0; p < nprob; p++) {
        hphi_ham *h = hams[p];
        BProb &P = hp[p];
        P = BProb{};
        const size_t need = batch_fill(h, P);
        dyn_bytes = need > dyn_bytes ? need : dyn_bytes;
        P.v0 = (const double *)v0[p];
        P.w = ws + off;
        off += 3 * (size_t)h->D;
        P.diag = ws + off;
        off += (size_t)h->D;
        P.alpha = alpha_all + p;
        P.beta2 = beta2_all + p;
        P.stride = nprob;
        P.scal = pp + (size_t)p * (M + 2);
        P.resid = P.scal + 1;
        P.y = P.scal + 2;
        P.state = iws + 2 * p;
    }
    HPHI_CUDA(ctx, cudaMemsetAsync(iws, 0, 2 * (size_t)nprob * sizeof(int), ctx->stream));
    // host mirrors of alpha / beta^2 (step-major) and the stopping state
    std::vector<double> ah((size_t)M * nprob, 0.0), b2h((size_t)(M + 1) * nprob, 0.0);
    std::vector<int> done(nprob, 0), mstop(nprob, 0), conv(nprob, 0), brk(nprob, 0), st(nprob, HPHI_OK);
    std::vector<double> theta(nprob, 0.0), rest(nprob, -1.0);
    std::vector<double> warm(nprob, std::nan(""));
    std::vector<int> ist(2 * (size_t)nprob);
    // the stopping rule of hphi_lanczos at step j (j >= 2) for problem p
    auto holds = [&](int p, int j, std::vector<double> &ap, std::vector<double> &bp, double *t, double *r) -> int {
        ap.resize(j);
        bp.resize(j + 1);
        for (int q = 0; q < j; q++) ap[q] = ah[(size_t)q * nprob + p];
        for (int q = 0; q <= j; q++) bp[q] = b2h[(size_t)q * nprob + p];
        double yl = 0.0;
        if (lowest_ritz_warm(j, ap.data(), bp.data(), &warm[p], t, &yl)) return -1;
        *r = sqrt(bp[j]) * yl;
        return (opts->tol > 0.0 && j >= 2 && *r <= opts->tol * (fabs(*t) > 1.0 ? fabs(*t) : 1.0)) ? 1 : 0;
    };
    // per problem, after a chunk that ended at step k (k_prev before it)
    auto check = [&](int p, int k_prev, std::vector<double> &ap, std::vector<double> &bp) {
        const int flag = ist[2 * p], steps = ist[2 * p + 1];
        int m = 0;
        double th = 0.0, re = -1.0;
        if (flag == 3) {
            st[p] = HPHI_E_INVAL;
        } else if (flag == 2) {
            st[p] = HPHI_E_NUMERIC;
            m = steps;
        } else {
            // first step of this chunk that meets the tolerance
            if (opts->tol > 0.0 && steps >= 2) {
                const int h = holds(p, steps, ap, bp, &th, &re);
                if (h < 0) {
                    st[p] = HPHI_E_NUMERIC;
                } else if (h == 1) {
                    for (int j = std::max(2, k_prev + 1); j <= steps; j++)
                        if (holds(p, j, ap, bp, &th, &re) == 1) {
                            m = j;
                            break;
                        }
                    conv[p] = 1;
                }
            }
            if (!m && !st[p] && flag == 1) {
                m = steps;
                brk[p] = 1;
            }
            if (!m && !st[p] && steps >= M) m = steps;
        }
        if (m || st[p]) {
            if (m && !st[p] && holds(p, m, ap, bp, &th, &re) < 0) st[p] = HPHI_E_NUMERIC;
            mstop[p] = m;
            theta[p] = th;
            rest[p] = re;
            done[p] = 1;
        }
    };
    const int nthreads = nprob >= 64 ? std::max(1, std::min(16, (int)std::thread::hardware_concurrency())) : 1;
    int k = 0, left = nprob;
    while (left > 0 && k < M) {
        const int c = std::min(chunk, M - k);
        for (int p = 0; p < nprob; p++) {
            hp[p].k0 = k;
            hp[p].nsteps = done[p] ? 0 : c;
        }
        HPHI_CUDA(ctx, cudaMemcpyAsync(dprob, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice, ctx->stream));
        int stl = batch_launch_steps(ctx, dprob, nprob, dyn_bytes);
        if (stl) return fail(stl);
        HPHI_CUDA(ctx, cudaMemcpyAsync(ist.data(), iws, sizeof(int) * 2 * nprob, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaMemcpyAsync(ah.data() + (size_t)k * nprob, alpha_all + (size_t)k * nprob,
                                       sizeof(double) * (size_t)c * nprob, cudaMemcpyDeviceToHost, ctx->stream));
        const int b0 = k == 0 ? 0 : k + 1;
        HPHI_CUDA(ctx, cudaMemcpyAsync(b2h.data() + (size_t)b0 * nprob, beta2_all + (size_t)b0 * nprob,
                                       sizeof(double) * (size_t)(k + c + 1 - b0) * nprob, cudaMemcpyDeviceToHost,
                                       ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const int k_prev = k;
        k += c;
        if (nthreads == 1) {
            std::vector<double> ap, bp;
            for (int p = 0; p < nprob; p++)
                if (!done[p]) check(p, k_prev, ap, bp);
        } else {
            std::vector<std::thread> pool;
            for (int t = 0; t < nthreads; t++)
                pool.emplace_back([&, t]() {
                    std::vector<double> ap, bp;
                    for (int p = t; p < nprob; p += nthreads)
                        if (!done[p]) check(p, k_prev, ap, bp);
                });
            for (auto &th : pool) th.join();
        }
        left = 0;
        for (int p = 0; p < nprob; p++) left += !done[p];
    }
    // energies (eigenvalues of T_m) and, where asked for, the Ritz vector of T_m
    // for the ground-state pass; spread over host threads for large batches
    bool any_gs = false;
    std::vector<std::vector<double>> yv(nprob);
    auto finish = [&](int p) {
        hp[p].nsteps = 0;
        hp[p].m = 0;
        hp[p].gs = nullptr;
        const int m = mstop[p];
        if (st[p] || m < 1) return;
        const bool want = gs_out && gs_out[p];
        std::vector<double> a(m), bb(m, 0.0), ev(m), Z(want ? (size_t)m * m : 0);
        for (int j = 0; j < m; j++) a[j] = ah[(size_t)j * nprob + p];
        for (int j = 1; j < m; j++) bb[j] = sqrt(b2h[(size_t)j * nprob + p]);
        int s2 = hphi_tridiag_eigen(m, a.data(), bb.data(), ev.data(), want ? Z.data() : nullptr);
        if (s2) {
            st[p] = s2;
            return;
        }
        theta[p] = ev[0];
        if (!want) return;
        yv[p].resize(m);
        for (int i = 0; i < m; i++) yv[p][i] = Z[(size_t)i * m];
    };
    if (nthreads == 1) {
        for (int p = 0; p < nprob; p++) finish(p);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nthreads; t++)
            pool.emplace_back([&, t]() {
                for (int p = t; p < nprob; p += nthreads) finish(p);
            });
        for (auto &th : pool) th.join();
    }
    for (int p = 0; p < nprob; p++) {
        if (yv[p].empty()) continue;
        const int m = (int)yv[p].size();
        HPHI_CUDA(ctx, cudaMemcpyAsync((double *)hp[p].y, yv[p].data(), sizeof(double) * m, cudaMemcpyHostToDevice,
                                       ctx->stream));
        hp[p].m = m;
        hp[p].theta = theta[p];
        hp[p].gs = (double *)gs_out[p];
        any_gs = true;
    }
    std::vector<double> gres(nprob, -1.0);
    if (any_gs) {
        HPHI_CUDA(ctx, cudaMemcpyAsync(dprob, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice, ctx->stream));
        int stg = batch_launch_gs(ctx, dprob, nprob, dyn_bytes);
        if (stg) return fail(stg);
        std::vector<double> pph(n_pp);
        HPHI_CUDA(ctx, cudaMemcpyAsync(pph.data(), pp, sizeof(double) * n_pp, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int p = 0; p < nprob; p++)
            if (hp[p].gs) gres[p] = pph[(size_t)p * (M + 2) + 1];
    }
    int worst = HPHI_OK;
    for (int p = 0; p < nprob; p++) {
        results[p].e0 = theta[p];
        results[p].resid_est = rest[p];
        results[p].e0_rq = std::nan("");
        results[p].resid = gres[p];
        results[p].steps = mstop[p];
        results[p].breakdown = brk[p];
        if (!st[p] && opts->tol > 0.0 && !conv[p] && !brk[p]) st[p] = HPHI_E_NOTCONV;
        status[p] = st[p];
        if (st[p] && (worst == HPHI_OK || worst == HPHI_E_NOTCONV)) worst = st[p];
    }
    fail(HPHI_OK);
    if (worst) set_err(ctx, worst, "batched Lanczos: see the per-problem status");
    return worst;
}
