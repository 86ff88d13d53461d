// Serving loop: ground-state and dynamical-structure-factor requests of many
// sizes on one GPU with continuous batching.
//
// Small problems run on the batched block engine (batch.cu): every running
// Lanczos recurrence owns one thread block, and one server step launches the
// next chunk of steps of all of them at once.  A request that arrives while
// others run is admitted at the next step, as soon as its workspace fits in
// the server's device arena and a block slot is free; a finished request frees
// both at once.  Between steps the host evaluates each recurrence's stopping
// rule at every step of the chunk (the stop step does not depend on the chunk
// length, the batch, or the other requests, so a result is bit-for-bit the
// same alone and in the mix).
//
// A spectrum request (Sec. 3.2) goes through three phases: the ground state
// (Lanczos + ground-state vector pass), the excitation
// Phi = sum_l e^{i q l} S^z_l Phi_0 (its real and imaginary parts become two
// real right-hand sides), and the Krylov recurrence of each part, stopped when
// every shift's residual  prod_k beta_k / |u_k(z)|  is below the tolerance;
// D(z) is the sum of the parts' continued fractions.  Problems larger than the
// block engine's limit go to a second lane: a host worker thread that runs the
// grid-wide drivers (hphi_lanczos, hphi_apply_sz_sum, hphi_shifted_krylov) on
// its own CUDA stream, concurrently with the block engine.
#include <float.h>
#include <math.h>

#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.cuh"

namespace hphi {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit arena over one device allocation (256-byte granules).
class Arena {
  public:
    int init(hphi_ctx *ctx, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        cudaError_t e = cudaMalloc(&base_, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return set_err(ctx, HPHI_E_NOMEM, "server arena of %zu bytes", bytes);
        }
        size_ = bytes;
        free_[0] = bytes;
        return HPHI_OK;
    }
    ~Arena() { cudaFree(base_); }
    // offset of a free range of `bytes`, or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *at(size_t off) const { return base_ + off; }

  private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

enum Phase { PH_QUEUED = 0, PH_GROUND, PH_GSPASS, PH_KRYLOV, PH_DONE };
enum Role { ROLE_GROUND = 0, ROLE_KRYLOV = 1 };

struct Request;

// One Lanczos recurrence on the block engine.
struct Task {
    Request *req = nullptr;
    int role = ROLE_GROUND;
    BProb P{};
    size_t dyn = 0;
    std::vector<double> a, b2;  // history: alpha_0.., beta_0^2..
    int k = 0;                  // steps done
    double warm = std::nan("");
    bool finished = false, brk = false, conv = false;
    int status = HPHI_OK, m = 0;
    // shifted-Krylov residual recurrences, one per shift
    std::vector<std::complex<double>> u;
    std::vector<double> rho;
    int folded = 0;
};

struct Request {
    int64_t id = 0;
    hphi_request r{};
    std::vector<double> omega;  // shifts relative to E0
    int phase = PH_QUEUED, lane = 0;
    size_t off = 0, bytes = 0;  // arena block
    double *base = nullptr;
    std::unique_ptr<Task> ground;
    std::vector<std::unique_ptr<Task>> kry;
    // results
    int status = HPHI_OK, steps = 0, kry_steps = 0;
    double e0 = 0.0, max_resid = 0.0;
    std::vector<double> d;  // D(z_j): re, im
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    double *gs = nullptr, *ex = nullptr;  // ground state, excitation [D][2]
};

}  // namespace
}  // namespace hphi

using namespace hphi;

struct hphi_server {
    hphi_ctx *ctx = nullptr;
    hphi_server_opts opts{};
    Arena arena;
    Clock::time_point t0;
    int64_t next_id = 1;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::map<int64_t, std::unique_ptr<Request>> all;
    BProb *dprob = nullptr;
    double *stage = nullptr, *stage_h = nullptr;
    int cap = 0;
    // grid lane
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> grid_queue;
    bool stop = false;
    int grid_busy = 0;
    // counters
    int64_t launches = 0, grid_done = 0, block_done = 0;
    size_t arena_used = 0, arena_peak = 0;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

size_t task_doubles(const hphi_ham *h, int M) { return 4 * (size_t)h->D + 2 * (size_t)M + 8 + (size_t)M; }

void init_task(Task &t, Request *q, int role, double *ws, const double *v0, int64_t v0_stride, int M) {
    t.req = q;
    t.role = role;
    t.P = BProb{};
    t.dyn = batch_fill(q->r.ham, t.P);
    const int64_t D = q->r.ham->D;
    t.P.v0 = v0;
    t.P.v0_stride = v0_stride;
    t.P.w = ws;
    t.P.diag = ws + 3 * D;
    t.P.alpha = ws + 4 * D;
    t.P.beta2 = t.P.alpha + M;
    t.P.stride = 1;
    t.P.scal = t.P.beta2 + M + 1;
    t.P.resid = t.P.scal + 1;
    t.P.state = (int *)(t.P.scal + 2);  // two ints in one double slot
    t.P.y = t.P.scal + 4;
}

// The ground-state stopping rule of hphi_lanczos at step j.
int ground_holds(Task &t, int j, double tol, double *th, double *re) {
    double yl = 0.0;
    if (lowest_ritz_warm(j, t.a.data(), t.b2.data(), &t.warm, th, &yl)) return -1;
    *re = sqrt(t.b2[j]) * yl;
    return (tol > 0.0 && j >= 2 && *re <= tol * (fabs(*th) > 1.0 ? fabs(*th) : 1.0)) ? 1 : 0;
}

// Host side of one finished chunk of a task.
void fold_chunk(Task &t, const double *stg, int nsteps, int M) {
    Request *q = t.req;
    const int flag = (int)stg[1 + 2 * nsteps], steps = (int)stg[2 + 2 * nsteps];
    if (t.k == 0) t.b2.assign(1, stg[0]);
    const int k_prev = t.k;
    for (int s = 0; s < steps - k_prev; s++) {
        t.a.push_back(stg[1 + 2 * s]);
        t.b2.push_back(stg[2 + 2 * s]);
    }
    t.k = steps;
    if (flag == 3) {  // zero start vector: an error for a ground state, D = 0 for a Krylov column
        t.finished = true;
        t.status = t.role == ROLE_GROUND ? HPHI_E_INVAL : HPHI_OK;
        return;
    }
    if (flag == 2) {
        t.finished = true;
        t.status = HPHI_E_NUMERIC;
        t.m = steps;
        return;
    }
    const double tol = q->r.tol;
    if (t.role == ROLE_GROUND) {
        double th = 0.0, re = -1.0;
        int m = 0;
        if (tol > 0.0 && steps >= 2) {
            const int h = ground_holds(t, steps, tol, &th, &re);
            if (h < 0) {
                t.finished = true;
                t.status = HPHI_E_NUMERIC;
                return;
            }
            if (h == 1) {
                for (int j = std::max(2, k_prev + 1); j <= steps; j++)
                    if (ground_holds(t, j, tol, &th, &re) == 1) {
                        m = j;
                        break;
                    }
                t.conv = true;
            }
        }
        if (!m && flag == 1) {
            m = steps;
            t.brk = true;
        }
        if (!m && steps >= M) {
            m = steps;
            t.status = tol > 0.0 ? HPHI_E_NOTCONV : HPHI_OK;
        }
        if (m) {
            t.finished = true;
            t.m = m;
        }
        return;
    }
    // Krylov column: residual of every shift after each new step
    const size_t nz = q->omega.size();
    if (t.u.empty()) {
        t.u.assign(nz, std::complex<double>(0.0, 0.0));
        t.rho.assign(nz, 1.0);
    }
    int m = 0;
    for (int j = t.folded; j < steps; j++) {
        double mx = 0.0;
        const double bj1 = sqrt(t.b2[j + 1] > 0.0 ? t.b2[j + 1] : 0.0), bj2 = j > 0 ? t.b2[j] : 0.0;
        for (size_t z = 0; z < nz; z++) {
            const std::complex<double> zz(q->e0 + q->omega[z], q->r.eta);
            t.u[z] = j == 0 ? zz - t.a[j] : zz - t.a[j] - bj2 / t.u[z];
            t.rho[z] *= bj1 / std::abs(t.u[z]);
            mx = t.rho[z] > mx ? t.rho[z] : mx;
        }
        t.folded = j + 1;
        if (tol > 0.0 && mx <= tol) {
            m = j + 1;
            t.conv = true;
            break;
        }
    }
    if (!m && flag == 1) {
        m = steps;
        t.brk = true;
    }
    if (!m && steps >= M) {
        m = steps;
        t.status = tol > 0.0 ? HPHI_E_NOTCONV : HPHI_OK;
    }
    if (m) {
        t.finished = true;
        t.m = m;
    }
}

// D(z) of a finished Krylov column over its own m steps (continued fraction).
void add_cf(const Task &t, Request *q) {
    const double n2 = t.b2.empty() ? 0.0 : t.b2[0];
    const int m = t.m;
    for (size_t z = 0; z < q->omega.size(); z++) {
        if (!(n2 > 0.0) || m < 1) continue;
        const std::complex<double> zz(q->e0 + q->omega[z], q->r.eta);
        std::complex<double> f = zz - t.a[m - 1];
        for (int j = m - 2; j >= 0; j--) f = zz - t.a[j] - t.b2[j + 1] / f;
        const std::complex<double> g = n2 / f;
        q->d[2 * z] += g.real();
        q->d[2 * z + 1] += g.imag();
    }
    double mx = 0.0;
    for (double r : t.rho) mx = r > mx ? r : mx;
    q->max_resid = mx > q->max_resid ? mx : q->max_resid;
}

void weights_of(const Request *q, std::vector<double> &w, bool *complex_part) {
    const int N = q->r.ham->basis->N;
    w.assign(2 * (size_t)N, 0.0);
    bool im = false;
    for (int l = 0; l < N; l++) {
        w[2 * l] = cos(q->r.q * l);
        w[2 * l + 1] = sin(q->r.q * l);
        im = im || fabs(w[2 * l + 1]) > 1e-12;
    }
    if (!im)
        for (int l = 0; l < N; l++) w[2 * l + 1] = 0.0;
    *complex_part = im;
}

// Grid lane: one request at a time with the grid-wide drivers, on its own stream.
void grid_worker(hphi_server *S) {
    hphi_ctx *gc = nullptr;
    cudaSetDevice(S->ctx->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (hphi_ctx_create(S->ctx->device, st, &gc) != HPHI_OK) gc = nullptr;
    for (;;) {
        Request *q = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->grid_queue.empty(); });
            if (S->stop && S->grid_queue.empty()) break;
            q = S->grid_queue.front();
            S->grid_queue.pop_front();
        }
        const hphi_ham *h = q->r.ham;
        const int64_t D = h->D;
        int status = gc ? HPHI_OK : HPHI_E_CUDA;
        double e0 = 0.0, mres = 0.0;
        int steps = 0, ksteps = 0;
        std::vector<double> dz;
        // vector storage: FP64, or FP32 with FP64 scalars (then a ground state
        // also takes the ground-state vector, whose FP64 Rayleigh quotient is the
        // reported energy)
        const int vdt = S->opts.grid_dtype == HPHI_F32 ? HPHI_F32 : HPHI_F64;
        const size_t es = vdt == HPHI_F32 ? 4 : 8;
        void *v = nullptr, *gs = nullptr, *ex = nullptr;
        if (!status && cudaMalloc(&v, es * (size_t)D) != cudaSuccess) status = HPHI_E_NOMEM;
        const bool spec = q->r.kind == HPHI_REQ_SPECTRUM;
        const bool want_gs = spec || vdt == HPHI_F32;
        if (!status && want_gs && cudaMalloc(&gs, es * (size_t)D) != cudaSuccess) status = HPHI_E_NOMEM;
        if (!status && spec && cudaMalloc(&ex, 2 * es * (size_t)D) != cudaSuccess) status = HPHI_E_NOMEM;
        if (!status) status = hphi_random_vector(gc, vdt, D, 1, q->r.seed, v, 1);
        if (!status) {
            // FP32 storage holds the vectors to about 1e-6 relative: the recurrence
            // stops there and the energy comes from the FP64 Rayleigh quotient,
            // whose error is quadratic in the vector's
            const double ltol = (vdt == HPHI_F32 && q->r.tol > 0.0 && q->r.tol < 1e-6) ? 1e-6 : q->r.tol;
            hphi_lanczos_opts o{q->r.max_steps, ltol, vdt, 1, 0};
            hphi_lanczos_result res{};
            status = hphi_lanczos(gc, h, &o, v, want_gs ? gs : nullptr, nullptr, nullptr, &res);
            e0 = (vdt == HPHI_F32 && !spec && res.e0_rq == res.e0_rq) ? res.e0_rq : res.e0;
            steps = res.steps;
        }
        if (!status && spec) {
            std::vector<double> w;
            bool im = false;
            weights_of(q, w, &im);
            status = hphi_apply_sz_sum(gc, h->basis, vdt, gs, 1, ex, 2, w.data());
            if (!status) {
                const int nz = (int)q->omega.size();
                std::vector<double> z(2 * (size_t)nz), g(4 * (size_t)nz), rr(2 * (size_t)nz);
                for (int j = 0; j < nz; j++) {
                    z[2 * j] = e0 + q->omega[j];
                    z[2 * j + 1] = q->r.eta;
                }
                hphi_krylov_opts ko{q->r.max_steps, q->r.tol, vdt, 4};
                hphi_krylov_result kr{};
                status = hphi_shifted_krylov(gc, (hphi_ham *)h, &ko, im ? 2 : 1, ex, 2, nz, z.data(), g.data(),
                                             rr.data(), nullptr, nullptr, &kr);
                ksteps = kr.steps;
                mres = kr.max_resid;
                dz.assign(2 * (size_t)nz, 0.0);
                for (int j = 0; j < nz; j++)
                    for (int c = 0; c < (im ? 2 : 1); c++) {
                        dz[2 * j] += g[2 * ((size_t)c * nz + j)];
                        dz[2 * j + 1] += g[2 * ((size_t)c * nz + j) + 1];
                    }
            }
        }
        cudaFree(v);
        cudaFree(gs);
        cudaFree(ex);
        std::lock_guard<std::mutex> lk(S->mu);
        q->status = status;
        q->e0 = e0;
        q->steps = steps;
        q->kry_steps = ksteps;
        q->max_resid = mres;
        q->d = dz;
        q->t_done = S->now();
        q->phase = PH_DONE;
        S->grid_busy--;
        S->grid_done++;
    }
    if (gc) hphi_ctx_destroy(gc);
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" int hphi_server_create(hphi_ctx *ctx, const hphi_server_opts *opts, hphi_server **out) {
    if (!ctx || !opts || !out) return HPHI_E_INVAL;
    ctx->err.clear();
    *out = nullptr;
    if (!(opts->mem_budget > 0) || opts->max_active < 0 || opts->chunk < 0 || opts->small_max_dim < 0 ||
        opts->grid_workers < 0 || opts->grid_workers > 16 ||
        (opts->grid_dtype != HPHI_F64 && opts->grid_dtype != HPHI_F32))
        return set_err(ctx, HPHI_E_INVAL, "server options");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    std::unique_ptr<hphi_server> S(new (std::nothrow) hphi_server());
    if (!S) return set_err(ctx, HPHI_E_NOMEM, "host allocation failed");
    S->ctx = ctx;
    S->opts = *opts;
    if (S->opts.max_active == 0) S->opts.max_active = 2 * ctx->sm_count;
    if (S->opts.chunk == 0) S->opts.chunk = 16;
    if (S->opts.small_max_dim == 0) S->opts.small_max_dim = (int64_t)1 << 17;
    if (S->opts.grid_workers == 0) S->opts.grid_workers = 2;
    int st = S->arena.init(ctx, (size_t)opts->mem_budget);
    if (st) return st;
    S->cap = S->opts.max_active;
    const size_t stage_n = (size_t)S->cap * (3 + 2 * (size_t)S->opts.chunk);
    if (cudaMalloc(&S->dprob, sizeof(BProb) * (size_t)S->cap) != cudaSuccess ||
        cudaMalloc(&S->stage, sizeof(double) * stage_n) != cudaSuccess ||
        cudaMallocHost(&S->stage_h, sizeof(double) * stage_n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(S->dprob);
        cudaFree(S->stage);
        return set_err(ctx, HPHI_E_NOMEM, "server descriptors");
    }
    S->t0 = Clock::now();
    hphi_server *raw = S.release();
    for (int w = 0; w < raw->opts.grid_workers; w++) raw->workers.emplace_back(grid_worker, raw);
    *out = raw;
    return HPHI_OK;
}

extern "C" void hphi_server_destroy(hphi_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &w : S->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(S->ctx->device);
    cudaStreamSynchronize(S->ctx->stream);
    cudaFree(S->dprob);
    cudaFree(S->stage);
    cudaFreeHost(S->stage_h);
    delete S;
}

extern "C" double hphi_server_clock(const hphi_server *S) { return S ? S->now() : -1.0; }

extern "C" int hphi_server_submit(hphi_server *S, const hphi_request *r, int64_t *id) {
    if (!S || !r || !id) return HPHI_E_INVAL;
    hphi_ctx *ctx = S->ctx;
    ctx->err.clear();
    if (!r->ham || r->ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "request: Hamiltonian");
    if (r->kind != HPHI_REQ_GROUND && r->kind != HPHI_REQ_SPECTRUM) return set_err(ctx, HPHI_E_INVAL, "request kind");
    if (r->max_steps < 1 || r->max_steps > 100000) return set_err(ctx, HPHI_E_INVAL, "request max_steps");
    if (r->kind == HPHI_REQ_SPECTRUM && (r->nz < 1 || !r->omega))
        return set_err(ctx, HPHI_E_INVAL, "spectrum request needs shifts");
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q) return set_err(ctx, HPHI_E_NOMEM, "host allocation failed");
    q->id = S->next_id++;
    q->r = *r;
    if (r->kind == HPHI_REQ_SPECTRUM) q->omega.assign(r->omega, r->omega + r->nz);
    q->r.omega = nullptr;
    q->t_submit = S->now();
    const bool small = r->ham->D <= S->opts.small_max_dim && (int)r->ham->dterms.size() <= kBatchMaxTerms &&
                       !(r->ham->model == HPHI_SPIN_HALF && r->ham->basis->N > 32);
    q->lane = small ? 0 : 1;
    *id = q->id;
    Request *raw = q.get();
    if (small) {
        int st = ensure_rowstate(ctx, r->ham);
        if (st) return st;
        std::lock_guard<std::mutex> lk(S->mu);
        S->all[raw->id] = std::move(q);
        S->queue.push_back(raw);
    } else {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->all[raw->id] = std::move(q);
            raw->phase = PH_GROUND;
            raw->t_start = S->now();
            S->grid_queue.push_back(raw);
            S->grid_busy++;
        }
        S->cv.notify_one();
    }
    return HPHI_OK;
}

extern "C" int hphi_server_step(hphi_server *S, int *n_running, int *n_queued) {
    if (!S) return HPHI_E_INVAL;
    hphi_ctx *ctx = S->ctx;
    ctx->err.clear();
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int M_cap = S->opts.chunk;
    int st;
    // 1. admission (FIFO) by free arena memory and block slots
    auto tasks_of = [](const Request *q) -> int { return q->r.kind == HPHI_REQ_SPECTRUM ? 3 : 1; };
    int slots = 0;
    for (Request *q : S->running) slots += tasks_of(q);
    while (!S->queue.empty()) {
        Request *q = S->queue.front();
        const int M = q->r.max_steps;
        const hphi_ham *h = q->r.ham;
        if (slots + tasks_of(q) > S->opts.max_active) break;
        size_t nd = task_doubles(h, M) + (size_t)h->D;  // ground task + start vector
        if (q->r.kind == HPHI_REQ_SPECTRUM) nd += 3 * (size_t)h->D + 2 * task_doubles(h, M);  // gs, excitation, 2 columns
        const size_t off = S->arena.alloc(nd * sizeof(double));
        if (off == SIZE_MAX) break;
        S->queue.pop_front();
        q->off = off;
        q->bytes = nd * sizeof(double);
        q->base = (double *)S->arena.at(off);
        double *v0 = q->base;
        double *ws = v0 + h->D;
        if ((st = hphi_random_vector(ctx, HPHI_F64, h->D, 1, q->r.seed, v0, 1))) return st;
        S->launches++;
        S->arena_used += q->bytes;
        S->arena_peak = S->arena_used > S->arena_peak ? S->arena_used : S->arena_peak;
        q->ground.reset(new Task());
        init_task(*q->ground, q, ROLE_GROUND, ws, v0, 1, M);
        HPHI_CUDA(ctx, cudaMemsetAsync(q->ground->P.state, 0, 2 * sizeof(int), ctx->stream));
        if (q->r.kind == HPHI_REQ_SPECTRUM) {
            q->gs = ws + task_doubles(h, M);
            q->ex = q->gs + h->D;
        }
        q->phase = PH_GROUND;
        q->t_start = S->now();
        S->running.push_back(q);
        slots += tasks_of(q);
    }
    // 2. ground-state vector passes (requests whose ground phase ended last step),
    //    then their excitations and Krylov columns
    std::vector<BProb> gsd;
    size_t gsdyn = 0;
    for (Request *q : S->running)
        if (q->phase == PH_GSPASS) {
            gsd.push_back(q->ground->P);
            gsdyn = q->ground->dyn > gsdyn ? q->ground->dyn : gsdyn;
        }
    if (!gsd.empty()) {
        HPHI_CUDA(ctx, cudaMemcpyAsync(S->dprob, gsd.data(), sizeof(BProb) * gsd.size(), cudaMemcpyHostToDevice,
                                       ctx->stream));
        if ((st = batch_launch_gs(ctx, S->dprob, (int)gsd.size(), gsdyn))) return st;
        S->launches++;
        // the descriptors are read by the launch before the next upload (same stream)
        for (Request *q : S->running) {
            if (q->phase != PH_GSPASS) continue;
            const hphi_ham *h = q->r.ham;
            const int M = q->r.max_steps;
            std::vector<double> w;
            bool im = false;
            weights_of(q, w, &im);
            if ((st = hphi_apply_sz_sum(ctx, h->basis, HPHI_F64, q->gs, 1, q->ex, 2, w.data()))) return st;
            S->launches++;
            double *kws = q->ex + 2 * h->D;
            for (int c = 0; c < (im ? 2 : 1); c++) {
                std::unique_ptr<Task> t(new Task());
                init_task(*t, q, ROLE_KRYLOV, kws + (size_t)c * task_doubles(h, M), q->ex + c, 2, M);
                HPHI_CUDA(ctx, cudaMemsetAsync(t->P.state, 0, 2 * sizeof(int), ctx->stream));
                q->kry.push_back(std::move(t));
            }
            q->d.assign(2 * q->omega.size(), 0.0);
            q->phase = PH_KRYLOV;
        }
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // before the descriptor buffer is rewritten
    }
    // 3. one chunk of every running recurrence
    std::vector<Task *> live;
    for (Request *q : S->running) {
        if (q->phase == PH_GROUND && !q->ground->finished) live.push_back(q->ground.get());
        if (q->phase == PH_KRYLOV)
            for (auto &t : q->kry)
                if (!t->finished) live.push_back(t.get());
    }
    const int n = (int)live.size();
    if (n > S->cap) return set_err(ctx, HPHI_E_INVAL, "more live recurrences than block slots");
    if (n > 0) {
        std::vector<BProb> d(n);
        size_t dyn = 0;
        for (int i = 0; i < n; i++) {
            Task *t = live[i];
            t->P.k0 = t->k;
            t->P.nsteps = std::min(M_cap, t->req->r.max_steps - t->k);
            t->P.stage = S->stage + (size_t)i * (3 + 2 * (size_t)M_cap);
            t->P.m = 0;
            t->P.gs = nullptr;
            d[i] = t->P;
            dyn = t->dyn > dyn ? t->dyn : dyn;
        }
        HPHI_CUDA(ctx, cudaMemcpyAsync(S->dprob, d.data(), sizeof(BProb) * n, cudaMemcpyHostToDevice, ctx->stream));
        if ((st = batch_launch_steps(ctx, S->dprob, n, dyn))) return st;
        S->launches++;
        const size_t sn = (size_t)n * (3 + 2 * (size_t)M_cap);
        HPHI_CUDA(ctx, cudaMemcpyAsync(S->stage_h, S->stage, sizeof(double) * sn, cudaMemcpyDeviceToHost, ctx->stream));
        HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int i = 0; i < n; i++) {
            Task *t = live[i];
            fold_chunk(*t, S->stage_h + (size_t)i * (3 + 2 * (size_t)M_cap), t->P.nsteps, t->req->r.max_steps);
        }
    }
    // 4. phase changes and retirement
    std::vector<Request *> keep;
    for (Request *q : S->running) {
        bool retire = false;
        if (q->phase == PH_GROUND && q->ground->finished) {
            Task &g = *q->ground;
            q->steps = g.m;
            q->status = g.status;
            if (!g.status && g.m >= 1) {
                const int m = g.m;
                std::vector<double> bb(m, 0.0), ev(m), Z((size_t)m * m);
                for (int j = 1; j < m; j++) bb[j] = sqrt(g.b2[j]);
                int s2 = hphi_tridiag_eigen(m, g.a.data(), bb.data(), ev.data(), Z.data());
                if (s2) q->status = s2;
                q->e0 = ev[0];
                if (!q->status && q->r.kind == HPHI_REQ_SPECTRUM) {
                    std::vector<double> y(m);
                    for (int i = 0; i < m; i++) y[i] = Z[(size_t)i * m];
                    HPHI_CUDA(ctx, cudaMemcpy((double *)g.P.y, y.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
                    g.P.m = m;
                    g.P.theta = q->e0;
                    g.P.gs = q->gs;
                    q->phase = PH_GSPASS;
                }
            }
            if (q->phase == PH_GROUND) retire = true;  // ground request done (or failed)
        } else if (q->phase == PH_KRYLOV) {
            bool all = true;
            for (auto &t : q->kry) all = all && t->finished;
            if (all) {
                for (auto &t : q->kry) {
                    add_cf(*t, q);
                    q->kry_steps = t->m > q->kry_steps ? t->m : q->kry_steps;
                    if (t->status && !q->status) q->status = t->status;
                }
                retire = true;
            }
        }
        if (retire) {
            q->phase = PH_DONE;
            q->t_done = S->now();
            S->arena.release(q->off, q->bytes);
            S->arena_used -= q->bytes;
            S->block_done++;
            q->ground.reset();
            q->kry.clear();
        } else {
            keep.push_back(q);
        }
    }
    S->running.swap(keep);
    if (n_running) {
        std::lock_guard<std::mutex> lk(S->mu);
        *n_running = (int)S->running.size() + S->grid_busy;
    }
    if (n_queued) *n_queued = (int)S->queue.size();
    return HPHI_OK;
}

extern "C" int hphi_server_get_stats(hphi_server *S, hphi_server_stats *out) {
    if (!S || !out) return HPHI_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    out->block_launches = S->launches;
    out->block_done = S->block_done;
    out->grid_done = S->grid_done;
    out->block_running = (int)S->running.size();
    out->grid_running = S->grid_busy;
    out->queued = (int)S->queue.size();
    out->arena_used = (double)S->arena_used;
    out->arena_peak = (double)S->arena_peak;
    return HPHI_OK;
}

extern "C" int hphi_server_result(hphi_server *S, int64_t id, hphi_reply *out, double *d_out) {
    if (!S || !out) return HPHI_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return set_err(S->ctx, HPHI_E_INVAL, "unknown request %lld", (long long)id);
    const Request *q = it->second.get();
    out->done = q->phase == PH_DONE;
    out->status = q->status;
    out->e0 = q->e0;
    out->steps = q->steps;
    out->krylov_steps = q->kry_steps;
    out->max_resid = q->max_resid;
    out->t_submit = q->t_submit;
    out->t_start = q->t_start;
    out->t_done = q->t_done;
    out->lane = q->lane;
    if (d_out && out->done)
        for (size_t j = 0; j < q->d.size(); j++) d_out[j] = q->d[j];
    return HPHI_OK;
}
