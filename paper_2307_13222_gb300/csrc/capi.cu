// C ABI: context, errors, workspace, H*x and vector-kernel entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <new>

#include <map>
#include <mutex>
#include <tuple>

#include "hphi_internal.cuh"

namespace hphi {

int set_err(hphi_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_err(hphi_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    int code = (e == cudaErrorMemoryAllocation) ? HPHI_E_NOMEM : HPHI_E_CUDA;
    return set_err(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

int ensure_partials(hphi_ctx *ctx, size_t n) {
    if (ctx->partials_n >= n) return HPHI_OK;
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->partials);
    ctx->partials = nullptr;
    ctx->partials_n = 0;
    size_t want = n < 65536 ? 65536 : n;
    cudaError_t e = cudaMalloc(&ctx->partials, want * sizeof(double));
    if (e != cudaSuccess) return cuda_err(ctx, e, "partials buffer");
    ctx->partials_n = want;
    return HPHI_OK;
}

int ensure_dscal(hphi_ctx *ctx, size_t n) {
    if (ctx->dscal_n >= n) return HPHI_OK;
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->dscal);
    cudaFreeHost(ctx->hscal);
    ctx->dscal = nullptr;
    ctx->hscal = nullptr;
    ctx->dscal_n = 0;
    cudaError_t e = cudaMalloc(&ctx->dscal, n * sizeof(double));
    if (e != cudaSuccess) return cuda_err(ctx, e, "scalar buffer");
    e = cudaMallocHost(&ctx->hscal, n * sizeof(double));
    if (e != cudaSuccess) return cuda_err(ctx, e, "pinned scalar buffer");
    ctx->dscal_n = n;
    return HPHI_OK;
}

int dyn_occupancy(hphi_ctx *ctx, const void *fn, int threads, size_t dyn) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> limit;              // raised limit per (kernel, device)
    static std::map<std::tuple<const void *, int, size_t>, int> occupancy;  // per (kernel, device, size)
    std::lock_guard<std::mutex> lk(mu);
    const int dev = ctx->device;
    auto key = std::make_pair(fn, dev);
    auto it = limit.find(key);
    if (it == limit.end()) {
        int optin = 0;
        cudaFuncAttributes fa{};
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const size_t mx = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        it = limit.emplace(key, mx).first;
    }
    if (dyn > it->second) return 0;
    auto ok = std::make_tuple(fn, dev, dyn);
    auto jt = occupancy.find(ok);
    if (jt != occupancy.end()) return jt->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, dyn) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    occupancy.emplace(ok, n);
    return n;
}

int ensure_vecs(hphi_ctx *ctx, size_t bytes) {
    if (ctx->vec_bytes >= bytes) return HPHI_OK;
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 4; i++) {
        cudaFree(ctx->vec[i]);
        ctx->vec[i] = nullptr;
    }
    ctx->vec_bytes = 0;
    for (int i = 0; i < 3; i++) {
        cudaError_t e = cudaMalloc(&ctx->vec[i], bytes);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; k++) {
                cudaFree(ctx->vec[k]);
                ctx->vec[k] = nullptr;
            }
            return cuda_err(ctx, e, "driver vectors");
        }
    }
    ctx->vec_bytes = bytes;
    return HPHI_OK;
}

static cudaEvent_t take_event(hphi_ctx *ctx) {
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int prof_begin(hphi_ctx *ctx, int kind) {
    if (!ctx->prof) return -1;
    cudaEvent_t a = take_event(ctx), b = take_event(ctx);
    if (!a || !b) return -1;
    cudaEventRecord(a, ctx->stream);
    ctx->ev_pending.push_back({kind, {a, b}});
    return (int)ctx->ev_pending.size() - 1;
}

void prof_end(hphi_ctx *ctx, int slot) {
    if (slot < 0 || slot >= (int)ctx->ev_pending.size()) return;
    cudaEventRecord(ctx->ev_pending[slot].second.second, ctx->stream);
}

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_ctx_profile(hphi_ctx *ctx, int enable) {
    if (!ctx) return HPHI_E_INVAL;
    ctx->prof = enable != 0;
    return HPHI_OK;
}

extern "C" int hphi_ctx_profile_read(hphi_ctx *ctx, int kind, int64_t *launches, double *total_ms) {
    if (!ctx || !launches || !total_ms) return HPHI_E_INVAL;
    ctx->err.clear();
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t n = 0;
    double t = 0.0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
    for (auto &p : ctx->ev_pending) {
        if (p.first != kind) {
            keep.push_back(p);
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            t += ms;
            n++;
        } else {
            cudaGetLastError();
        }
        ctx->ev_free.push_back(p.second.first);
        ctx->ev_free.push_back(p.second.second);
    }
    ctx->ev_pending.swap(keep);
    *launches = n;
    *total_ms = t;
    return HPHI_OK;
}

extern "C" int hphi_ctx_create(int device, void *stream, hphi_ctx **out) {
    if (!out) return HPHI_E_INVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n || device >= 64) {
        cudaGetLastError();
        return HPHI_E_INVAL;
    }
    hphi_ctx *c = new (std::nothrow) hphi_ctx();
    if (!c) return HPHI_E_NOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        ensure_dscal(c, 4096) != HPHI_OK || cudaMalloc(&c->dflag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        hphi_ctx_destroy(c);
        return HPHI_E_CUDA;
    }
    *out = c;
    return HPHI_OK;
}

extern "C" int hphi_ctx_set_stream(hphi_ctx *ctx, void *stream) {
    if (!ctx) return HPHI_E_INVAL;
    ctx->stream = (cudaStream_t)stream;
    return HPHI_OK;
}

extern "C" void hphi_ctx_destroy(hphi_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->partials);
    cudaFree(ctx->dscal);
    cudaFreeHost(ctx->hscal);
    for (int i = 0; i < 4; i++) cudaFree(ctx->vec[i]);
    for (int i = 0; i < 4; i++) cudaFree(ctx->io[i]);
    for (int i = 0; i < 2; i++)
        if (ctx->io_stream[i]) {
            cudaStreamSynchronize(ctx->io_stream[i]);
            cudaStreamDestroy(ctx->io_stream[i]);
        }
    for (auto e : ctx->io_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(ctx->dflag);
    cudaFree(ctx->seg_tmp);
    for (auto &p : ctx->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    cudaGetLastError();
    delete ctx;
}

extern "C" const char *hphi_last_error(const hphi_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }
extern "C" const char *hphi_last_kernel(const hphi_ctx *ctx) { return ctx ? ctx->last_kernel : ""; }

extern "C" int hphi_ctx_sm_count(const hphi_ctx *ctx) { return ctx ? ctx->sm_count : 0; }

namespace {

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    uintptr_t a0 = (uintptr_t)a, a1 = a0 + abytes, b0 = (uintptr_t)b, b1 = b0 + bbytes;
    return a0 < b1 && b0 < a1;
}

size_t span_bytes(int64_t n, int64_t ld, int nr, size_t es) { return n > 0 ? ((size_t)(n - 1) * ld + nr) * es : 0; }

int check_vec(hphi_ctx *ctx, int dtype, int64_t n, int nvec, int64_t ld, const void *p, const char *name) {
    if (!valid_dtype(dtype)) return set_err(ctx, HPHI_E_INVAL, "unknown dtype %d", dtype);
    if (nvec < 1) return set_err(ctx, HPHI_E_INVAL, "nvec must be >= 1");
    if (ld < nvec) return set_err(ctx, HPHI_E_INVAL, "%s: leading dimension %lld < nvec %d", name, (long long)ld, nvec);
    if (n > 0 && !p) return set_err(ctx, HPHI_E_INVAL, "%s is NULL", name);
    return HPHI_OK;
}

}  // namespace

extern "C" int hphi_apply_H(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, const void *x, int64_t ldx,
                            void *y, int64_t ldy, double alpha, double beta) {
    if (!ctx || !ham) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, ham->D, nvec, ldx, x, "x")) || (st = check_vec(ctx, dtype, ham->D, nvec, ldy, y, "y")))
        return st;
    const int cpl = is_complex(dtype) ? 2 : 1;
    const int nr = nvec * cpl;
    if (nr > kMaxCols) return set_err(ctx, HPHI_E_INVAL, "at most %d real columns per call", kMaxCols);
    const size_t es = real_size(real_of(dtype));
    if (overlaps(x, span_bytes(ham->D, ldx * cpl, nr, es), y, span_bytes(ham->D, ldy * cpl, nr, es)))
        return set_err(ctx, HPHI_E_INVAL, "x and y overlap");
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    HvLaunch L{};
    L.dtype_real = real_of(dtype);
    L.ncol = nr;
    L.x = x;
    L.ldx = ldx * cpl;
    L.y = y;
    L.ldy = ldy * cpl;
    L.v = nullptr;
    L.ldv = 0;
    L.beta = beta;
    L.alpha_s = alpha;
    L.gamma_s = 0.0;
    return launch_hv(ctx, ham, L);
}

namespace {

// Device buffers, copy streams and events of hphi_apply_H_host, made on first use.
int ensure_io(hphi_ctx *ctx, size_t bytes) {
    for (int i = 0; i < 2; i++)
        if (!ctx->io_stream[i]) HPHI_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->io_stream[i], cudaStreamNonBlocking));
    for (auto &e : ctx->io_ev)
        if (!e) HPHI_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (ctx->io_bytes >= bytes) return HPHI_OK;
    HPHI_CUDA(ctx, cudaDeviceSynchronize());
    for (int i = 0; i < 4; i++) {
        cudaFree(ctx->io[i]);
        ctx->io[i] = nullptr;
    }
    ctx->io_bytes = 0;
    for (int i = 0; i < 4; i++) {
        cudaError_t e = cudaMalloc(&ctx->io[i], bytes);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; k++) {
                cudaFree(ctx->io[k]);
                ctx->io[k] = nullptr;
            }
            return cuda_err(ctx, e, "host-vector buffers");
        }
    }
    ctx->io_bytes = bytes;
    return HPHI_OK;
}

}  // namespace

extern "C" int hphi_apply_H_host(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, int64_t nbatch,
                                 const void *x_host, void *y_host, double alpha) {
    if (!ctx || !ham) return HPHI_E_INVAL;
    ctx->err.clear();
    if (!valid_dtype(dtype)) return set_err(ctx, HPHI_E_INVAL, "unknown dtype %d", dtype);
    if (nvec < 1 || nbatch < 0) return set_err(ctx, HPHI_E_INVAL, "nvec >= 1 and nbatch >= 0 required");
    if (nbatch > 0 && (!x_host || !y_host)) return set_err(ctx, HPHI_E_INVAL, "x_host / y_host is NULL");
    const int cpl = is_complex(dtype) ? 2 : 1;
    if (nvec * cpl > kMaxCols) return set_err(ctx, HPHI_E_INVAL, "at most %d real columns per call", kMaxCols);
    if (ham->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "hamiltonian belongs to another device");
    const size_t bytes = (size_t)ham->D * nvec * cpl * real_size(real_of(dtype));
    if (overlaps(x_host, bytes * nbatch, y_host, bytes * nbatch)) return set_err(ctx, HPHI_E_INVAL, "x and y overlap");
    if (nbatch == 0) return HPHI_OK;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    int st = ensure_io(ctx, bytes);
    if (st) return st;
    cudaStream_t comp = ctx->stream, up = ctx->io_stream[0], down = ctx->io_stream[1];
    // events: [0] start of the call on the compute stream, [1 + s] x slot s on the
    // device, [3 + s] product of slot s done, [5 + s] y slot s copied back
    cudaEvent_t *ev = ctx->io_ev;
    HPHI_CUDA(ctx, cudaEventRecord(ev[0], comp));  // buffers free of earlier work on the stream
    HPHI_CUDA(ctx, cudaStreamWaitEvent(up, ev[0], 0));
    HPHI_CUDA(ctx, cudaStreamWaitEvent(down, ev[0], 0));
    const char *xh = (const char *)x_host;
    char *yh = (char *)y_host;
    for (int64_t b = 0; b < nbatch && !st; b++) {
        const int s = (int)(b & 1);
        void *xd = ctx->io[s], *yd = ctx->io[2 + s];
        // x_b up once the product of b - 2 has read the slot
        if (b >= 2) HPHI_CUDA(ctx, cudaStreamWaitEvent(up, ev[3 + s], 0));
        HPHI_CUDA(ctx, cudaMemcpyAsync(xd, xh + b * bytes, bytes, cudaMemcpyHostToDevice, up));
        HPHI_CUDA(ctx, cudaEventRecord(ev[1 + s], up));
        // product once x_b is there and y_{b-2} has left the slot
        HPHI_CUDA(ctx, cudaStreamWaitEvent(comp, ev[1 + s], 0));
        if (b >= 2) HPHI_CUDA(ctx, cudaStreamWaitEvent(comp, ev[5 + s], 0));
        st = hphi_apply_H(ctx, ham, dtype, nvec, xd, nvec, yd, nvec, alpha, 0.0);
        if (st) break;
        HPHI_CUDA(ctx, cudaEventRecord(ev[3 + s], comp));
        // y_b down after its product
        HPHI_CUDA(ctx, cudaStreamWaitEvent(down, ev[3 + s], 0));
        HPHI_CUDA(ctx, cudaMemcpyAsync(yh + b * bytes, yd, bytes, cudaMemcpyDeviceToHost, down));
        HPHI_CUDA(ctx, cudaEventRecord(ev[5 + s], down));
    }
    // the caller's stream resumes after the last copy back; the call returns with
    // every y_b on the host
    cudaError_t e1 = cudaStreamSynchronize(up), e2 = cudaStreamSynchronize(down), e3 = cudaStreamSynchronize(comp);
    if (st) return st;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return cuda_err(ctx, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "hphi_apply_H_host");
    return HPHI_OK;
}

extern "C" int hphi_dot(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const void *x, int64_t ldx, const void *y,
                        int64_t ldy, double *out) {
    if (!ctx || !out || n < 0) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, n, nvec, ldx, x, "x")) || (st = check_vec(ctx, dtype, n, nvec, ldy, y, "y")))
        return st;
    const int cpl = is_complex(dtype) ? 2 : 1, nr = nvec * cpl;
    if (nr > 2 * kMaxCols) return set_err(ctx, HPHI_E_INVAL, "too many columns");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    if (n == 0) {
        for (int k = 0; k < nvec * cpl; k++) out[k] = 0.0;
        return HPHI_OK;
    }
    if ((st = launch_dot(ctx, real_of(dtype), cpl == 2, n, nr, x, ldx * cpl, y, ldy * cpl, ctx->dscal))) return st;
    HPHI_CUDA(ctx, cudaMemcpyAsync(ctx->hscal, ctx->dscal, 2 * nr * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const double *S = ctx->hscal, *X = ctx->hscal + nr;
    for (int q = 0; q < nvec; q++) {
        if (cpl == 1) {
            out[q] = S[q];
        } else {
            out[2 * q] = S[2 * q] + S[2 * q + 1];           // re x re + im x im
            out[2 * q + 1] = X[2 * q] - X[2 * q + 1];       // re x im - im x re
        }
    }
    return HPHI_OK;
}

extern "C" int hphi_nrm2(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const void *x, int64_t ldx, double *out) {
    if (!ctx || !out || n < 0) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, n, nvec, ldx, x, "x"))) return st;
    const int cpl = is_complex(dtype) ? 2 : 1, nr = nvec * cpl;
    if (nr > 2 * kMaxCols) return set_err(ctx, HPHI_E_INVAL, "too many columns");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    if (n == 0) {
        for (int k = 0; k < nvec; k++) out[k] = 0.0;
        return HPHI_OK;
    }
    if ((st = launch_dot(ctx, real_of(dtype), 0, n, nr, x, ldx * cpl, x, ldx * cpl, ctx->dscal))) return st;
    HPHI_CUDA(ctx, cudaMemcpyAsync(ctx->hscal, ctx->dscal, nr * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < nvec; q++) {
        double s = ctx->hscal[q * cpl] + (cpl == 2 ? ctx->hscal[q * cpl + 1] : 0.0);
        out[q] = sqrt(s);
    }
    return HPHI_OK;
}

namespace {

int axpby_common(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const double *a, const void *x, int64_t ldx, void *y,
                 int64_t ldy, bool scal) {
    const int cpl = is_complex(dtype) ? 2 : 1, nr = nvec * cpl;
    if (nr > 256) return set_err(ctx, HPHI_E_INVAL, "too many columns");
    double A[256], B[256], G[256];
    for (int q = 0; q < nvec; q++) {
        if (cpl == 1) {
            A[q] = a[q];
            B[q] = 0.0;
        } else {
            double re = a[2 * q], im = a[2 * q + 1];
            A[2 * q] = re;
            B[2 * q] = -im;  // re part: re*x_re - im*x_im
            A[2 * q + 1] = re;
            B[2 * q + 1] = im;  // im part: re*x_im + im*x_re
        }
    }
    for (int c = 0; c < nr; c++) G[c] = scal ? 0.0 : 1.0;
    LinComb L{};
    L.real_dtype = real_of(dtype);
    L.n = n;
    L.nr = nr;
    L.x = x;
    L.ldx = ldx * cpl;
    L.y = scal ? nullptr : y;
    L.ldy = ldy * cpl;
    L.out = y;
    L.ldo = ldy * cpl;
    L.a_h = A;
    L.b_h = B;
    L.g_h = G;
    L.coef_dev = nullptr;
    L.red_oo = 0;
    L.partials = nullptr;
    return launch_lincomb(ctx, L);
}

}  // namespace

extern "C" int hphi_axpy(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const double *a, const void *x, int64_t ldx,
                         void *y, int64_t ldy) {
    if (!ctx || !a || n < 0) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, n, nvec, ldx, x, "x")) || (st = check_vec(ctx, dtype, n, nvec, ldy, y, "y")))
        return st;
    if (n == 0) return HPHI_OK;
    const int cpl = is_complex(dtype) ? 2 : 1;
    const size_t es = real_size(real_of(dtype));
    if (overlaps(x, span_bytes(n, ldx * cpl, nvec * cpl, es), y, span_bytes(n, ldy * cpl, nvec * cpl, es)) && x != y)
        return set_err(ctx, HPHI_E_INVAL, "x and y overlap partially");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    return axpby_common(ctx, dtype, n, nvec, a, x, ldx, y, ldy, false);
}

extern "C" int hphi_scal(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const double *a, void *x, int64_t ldx) {
    if (!ctx || !a || n < 0) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, n, nvec, ldx, x, "x"))) return st;
    if (n == 0) return HPHI_OK;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    return axpby_common(ctx, dtype, n, nvec, a, x, ldx, x, ldx, true);
}

extern "C" int hphi_random_vector(hphi_ctx *ctx, int dtype, int64_t n, int nvec, uint64_t seed, void *x,
                                  int64_t ldx) {
    if (!ctx || n < 0) return HPHI_E_INVAL;
    ctx->err.clear();
    int st;
    if ((st = check_vec(ctx, dtype, n, nvec, ldx, x, "x"))) return st;
    if (n == 0) return HPHI_OK;
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const int cpl = is_complex(dtype) ? 2 : 1;
    return launch_random(ctx, real_of(dtype), n, nvec * cpl, seed, x, ldx * cpl);
}
