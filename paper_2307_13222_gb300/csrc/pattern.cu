// Debug export of the matrix pattern (the paper's Matrix Market output of H,
// Sec. 3.1.2): rows [row0, row1) enumerated by the same row visitor as the
// H*x kernel, then sorted and merged per row on the host.
#include <algorithm>
#include <vector>

#include "rowvisit.cuh"

namespace hphi {

namespace {

struct DumpSink {
    int64_t *cols;
    double *vals;
    int n, cap;
    __device__ __forceinline__ void diag(int64_t r, double d) {
        cols[0] = r;
        vals[0] = d;
        n = 1;
    }
    __device__ __forceinline__ void add8(const int64_t (&t)[kChunk], const double (&c)[kChunk]) {
        for (int u = 0; u < kChunk; u++) {
            if (t[u] < 0) continue;
            if (n < cap) {
                cols[n] = t[u];
                vals[n] = c[u];
            }
            n++;
        }
    }
};

__global__ void k_dump(HvTables P, int64_t h0, int64_t h1, int64_t r0, int64_t r1, int stride, int64_t *cols,
                       double *vals, int32_t *cnt) {
    __shared__ HBlock<double> hb;
    __shared__ double coef_sm[kMaxCoef];
    for (int i = threadIdx.x; i < P.desc->n_ncoef; i += blockDim.x) coef_sm[i] = P.desc->coef[i];
    for (int64_t h = h0 + blockIdx.x; h < h1; h += gridDim.x) {
        __syncthreads();
        setup_block<double>(P, h, hb);
        if (!hb.valid) continue;
        if (hb.base >= r1 || hb.base + (int64_t)hb.len <= r0) continue;
        for (uint32_t q = threadIdx.x; q < hb.len; q += blockDim.x) {
            int64_t row = hb.base + q;
            if (row < r0 || row >= r1) continue;
            DumpSink s{cols + (row - r0) * stride, vals + (row - r0) * stride, 0, stride};
            visit_row<double>(P, hb, coef_sm, q, s);
            cnt[row - r0] = s.n;
        }
    }
}

HvTables tables_f64(const hphi_ham *ham) {
    const hphi_basis *b = ham->basis;
    HvTables P{};
    P.desc = ham->desc;
    P.model = ham->model;
    P.nlo = ham->nlo;
    P.ngroups = ham->host.ngroups;
    P.n = ham->host.n;
    P.nh = ham->nh;
    P.L = ham->L;
    P.ddn = ham->host.ddn;
    P.jb = b->sp[0].jb;
    P.loff = b->sp[0].loff;
    P.lstate = b->sp[0].lstate;
    P.states_up = b->sp[0].states;
    P.states_dn = b->sp[1].states;
    P.dlow = ham->dlow_d;
    P.ll_cnt = ham->ll_cnt;
    P.ll_tgt = ham->ll_tgt;
    P.ll_cf = ham->ll_cf;
    P.flipq = ham->flipq;
    P.up_cnt = ham->up_cnt;
    P.up_tgt = ham->up_tgt;
    P.up_cf = ham->up_cf;
    P.aup = ham->aup;
    return P;
}

}  // namespace

int dump_rows(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1, std::vector<int64_t> &cols,
              std::vector<double> &vals, std::vector<int32_t> &cnt, int &stride) {
    const hphi_basis *b = ham->basis;
    const int64_t nr = row1 - row0;
    stride = ham->max_row_entries;
    // block range covering the rows
    int64_t h0, h1;
    if (ham->model == HPHI_SPIN_HALF_GC) {
        h0 = row0 >> ham->nlo;
        h1 = ((row1 - 1) >> ham->nlo) + 1;
    } else if (ham->model == HPHI_HUBBARD) {
        h0 = row0 / ham->host.ddn;
        h1 = (row1 - 1) / ham->host.ddn + 1;
    } else {
        const int64_t H = ham->nh;
        std::vector<uint64_t> jbp(H + 1);
        HPHI_CUDA(ctx, cudaMemcpy(jbp.data(), b->sp[0].jbp, (H + 1) * 8, cudaMemcpyDeviceToHost));
        // largest h with jbp[h] <= row
        h0 = (int64_t)(std::upper_bound(jbp.begin(), jbp.begin() + H, (uint64_t)row0) - jbp.begin()) - 1;
        h1 = (int64_t)(std::upper_bound(jbp.begin(), jbp.begin() + H, (uint64_t)(row1 - 1)) - jbp.begin());
        if (h0 < 0) h0 = 0;
    }
    int64_t *d_cols = nullptr;
    double *d_vals = nullptr;
    int32_t *d_cnt = nullptr;
    size_t ne = (size_t)nr * stride;
    if (cudaMalloc(&d_cols, ne * 8) != cudaSuccess || cudaMalloc(&d_vals, ne * 8) != cudaSuccess ||
        cudaMalloc(&d_cnt, nr * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_cols);
        cudaFree(d_vals);
        return set_err(ctx, HPHI_E_NOMEM, "pattern buffers");
    }
    int64_t nb = h1 - h0;
    int grid = (int)(nb < 1024 ? (nb < 1 ? 1 : nb) : 1024);
    k_dump<<<grid, 256, 0, ctx->stream>>>(tables_f64(ham), h0, h1, row0, row1, stride, d_cols, d_vals, d_cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) {
        cols.resize(ne);
        vals.resize(ne);
        cnt.resize(nr);
        e = cudaMemcpy(cols.data(), d_cols, ne * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(vals.data(), d_vals, ne * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), d_cnt, nr * 4, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_cols);
    cudaFree(d_vals);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return cuda_err(ctx, e, "pattern dump");
    return HPHI_OK;
}

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_dump_pattern(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1,
                                 int64_t *rowptr, int64_t *cols_out, double *vals_out, int64_t *cap) {
    if (!ctx || !ham || !rowptr || !cap) return HPHI_E_INVAL;
    ctx->err.clear();
    if (row0 < 0 || row1 > ham->D || row0 >= row1) return set_err(ctx, HPHI_E_INVAL, "bad row range");
    if (row1 - row0 > (1 << 22)) return set_err(ctx, HPHI_E_INVAL, "at most 2^22 rows per dump");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<int64_t> cols;
    std::vector<double> vals;
    std::vector<int32_t> cnt;
    int stride = 0;
    int st = dump_rows(ctx, ham, row0, row1, cols, vals, cnt, stride);
    if (st) return st;
    const int64_t nr = row1 - row0;
    std::vector<std::pair<int64_t, double>> ent;
    int64_t pos = 0;
    // first pass: count merged entries
    std::vector<int64_t> merged_counts(nr);
    for (int64_t r = 0; r < nr; r++) {
        int n = cnt[r];
        if (n > stride || n < 1) return set_err(ctx, HPHI_E_DEVICE_CHECK, "row %lld: %d entries", (long long)(row0 + r), n);
        ent.clear();
        for (int k = 0; k < n; k++) ent.emplace_back(cols[r * stride + k], vals[r * stride + k]);
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
                             return a.first < b.first;
                         });
        int64_t m = 0;
        for (size_t k = 0; k < ent.size(); k++)
            if (k == 0 || ent[k].first != ent[k - 1].first) m++;
        merged_counts[r] = m;
        pos += m;
    }
    if (pos > *cap || !cols_out || !vals_out) {
        *cap = pos;
        return set_err(ctx, HPHI_E_INVAL, "pattern needs %lld entries", (long long)pos);
    }
    pos = 0;
    for (int64_t r = 0; r < nr; r++) {
        rowptr[r] = pos;
        int n = cnt[r];
        ent.clear();
        for (int k = 0; k < n; k++) ent.emplace_back(cols[r * stride + k], vals[r * stride + k]);
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
                             return a.first < b.first;
                         });
        for (size_t k = 0; k < ent.size(); k++) {
            if (k > 0 && ent[k].first == ent[k - 1].first) {
                vals_out[pos - 1] += ent[k].second;
            } else {
                cols_out[pos] = ent[k].first;
                vals_out[pos] = ent[k].second;
                pos++;
            }
        }
    }
    rowptr[nr] = pos;
    *cap = pos;
    return HPHI_OK;
}
