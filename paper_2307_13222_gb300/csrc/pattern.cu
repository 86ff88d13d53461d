// Debug exports of the matrix pattern (the paper's Matrix Market output of H,
// Sec. 3.1.2).
//   hphi_dump_pattern: every off-diagonal entry of rows [row0, row1) as
//     (row, col, fermion sign, term id), one entry per term (and species)
//     acting on the row's state, in term order: the row's state from the
//     basis (Lin-table unrank), the target's row from the basis rank (Lin's
//     two tables), the sign from the popcount of the occupied sites between
//     the hop's ends.  Duplicate and cancelling terms stay separate entries.
//   hphi_dump_pattern_merged: rows enumerated by the same row visitor as the
//     H*x kernel, then sorted and merged per row on the host.
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

// ---- term-order export ---------------------------------------------------------
struct TermSp {             // Lin tables and unrank data of one species
    const uint32_t *ja;
    const uint64_t *jb, *jbp;
    const uint32_t *loff, *lstate;
    int N, n, nlo, nhi;
};

__device__ __forceinline__ int64_t tsp_rank(const TermSp &s, uint64_t x) {
    if (s.N < 64 && (x >> s.N) != 0) return -1;
    if (__popcll(x) != s.n) return -1;
    const uint64_t b = s.jb[x >> s.nlo];
    if (b == ~0ull) return -1;
    return (int64_t)(b + s.ja[x & ((1ull << s.nlo) - 1)]);
}

__device__ __forceinline__ uint64_t tsp_state(const TermSp &s, uint64_t r) {
    uint64_t lo = 0, hi = 1ull << s.nhi;  // largest h with jbp[h] <= r
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (s.jbp[mid] <= r) lo = mid;
        else hi = mid;
    }
    const int p = s.n - __popcll(lo);
    return (lo << s.nlo) | s.lstate[s.loff[p] + (uint32_t)(r - s.jbp[lo])];
}

// One thread per row: the row's off-diagonal entries in term order.  stride
// = 2 n_terms slots per row (a hop on both species gives two entries).
__global__ void k_dump_terms(int model, TermSp up, TermSp dn, int64_t ddn, const hphi_term *terms, int nt,
                             int64_t r0, int64_t nr, int stride, int64_t *cols, int8_t *signs, int32_t *tids,
                             int32_t *cnt, int *bad) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nr; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = r0 + k;
        uint64_t su, sd = 0;
        if (model == HPHI_SPIN_HALF_GC) {
            su = (uint64_t)r;
        } else if (model == HPHI_SPIN_HALF) {
            su = tsp_state(up, (uint64_t)r);
        } else {
            su = tsp_state(up, (uint64_t)(r / ddn));
            sd = tsp_state(dn, (uint64_t)(r % ddn));
        }
        int n = 0;
        int64_t *c = cols + k * stride;
        int8_t *g = signs + k * stride;
        int32_t *t = tids + k * stride;
        for (int q = 0; q < nt; q++) {
            const hphi_term T = terms[q];
            const uint64_t m = (1ull << T.i) | (1ull << T.j);
            if (T.kind == HPHI_EXCHANGE || T.kind == HPHI_XXZ) {
                const double jxy = T.kind == HPHI_EXCHANGE ? T.v0 : T.v1;
                if (jxy == 0.0 || __popcll(su & m) != 1) continue;
                const uint64_t s2 = su ^ m;
                const int64_t col = model == HPHI_SPIN_HALF_GC ? (int64_t)s2 : tsp_rank(up, s2);
                if (col < 0) atomicExch(bad, 1);
                c[n] = col;
                g[n] = 1;
                t[n] = q;
                n++;
            } else if (T.kind == HPHI_HOP) {
                if (T.v0 == 0.0) continue;
                const int lo = T.i < T.j ? T.i : T.j, hi = T.i < T.j ? T.j : T.i;
                // occupied sites strictly between the ends
                const uint64_t between = ((1ull << hi) - 1) & ~((2ull << lo) - 1);
                for (int sp = 0; sp < 2; sp++) {
                    if (T.spin != -1 && T.spin != sp) continue;
                    const uint64_t s = sp ? sd : su;
                    if (__popcll(s & m) != 1) continue;
                    const uint64_t s2 = s ^ m;
                    const int64_t a = sp ? tsp_rank(up, su) : tsp_rank(up, s2);
                    const int64_t b = sp ? tsp_rank(dn, s2) : tsp_rank(dn, sd);
                    if (a < 0 || b < 0) atomicExch(bad, 1);
                    c[n] = a * ddn + b;
                    g[n] = (__popcll(s & between) & 1) ? -1 : 1;
                    t[n] = q;
                    n++;
                }
            }
        }
        cnt[k] = n;
    }
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

extern "C" int hphi_dump_pattern_merged(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1,
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

extern "C" int hphi_dump_pattern(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1, int64_t *rows_out,
                                 int64_t *cols_out, int8_t *signs_out, int32_t *term_ids_out, int64_t *count) {
    if (!ctx || !ham || !count) return HPHI_E_INVAL;
    ctx->err.clear();
    if (row0 < 0 || row1 > ham->D || row0 >= row1) return set_err(ctx, HPHI_E_INVAL, "bad row range");
    if (row1 - row0 > (1 << 22)) return set_err(ctx, HPHI_E_INVAL, "at most 2^22 rows per dump");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    const hphi_basis *b = ham->basis;
    const int nt = (int)ham->terms.size();
    const int stride = nt > 0 ? 2 * nt : 1;
    auto sp_of = [&](const Species &s) {
        return TermSp{s.ja, s.jb, s.jbp, s.loff, s.lstate, s.N, s.n, s.nlo, s.nhi};
    };
    const TermSp up = b->model == HPHI_SPIN_HALF_GC ? TermSp{} : sp_of(b->sp[0]);
    const TermSp dn = b->model == HPHI_HUBBARD ? sp_of(b->sp[1]) : TermSp{};
    const int64_t ddn = b->model == HPHI_HUBBARD ? b->sp[1].dim : 1;
    // rows in chunks of at most 2^24 entry slots
    const int64_t total = row1 - row0;
    int64_t chunk = ((int64_t)1 << 24) / stride;
    if (chunk < 1) chunk = 1;
    if (chunk > total) chunk = total;
    hphi_term *dterm = nullptr;
    int64_t *dc = nullptr;
    int8_t *dg = nullptr;
    int32_t *dt = nullptr, *dn_ = nullptr;
    int *dbad = nullptr;
    const size_t slots = (size_t)chunk * stride;
    if (cudaMalloc(&dterm, sizeof(hphi_term) * (nt > 0 ? nt : 1)) != cudaSuccess ||
        cudaMalloc(&dc, slots * 8) != cudaSuccess || cudaMalloc(&dg, slots) != cudaSuccess ||
        cudaMalloc(&dt, slots * 4) != cudaSuccess || cudaMalloc(&dn_, (size_t)chunk * 4) != cudaSuccess ||
        cudaMalloc(&dbad, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dterm);
        cudaFree(dc);
        cudaFree(dg);
        cudaFree(dt);
        cudaFree(dn_);
        return set_err(ctx, HPHI_E_NOMEM, "pattern buffers");
    }
    std::vector<int64_t> hc(slots);
    std::vector<int8_t> hg(slots);
    std::vector<int32_t> ht(slots), hn(chunk);
    const int64_t cap = *count;
    const bool write = rows_out && cols_out && signs_out && term_ids_out;
    int64_t pos = 0;
    int bad = 0;
    cudaError_t e = cudaSuccess;
    if (nt > 0) e = cudaMemcpy(dterm, ham->terms.data(), sizeof(hphi_term) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(int), ctx->stream);
    for (int64_t r0 = row0; r0 < row1 && e == cudaSuccess; r0 += chunk) {
        const int64_t nr = (row1 - r0) < chunk ? (row1 - r0) : chunk;
        const int grid = (int)((nr + 255) / 256 < 4096 ? (nr + 255) / 256 : 4096);
        k_dump_terms<<<grid, 256, 0, ctx->stream>>>(b->model, up, dn, ddn, dterm, nt, r0, nr, stride, dc, dg, dt,
                                                     dn_, dbad);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpy(hn.data(), dn_, (size_t)nr * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && write) {
            const size_t ns = (size_t)nr * stride;
            e = cudaMemcpy(hc.data(), dc, ns * 8, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(hg.data(), dg, ns, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(ht.data(), dt, ns * 4, cudaMemcpyDeviceToHost);
        }
        if (e != cudaSuccess) break;
        for (int64_t k = 0; k < nr; k++) {
            const int n = hn[k];
            if (n < 0 || n > stride) {
                bad = 2;
                break;
            }
            if (write && pos + n <= cap) {
                for (int u = 0; u < n; u++) {
                    rows_out[pos + u] = r0 + k;
                    cols_out[pos + u] = hc[k * stride + u];
                    signs_out[pos + u] = hg[k * stride + u];
                    term_ids_out[pos + u] = ht[k * stride + u];
                }
            }
            pos += n;
        }
        if (bad) break;
    }
    if (e == cudaSuccess && !bad) {
        int fl = 0;
        e = cudaMemcpy(&fl, dbad, sizeof(int), cudaMemcpyDeviceToHost);
        if (fl) bad = 1;
    }
    cudaFree(dterm);
    cudaFree(dc);
    cudaFree(dg);
    cudaFree(dt);
    cudaFree(dn_);
    cudaFree(dbad);
    if (e != cudaSuccess) return cuda_err(ctx, e, "pattern export");
    if (bad) return set_err(ctx, HPHI_E_DEVICE_CHECK, "pattern export: a target state outside the sector");
    if (!write || pos > cap) {
        *count = pos;
        return set_err(ctx, HPHI_E_INVAL, "pattern needs %lld entries", (long long)pos);
    }
    *count = pos;
    return HPHI_OK;
}
