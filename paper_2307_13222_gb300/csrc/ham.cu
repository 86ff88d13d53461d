// Term compiler: interaction list -> per-sector tables of the H*x kernel.
//
// Spin models (Sec. 3.1.1 Heisenberg example, XXZ generalisation): repeated
// pairs are summed; each bond (i, j) contributes Jz/4 (+1 parallel, -1
// antiparallel) to the diagonal, written as C0 + sum_b (-Jz_b/2)[s_i != s_j]
// with C0 = sum_b Jz_b/4, and Jxy/2 between s and s ^ (bit i | bit j) when the
// spins differ.  Bonds are classified by where their sites fall in the split
// of the spin string into low (N_lo) and high halves: low-low bonds become the
// per-low-half ELL tables, high-high bonds are resolved per block, mixed bonds
// use the per-low-half flip tables.
//
// Hubbard (Sec. 3.4 H_quench, Sec. 5 Eq. ham_general): hops -t between the
// same-spin orbitals of sites i and j, with the fermion sign
// (-1)^(# same-spin fermions strictly between i and j) of the ordering
// prod_{i asc} c^+_{i up} prod_{i asc} c^+_{i dn}; the down-string hop matrix
// is tabulated per down string (ELL), the up-string one per up string;
// U n_up n_dn and V n_i n_j go to the diagonal.
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "hphi_internal.cuh"

namespace hphi {

namespace {

struct LLBond {
    int i, j, ci;  // low bits, coefficient index
    double cz;     // -Jz/2
    double cxy;
};

__global__ void k_ja16(const uint32_t *ja, int64_t n, uint16_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint16_t)ja[i];
}

// Packs ELL entries as target | coefficient index << 24 when both fit.
__global__ void k_pack_ll(const uint32_t *tgt, const uint16_t *cf, int64_t n, uint32_t *pk) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pk[i] = (tgt[i] & 0xFFFFFFu) | ((uint32_t)cf[i] << 24);
}

__global__ void k_spin_tables(int sector, const uint32_t *lstate, const uint32_t *ja, int64_t L, double c0,
                              const LLBond *ll, int nll, const int *lowbits, int nlb, double *dlow_d, float *dlow_f,
                              uint8_t *cnt, uint32_t *tgt, uint16_t *cf, uint32_t *flipq) {
    for (int64_t cp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cp < L; cp += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = sector ? lstate[cp] : (uint32_t)cp;
        double d = c0;
        int c = 0;
        for (int k = 0; k < nll; k++) {
            uint32_t bi = (l >> ll[k].i) & 1u, bj = (l >> ll[k].j) & 1u;
            if (bi != bj) {
                d += ll[k].cz;
                if (ll[k].cxy != 0.0) {
                    uint32_t l2 = l ^ ((1u << ll[k].i) | (1u << ll[k].j));
                    tgt[(int64_t)c * L + cp] = sector ? ja[l2] : l2;
                    cf[(int64_t)c * L + cp] = (uint16_t)ll[k].ci;
                    c++;
                }
            }
        }
        cnt[cp] = (uint8_t)c;
        dlow_d[cp] = d;
        dlow_f[cp] = (float)d;
        for (int b = 0; b < nlb; b++) {
            uint32_t l2 = l ^ (1u << lowbits[b]);
            flipq[(int64_t)b * L + cp] = sector ? ja[l2] : l2;
        }
    }
}

struct HopPair {
    int i, j, ci;  // sites, coefficient index base (ci: sign +, ci+1: sign -)
};

// Tables of one Hubbard species: diagonal part of that string alone (V terms),
// and the ELL hop list over its states.
__global__ void k_hub_tables(const uint32_t *states, int64_t dim, const uint32_t *ja, const uint64_t *jb, int nlo,
                             const HopPair *hops, int nhop, const VTerm *vt, int nv, double *diag, float *diag_f,
                             uint8_t *cnt, uint32_t *tgt, uint16_t *cf) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = states[r];
        double d = 0.0;
        for (int k = 0; k < nv; k++) d += vt[k].v * (double)(((s >> vt[k].i) & 1u) * ((s >> vt[k].j) & 1u));
        diag[r] = d;
        if (diag_f) diag_f[r] = (float)d;
        int c = 0;
        for (int k = 0; k < nhop; k++) {
            int i = hops[k].i, j = hops[k].j;
            if (((s >> i) & 1u) == ((s >> j) & 1u)) continue;
            uint32_t s2 = s ^ ((1u << i) | (1u << j));
            int lo = i < j ? i : j, hi = i < j ? j : i;
            uint32_t between = (hi - lo > 1) ? (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u)) : 0u;
            int sign = __popc(s & between) & 1;
            uint64_t r2 = jb[s2 >> nlo] + ja[s2 & ((1u << nlo) - 1u)];
            tgt[(int64_t)c * dim + r] = (uint32_t)r2;
            cf[(int64_t)c * dim + r] = (uint16_t)(hops[k].ci + sign);
            c++;
        }
        cnt[r] = (uint8_t)c;
    }
}

template <typename T>
int dev_alloc(hphi_ctx *ctx, T **p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(ctx, HPHI_E_NOMEM, "hamiltonian tables: cudaMalloc(%zu) failed", n * sizeof(T));
    }
    return HPHI_OK;
}

template <typename T>
int to_dev(hphi_ctx *ctx, T **p, const std::vector<T> &h) {
    int st = dev_alloc(ctx, p, h.size());
    if (st) return st;
    if (!h.empty()) HPHI_CUDA(ctx, cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HPHI_OK;
}

void free_ham(hphi_ham *h) {
    if (!h) return;
    cudaFree(h->desc);
    cudaFree(h->dlow_d);
    cudaFree(h->dlow_f);
    cudaFree(h->ll_cnt);
    cudaFree(h->ll_tgt);
    cudaFree(h->ll_cf);
    cudaFree(h->flipq);
    cudaFree(h->up_cnt);
    cudaFree(h->up_tgt);
    cudaFree(h->up_cf);
    cudaFree(h->aup);
    cudaFree(h->ll_pk);
    cudaFree(h->ja16);
    cudaFree(h->ph_ent);
    cudaFree(h->ph_off);
    cudaFree(h->dterms_d);
    cudaFree(h->rowstate);
    cudaFree(h->seg_so);
    for (int p = 0; p < 2; p++) {
        cudaFree(h->tile_tab[p]);
        cudaFree(h->tile_diag[p]);
        delete h->tile[p];
    }
    delete h->seg;
    delete h;
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

// Per-class bond lists of the bond-major H*x kernel (S^z sector, N_lo <= 16).
// Low halves of popcount p, in ascending order, have class positions
// q = 0 .. C(N_lo, p) - 1 (Lin's ja).  For every class p:
//   low-low bond k = (i, j) with Jxy != 0: the q whose bits i, j differ, each
//     with q' = position of l ^ (2^i | 2^j) (same class);
//   low bit b of a mixed bond, need in {0, 1}: the q with bit b = need, each
//     with r = position of l ^ 2^b (class p - 1 if need = 1, else p + 1).
// Entries q | q' << 16 in ascending q.  Each group also gets the offsets of
// the kPhRanges + 1 boundaries q_r = len * r / kPhRanges, so that the warp that
// owns rows [q_r, q_r') of a block finds its entries without searching.
int build_bond_lists(hphi_ctx *ctx, hphi_ham *H, const std::vector<LLBond> &ll, const std::vector<int> &lowbits) {
    const int nlo = H->nlo, nll = (int)ll.size(), nlb = (int)lowbits.size();
    std::vector<std::vector<uint32_t>> cls(nlo + 1);
    std::vector<uint32_t> pos((size_t)1 << nlo);
    for (uint32_t l = 0; l < (1u << nlo); l++) {
        std::vector<uint32_t> &c = cls[__builtin_popcount(l)];
        pos[l] = (uint32_t)c.size();
        c.push_back(l);
    }
    std::vector<uint32_t> ent;
    std::vector<int32_t> off;
    auto close_group = [&](size_t start, uint32_t len) {
        size_t i = start;
        for (int r = 0; r <= kPhRanges; r++) {
            const uint32_t qb = (uint32_t)(((uint64_t)len * r) / kPhRanges);
            while (i < ent.size() && (ent[i] & 0xFFFFu) < qb) i++;
            off.push_back((int32_t)i);
        }
    };
    for (int p = 0; p <= nlo; p++) {
        const std::vector<uint32_t> &c = cls[p];
        for (int k = 0; k < nll; k++) {
            const size_t start = ent.size();
            const uint32_t m = (1u << ll[k].i) | (1u << ll[k].j);
            if (ll[k].cxy != 0.0)
                for (uint32_t q = 0; q < c.size(); q++) {
                    const uint32_t lm = c[q] & m;
                    if (lm != 0 && lm != m) ent.push_back(q | pos[c[q] ^ m] << 16);
                }
            close_group(start, (uint32_t)c.size());
        }
    }
    H->ph_mx0 = (int64_t)off.size();
    for (int p = 0; p <= nlo; p++) {
        const std::vector<uint32_t> &c = cls[p];
        for (int bi = 0; bi < nlb; bi++)
            for (uint32_t need = 0; need < 2; need++) {
                const size_t start = ent.size();
                const int b = lowbits[bi];
                for (uint32_t q = 0; q < c.size(); q++)
                    if (((c[q] >> b) & 1u) == need) ent.push_back(q | pos[c[q] ^ (1u << b)] << 16);
                close_group(start, (uint32_t)c.size());
            }
    }
    if (ent.size() >= ((size_t)1 << 31)) return HPHI_OK;  // lists unavailable: the kernel is not offered
    int st;
    if ((st = to_dev(ctx, &H->ph_ent, ent)) || (st = to_dev(ctx, &H->ph_off, off))) return st;
    return HPHI_OK;
}

int build_spin(hphi_ctx *ctx, hphi_ham *H, const hphi_term *terms, int n_terms) {
    const hphi_basis *B = H->basis;
    const int N = B->N;
    const bool sector = B->model == HPHI_SPIN_HALF;
    std::map<std::pair<int, int>, std::pair<double, double>> pairs;  // (i<j) -> (Jz, Jxy)
    for (int k = 0; k < n_terms; k++) {
        const hphi_term &t = terms[k];
        if (t.kind != HPHI_EXCHANGE && t.kind != HPHI_XXZ)
            return set_err(ctx, HPHI_E_INVAL, "term %d: kind %d is not a spin term", k, t.kind);
        if (t.i < 0 || t.i >= N || t.j < 0 || t.j >= N || t.i == t.j)
            return set_err(ctx, HPHI_E_INVAL, "term %d: bad sites (%d, %d) for %d sites", k, t.i, t.j, N);
        auto key = std::make_pair(t.i < t.j ? t.i : t.j, t.i < t.j ? t.j : t.i);
        auto &v = pairs[key];
        v.first += t.v0;
        v.second += t.kind == HPHI_EXCHANGE ? t.v0 : t.v1;
    }
    const int nlo = N - N / 2;
    HamDesc &D = H->host;
    D.model = B->model;
    D.N = N;
    D.nlo = nlo;
    D.nhi = N / 2;
    D.n = sector ? B->nup : -1;
    D.ddn = 0;
    double c0 = 0.0;
    std::vector<LLBond> ll;
    std::vector<int> lowbits;
    std::map<int, int> lowbit_row;
    int nhh = 0, nlh = 0, ncoef = 0;
    for (auto &kv : pairs) {
        int i = kv.first.first, j = kv.first.second;
        double Jz = kv.second.first, Jxy = kv.second.second;
        H->dterms.push_back(DTerm{DT_SPIN, i, j, 0, Jz, Jxy});
        c0 += 0.25 * Jz;
        if (j < nlo) {
            if (ncoef >= kMaxCoef) return set_err(ctx, HPHI_E_INVAL, "too many low-low bonds");
            D.coef[ncoef] = 0.5 * Jxy;
            ll.push_back(LLBond{i, j, ncoef, -0.5 * Jz, 0.5 * Jxy});
            ncoef++;
        } else if (i >= nlo) {
            if (nhh >= kMaxHH) return set_err(ctx, HPHI_E_INVAL, "too many high-high bonds (max %d)", kMaxHH);
            D.hh[nhh++] = HHBond{i - nlo, j - nlo, -0.5 * Jz, 0.5 * Jxy};
        } else {
            if (nlh >= kMaxLH) return set_err(ctx, HPHI_E_INVAL, "too many mixed bonds (max %d)", kMaxLH);
            int b = i, a = j - nlo;
            int bi = 0;
            if (Jxy != 0.0) {
                auto it = lowbit_row.find(b);
                if (it == lowbit_row.end()) {
                    bi = (int)lowbits.size();
                    lowbit_row[b] = bi;
                    lowbits.push_back(b);
                } else {
                    bi = it->second;
                }
            }
            D.lh[nlh++] = LHBond{a, b, bi, -0.5 * Jz, 0.5 * Jxy};
        }
    }
    if ((int)ll.size() > 255) return set_err(ctx, HPHI_E_INVAL, "too many low-low bonds (max 255)");
    if ((int)ll.size() > kMaxBond) return set_err(ctx, HPHI_E_INVAL, "too many low-low bonds (max %d)", kMaxBond);
    for (size_t k = 0; k < ll.size(); k++) D.ll[k] = LLBondD{ll[k].i, ll[k].j, ll[k].cz, ll[k].cxy};
    D.n_ll = (int)ll.size();
    D.n_hh = nhh;
    D.n_lh = nlh;
    D.n_ncoef = ncoef;
    D.n_v = 0;
    D.ngroups = nlh > 0 ? (nlo + 7) / 8 : 0;
    H->nlo = nlo;
    H->nh = (int64_t)1 << (N / 2);
    H->L = (int64_t)1 << nlo;
    H->ll_w = (int)ll.size();
    H->nlb = (int)lowbits.size();
    H->max_row_entries = 1 + nhh + (int)ll.size() + nlh;
    const int64_t L = H->L;
    int st;
    if ((st = dev_alloc(ctx, &H->dlow_d, L)) || (st = dev_alloc(ctx, &H->dlow_f, L)) ||
        (st = dev_alloc(ctx, &H->ll_cnt, L)) || (st = dev_alloc(ctx, &H->ll_tgt, (size_t)L * H->ll_w)) ||
        (st = dev_alloc(ctx, &H->ll_cf, (size_t)L * H->ll_w)) || (st = dev_alloc(ctx, &H->flipq, (size_t)L * H->nlb)))
        return st;
    LLBond *d_ll = nullptr;
    int *d_lb = nullptr;
    if ((st = to_dev(ctx, &d_ll, ll)) || (st = to_dev(ctx, &d_lb, lowbits))) {
        cudaFree(d_ll);
        return st;
    }
    k_spin_tables<<<grid_of(L), 256, 0, ctx->stream>>>(sector ? 1 : 0, B->sp[0].lstate, B->sp[0].ja, L, c0, d_ll,
                                                       (int)ll.size(), d_lb, H->nlb, H->dlow_d, H->dlow_f, H->ll_cnt,
                                                       H->ll_tgt, H->ll_cf, H->flipq);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_ll);
    cudaFree(d_lb);
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_spin_tables");
    if (sector && nlo <= 16 && ll.size() <= 128 && (st = build_bond_lists(ctx, H, ll, lowbits))) return st;
    if (sector && (st = build_seg_tables(ctx, H))) return st;
    return HPHI_OK;
}

// Down-hop lists of the bond-major H*x kernel for Hubbard models (row block =
// the D_dn rows of one up string): group g = coefficient index (a down hop
// pair with one fermion sign), entries q | q' << 16 for the down states q that
// hop to q' with that coefficient, ascending in q, with the segment starts of
// kPhRanges row ranges as in the spin lists.  Built from the ELL tables; not
// built when D_dn >= 2^16 or there are more than 128 coefficients.
int build_hub_lists(hphi_ctx *ctx, hphi_ham *H) {
    const int64_t L = H->L;
    const int w = H->ll_w, nc = H->host.n_ncoef;
    if (L >= 65536 || nc > 128 || w == 0) return HPHI_OK;
    std::vector<uint8_t> cnt((size_t)L);
    std::vector<uint32_t> tgt((size_t)L * w);
    std::vector<uint16_t> cf((size_t)L * w);
    HPHI_CUDA(ctx, cudaMemcpy(cnt.data(), H->ll_cnt, cnt.size(), cudaMemcpyDeviceToHost));
    HPHI_CUDA(ctx, cudaMemcpy(tgt.data(), H->ll_tgt, tgt.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    HPHI_CUDA(ctx, cudaMemcpy(cf.data(), H->ll_cf, cf.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    std::vector<std::vector<uint32_t>> grp(nc);
    for (int64_t q = 0; q < L; q++)
        for (int e = 0; e < cnt[q]; e++) {
            const size_t o = (size_t)e * L + q;
            if (cf[o] < nc) grp[cf[o]].push_back((uint32_t)q | tgt[o] << 16);
        }
    std::vector<uint32_t> ent;
    std::vector<int32_t> off;
    for (int g = 0; g < nc; g++) {
        size_t i = 0;
        for (int r = 0; r < kPhRanges; r++) {
            const uint32_t qe = (uint32_t)(((uint64_t)L * (uint32_t)(r + 1)) / kPhRanges);
            off.push_back((int32_t)ent.size());
            while (i < grp[g].size() && (grp[g][i] & 0xFFFFu) < qe) ent.push_back(grp[g][i++]);
        }
        off.push_back((int32_t)ent.size());
    }
    H->ph_mx0 = (int64_t)off.size();
    int st;
    if ((st = to_dev(ctx, &H->ph_ent, ent)) || (st = to_dev(ctx, &H->ph_off, off))) return st;
    return HPHI_OK;
}

int build_hubbard(hphi_ctx *ctx, hphi_ham *H, const hphi_term *terms, int n_terms) {
    const hphi_basis *B = H->basis;
    const int N = B->N;
    std::map<std::tuple<int, int, int>, double> hops;  // (species, i<j) -> t
    std::map<std::pair<int, int>, double> vpairs;
    std::vector<double> U(N, 0.0);
    for (int k = 0; k < n_terms; k++) {
        const hphi_term &t = terms[k];
        if (t.i < 0 || t.i >= N) return set_err(ctx, HPHI_E_INVAL, "term %d: site %d out of range", k, t.i);
        if (t.kind == HPHI_HOP) {
            if (t.j < 0 || t.j >= N || t.j == t.i)
                return set_err(ctx, HPHI_E_INVAL, "term %d: bad sites (%d, %d)", k, t.i, t.j);
            if (t.spin < -1 || t.spin > 1) return set_err(ctx, HPHI_E_INVAL, "term %d: spin must be -1, 0 or 1", k);
            int a = t.i < t.j ? t.i : t.j, b = t.i < t.j ? t.j : t.i;
            for (int s = 0; s < 2; s++)
                if (t.spin == -1 || t.spin == s) hops[std::make_tuple(s, a, b)] += t.v0;
        } else if (t.kind == HPHI_HUBBARD_U) {
            U[t.i] += t.v0;
        } else if (t.kind == HPHI_DENS_DENS) {
            if (t.j < 0 || t.j >= N || t.j == t.i)
                return set_err(ctx, HPHI_E_INVAL, "term %d: bad sites (%d, %d)", k, t.i, t.j);
            vpairs[std::make_pair(t.i < t.j ? t.i : t.j, t.i < t.j ? t.j : t.i)] += t.v0;
        } else {
            return set_err(ctx, HPHI_E_INVAL, "term %d: kind %d is not a Hubbard term", k, t.kind);
        }
    }
    HamDesc &D = H->host;
    D.model = HPHI_HUBBARD;
    D.n_ll = 0;
    D.N = N;
    D.nlo = N;
    D.nhi = 0;
    D.n = -1;
    D.n_hh = 0;
    D.n_lh = 0;
    D.ddn = B->sp[1].dim;
    std::vector<HopPair> hp[2];
    int ncoef = 0;
    for (int i = 0; i < N; i++)
        if (U[i] != 0.0) H->dterms.push_back(DTerm{DT_U, i, i, 0, U[i], 0.0});
    for (auto &kv : vpairs) H->dterms.push_back(DTerm{DT_V, kv.first.first, kv.first.second, 0, kv.second, 0.0});
    for (auto &kv : hops) {
        if (kv.second == 0.0) continue;
        int s = std::get<0>(kv.first);
        H->dterms.push_back(DTerm{DT_HOP, std::get<1>(kv.first), std::get<2>(kv.first), s, kv.second, 0.0});
        if (ncoef + 2 > kMaxCoef) return set_err(ctx, HPHI_E_INVAL, "too many hopping pairs");
        D.coef[ncoef] = -kv.second;     // sign +: -t
        D.coef[ncoef + 1] = kv.second;  // sign -: +t
        hp[s].push_back(HopPair{std::get<1>(kv.first), std::get<2>(kv.first), ncoef});
        ncoef += 2;
    }
    if ((int)hp[0].size() > kMaxHH || (int)hp[1].size() > 255)
        return set_err(ctx, HPHI_E_INVAL, "too many hopping pairs per species");
    D.n_ncoef = ncoef;
    std::vector<VTerm> vt;
    for (auto &kv : vpairs) vt.push_back(VTerm{kv.first.first, kv.first.second, kv.second});
    if ((int)vt.size() > kMaxBond) return set_err(ctx, HPHI_E_INVAL, "too many V terms");
    for (size_t k = 0; k < vt.size(); k++) D.v[k] = vt[k];
    D.n_v = (int)vt.size();
    bool anyU = false;
    for (int i = 0; i < 64; i++) D.U[i] = i < N ? U[i] : 0.0;
    for (int i = 0; i < N; i++) anyU = anyU || U[i] != 0.0;
    D.ngroups = (anyU || !vt.empty()) ? (N + 7) / 8 : 0;
    H->nlo = N;
    H->nh = B->sp[0].dim;
    H->L = B->sp[1].dim;
    H->ll_w = (int)hp[1].size();
    H->up_w = (int)hp[0].size();
    H->nlb = 0;
    H->max_row_entries = 1 + H->up_w + H->ll_w;
    int st;
    HopPair *d_h0 = nullptr, *d_h1 = nullptr;
    VTerm *d_v = nullptr;
    if ((st = dev_alloc(ctx, &H->dlow_d, H->L)) || (st = dev_alloc(ctx, &H->dlow_f, H->L)) ||
        (st = dev_alloc(ctx, &H->ll_cnt, H->L)) || (st = dev_alloc(ctx, &H->ll_tgt, (size_t)H->L * H->ll_w)) ||
        (st = dev_alloc(ctx, &H->ll_cf, (size_t)H->L * H->ll_w)) || (st = dev_alloc(ctx, &H->up_cnt, H->nh)) ||
        (st = dev_alloc(ctx, &H->up_tgt, (size_t)H->nh * H->up_w)) ||
        (st = dev_alloc(ctx, &H->up_cf, (size_t)H->nh * H->up_w)) || (st = dev_alloc(ctx, &H->aup, H->nh)) ||
        (st = dev_alloc(ctx, &H->flipq, 1)))
        return st;
    if ((st = to_dev(ctx, &d_h0, hp[0])) || (st = to_dev(ctx, &d_h1, hp[1])) || (st = to_dev(ctx, &d_v, vt))) {
        cudaFree(d_h0);
        cudaFree(d_h1);
        return st;
    }
    const Species &su = B->sp[0], &sd = B->sp[1];
    k_hub_tables<<<grid_of(sd.dim), 256, 0, ctx->stream>>>(sd.states, sd.dim, sd.ja, sd.jb, sd.nlo, d_h1,
                                                           (int)hp[1].size(), d_v, (int)vt.size(), H->dlow_d,
                                                           H->dlow_f, H->ll_cnt, H->ll_tgt, H->ll_cf);
    k_hub_tables<<<grid_of(su.dim), 256, 0, ctx->stream>>>(su.states, su.dim, su.ja, su.jb, su.nlo, d_h0,
                                                           (int)hp[0].size(), d_v, (int)vt.size(), H->aup, nullptr,
                                                           H->up_cnt, H->up_tgt, H->up_cf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_h0);
    cudaFree(d_h1);
    cudaFree(d_v);
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_hub_tables");
    return build_hub_lists(ctx, H);
}

}  // namespace

}  // namespace hphi

using namespace hphi;

extern "C" int hphi_build_hamiltonian(hphi_ctx *ctx, const hphi_basis *basis, const hphi_term *terms, int n_terms,
                                      hphi_ham **out) {
    if (!ctx || !basis || !out || n_terms < 0 || (n_terms > 0 && !terms)) return HPHI_E_INVAL;
    *out = nullptr;
    ctx->err.clear();
    if (basis->device != ctx->device) return set_err(ctx, HPHI_E_INVAL, "basis belongs to another device");
    HPHI_CUDA(ctx, cudaSetDevice(ctx->device));
    hphi_ham *H = new (std::nothrow) hphi_ham();
    if (!H) return set_err(ctx, HPHI_E_NOMEM, "host allocation failed");
    H->basis = basis;
    H->model = basis->model;
    H->device = ctx->device;
    H->D = basis->D;
    int st = basis->model == HPHI_HUBBARD ? build_hubbard(ctx, H, terms, n_terms) : build_spin(ctx, H, terms, n_terms);
    if (!st && n_terms > 0) H->terms.assign(terms, terms + n_terms);
    if (!st) {
        st = dev_alloc(ctx, &H->desc, 1);
        if (!st) {
            cudaError_t e = cudaMemcpy(H->desc, &H->host, sizeof(HamDesc), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_err(ctx, e, "descriptor copy");
        }
    }
    if (!st) {
        st = dev_alloc(ctx, &H->dterms_d, H->dterms.size() > 0 ? H->dterms.size() : 1);
        if (!st && !H->dterms.empty()) {
            cudaError_t e = cudaMemcpy(H->dterms_d, H->dterms.data(), sizeof(DTerm) * H->dterms.size(),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_err(ctx, e, "term list copy");
        }
    }
    // 16-bit copy of Lin's ja for the on-the-fly ranks of the H*x kernel
    if (!st && basis->model == HPHI_SPIN_HALF && basis->sp[0].nlo <= 16) {
        const size_t n = (size_t)1 << basis->sp[0].nlo;
        st = dev_alloc(ctx, &H->ja16, n);
        if (!st) {
            k_ja16<<<grid_of((int64_t)n), 256, 0, ctx->stream>>>(basis->sp[0].ja, (int64_t)n, H->ja16);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) st = cuda_err(ctx, e, "k_ja16");
        }
    }
    // packed low-low lists: target < 2^24 and coefficient index < 256
    if (!st && H->ll_w > 0 && H->L < (1 << 24) && H->host.n_ncoef <= 256) {
        const size_t n = (size_t)H->L * H->ll_w;
        st = dev_alloc(ctx, &H->ll_pk, n);
        if (!st) {
            k_pack_ll<<<grid_of((int64_t)n), 256, 0, ctx->stream>>>(H->ll_tgt, H->ll_cf, (int64_t)n, H->ll_pk);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) st = cuda_err(ctx, e, "k_pack_ll");
        }
    }
    if (st) {
        free_ham(H);
        return st;
    }
    *out = H;
    return HPHI_OK;
}

extern "C" void hphi_ham_destroy(hphi_ham *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    free_ham(h);
}

extern "C" int64_t hphi_ham_dim(const hphi_ham *h) { return h ? h->D : -1; }
