// Row enumeration of H shared by the H*x kernel and the pattern dump.
//
// A thread block owns one block h of rows at a time.  setup_block() fills a
// shared-memory HBlock with everything that depends on h only; visit_row()
// then enumerates, for row q of the block, the diagonal element and every
// off-diagonal (target row, coefficient) pair, calling a visitor.  Terms:
//   spin: diagonal  C0 + sum_b (-Jz_b/2) [s_i != s_j]
//         off-diag  Jxy_b/2 to s ^ (bit i | bit j) when s_i != s_j
//   Hubbard: diagonal sum_i U_i n_iu n_id + sum V_ij n_i n_j
//         off-diag  -t (-1)^(# same-spin fermions strictly between i and j)
// (Sec. 3.1.1, Sec. 3.4 H_quench, Sec. 5 Eq. ham_general; the sign follows
// the ordering prod c^+_{up} prod c^+_{dn} of the basis convention.)
#pragma once

#include "hphi_internal.cuh"

namespace hphi {

struct HvTables {
    const HamDesc *desc;
    int model;
    int nlo, ngroups, n;
    int64_t nh, L, ddn;
    // spin species tables
    const uint64_t *jb;
    const uint32_t *loff;
    const uint32_t *lstate;
    // Hubbard species states
    const uint32_t *states_up;
    const uint32_t *states_dn;
    // per-class-position tables
    const void *dlow;        // double or float, [L]
    const uint8_t *ll_cnt;
    const uint32_t *ll_tgt;  // [ll_w][L]
    const uint16_t *ll_cf;
    const uint32_t *flipq;   // [nlb][L]
    // Hubbard up tables, [up_w][nh]
    const uint8_t *up_cnt;
    const uint32_t *up_tgt;
    const uint16_t *up_cf;
    const double *aup;
    // packed low-low lists (target | coefficient index << 24), null if unavailable
    const uint32_t *ll_pk;
    // traversal of the row blocks: counter bit k -> bit hperm[k] of h; bits of
    // h in outer_mask are outside the L2-resident subcube of the traversal
    int use_perm;
    uint32_t outer_mask;
    uint8_t hperm[32];
    int split;   // thread blocks sharing one row block
    int hints;   // L2 eviction-priority hints on
    const uint16_t *ja16;  // Lin's ja (16-bit), spin sector
    const uint32_t *ph_ent;  // bond-major kernel: per-class bond lists, null if unavailable
    const int32_t *ph_off;
    int64_t ph_mx0;
    int ph_nlb;              // low bits of the mixed bonds (list groups per class: 2 ph_nlb)
};

// Row block visited at traversal position c.
__device__ __forceinline__ int64_t block_of(const HvTables &P, int64_t c) {
    if (!P.use_perm) return c;
    int64_t h = 0;
    for (int k = 0; k < 32 && (c >> k) != 0; k++) h |= ((c >> k) & 1) << P.hperm[k];
    return h;
}

template <typename T>
struct HBlock {
    int64_t base;
    uint32_t cp0, len;
    int valid, nhh, nlh;
    T dh;
    uint64_t hbits;
    double dh_part[2];
    int64_t hh_delta[kMaxHH];
    T hh_coef[kMaxHH];
    int64_t lh_base[kMaxLH];
    T lh_coef[kMaxLH];
    uint16_t lh_bi[kMaxLH];
    uint8_t lh_b[kMaxLH], lh_need[kMaxLH];
    uint8_t hh_outer[kMaxHH], lh_outer[kMaxLH];  // target block outside the resident subcube
    double w[kMaxGroups * 8];
    T tab[kMaxGroups][256];
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Block set-up, shared by every kernel that walks rows block by block.  All
// threads of the thread block (>= 64 of them) must call it; it ends with
// __syncthreads().  Warp 0 resolves the high-high bonds (or the up hops) and
// warp 1 the mixed bonds, one bond per lane, compacting the off-diagonal ones
// with ballots; then the diagonal weights and byte tables are built.
template <typename T>
__device__ void setup_block(const HvTables &P, int64_t h, HBlock<T> &hb) {
    const HamDesc &D = *P.desc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const bool spin = P.model != kHubbard;
    if (warp < 2) {
        // every participating warp derives the block placement itself
        int64_t base = 0;
        uint32_t cp0 = 0, len = 0;
        int valid = 1;
        if (P.model == kSpin) {
            const uint64_t b = P.jb[h];
            valid = b != ~0ull;
            base = (int64_t)b;
            if (valid) {
                const int p = P.n - __popcll((unsigned long long)h);
                cp0 = P.loff[p];
                len = P.loff[p + 1] - cp0;
            }
        } else if (P.model == kSpinGC) {
            base = h << P.nlo;
            len = 1u << P.nlo;
        } else {
            base = h * P.ddn;
            len = (uint32_t)P.ddn;
        }
        double dpart = 0.0;
        if (warp == 0) {
            int nhh = 0;
            if (spin && valid) {
                for (int k0 = 0; k0 < D.n_hh; k0 += 32) {
                    const int k = k0 + lane;
                    bool off = false;
                    int64_t delta = 0;
                    double cxy = 0.0;
                    if (k < D.n_hh) {
                        const HHBond &bd = D.hh[k];
                        const bool differ = ((h >> bd.i) & 1) != ((h >> bd.j) & 1);
                        if (differ) {
                            dpart += bd.cz;
                            off = bd.cxy != 0.0;
                            if (off) {
                                const uint64_t h2 = (uint64_t)h ^ ((1ull << bd.i) | (1ull << bd.j));
                                delta = (P.model == kSpin ? (int64_t)P.jb[h2] : (int64_t)(h2 << P.nlo)) - base;
                                cxy = bd.cxy;
                            }
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, off);
                    const int pos = nhh + __popc(m & lt);
                    if (off && pos < kMaxHH) {
                        const HHBond &bd = D.hh[k];
                        hb.hh_delta[pos] = delta;
                        hb.hh_coef[pos] = (T)cxy;
                        hb.hh_outer[pos] = (uint8_t)((P.outer_mask >> bd.i) & 1 || (P.outer_mask >> bd.j) & 1);
                    }
                    nhh += __popc(m);
                }
            } else if (!spin) {
                const int c = P.up_cnt[h];
                for (int e = lane; e < c && e < kMaxHH; e += 32) {
                    const int64_t h2 = P.up_tgt[(int64_t)e * P.nh + h];
                    hb.hh_delta[e] = (h2 - h) * P.ddn;
                    hb.hh_coef[e] = (T)D.coef[P.up_cf[(int64_t)e * P.nh + h]];
                    hb.hh_outer[e] = 0;
                }
                nhh = c;
                if (lane == 0) dpart = P.aup[h];
            }
            dpart = warp_sum_d(dpart);
            if (lane == 0) {
                hb.nhh = nhh < kMaxHH ? nhh : kMaxHH;
                hb.dh_part[0] = dpart;
                hb.base = base;
                hb.cp0 = cp0;
                hb.len = valid ? len : 0;
                hb.valid = valid;
                hb.hbits = spin ? (uint64_t)h : (uint64_t)P.states_up[h];
            }
        } else {
            int nlh = 0;
            if (spin && valid) {
                for (int k0 = 0; k0 < D.n_lh; k0 += 32) {
                    const int k = k0 + lane;
                    bool keep = false;
                    if (k < D.n_lh) {
                        const LHBond &bd = D.lh[k];
                        const int ha = (int)((h >> bd.a) & 1);
                        dpart += bd.cz * ha;
                        keep = bd.cxy != 0.0;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    const int pos = nlh + __popc(m & lt);
                    if (keep && pos < kMaxLH) {
                        const LHBond &bd = D.lh[k];
                        const int ha = (int)((h >> bd.a) & 1);
                        const uint64_t h2 = (uint64_t)h ^ (1ull << bd.a);
                        hb.lh_base[pos] = P.model == kSpin ? (int64_t)P.jb[h2] : (int64_t)(h2 << P.nlo);
                        hb.lh_coef[pos] = (T)bd.cxy;
                        hb.lh_b[pos] = (uint8_t)bd.b;
                        hb.lh_need[pos] = (uint8_t)(1 - ha);
                        hb.lh_bi[pos] = (uint16_t)bd.bi;
                        hb.lh_outer[pos] = (uint8_t)((P.outer_mask >> bd.a) & 1);
                    }
                    nlh += __popc(m);
                }
            }
            dpart = warp_sum_d(dpart);
            if (lane == 0) {
                hb.nlh = nlh < kMaxLH ? nlh : kMaxLH;
                hb.dh_part[1] = dpart;
            }
        }
    }
    __syncthreads();
    // weights of the mixed diagonal part, one per low bit / down site:
    //   spin:    w_b = sum_{mixed bonds (a,b)} (-Jz/2) (1 - 2 h_a)
    //   Hubbard: w_j = U_j n_j,up + sum_{V terms with j} V n_other,up
    const int nbits = P.ngroups * 8;
    if ((int)threadIdx.x < nbits) {
        const int b = threadIdx.x;
        double w = 0.0;
        if (hb.valid) {
            if (spin) {
                for (int k = 0; k < D.n_lh; k++)
                    if (D.lh[k].b == b) w += D.lh[k].cz * (1 - 2 * (int)((hb.hbits >> D.lh[k].a) & 1));
            } else if (b < D.N) {
                const uint64_t su = hb.hbits;
                w = D.U[b] * (double)((su >> b) & 1);
                for (int k = 0; k < D.n_v; k++) {
                    if (D.v[k].j == b) w += D.v[k].v * (double)((su >> D.v[k].i) & 1);
                    if (D.v[k].i == b) w += D.v[k].v * (double)((su >> D.v[k].j) & 1);
                }
            }
        }
        hb.w[b] = w;
    }
    if (threadIdx.x == 32 * 2) hb.dh = (T)(hb.dh_part[0] + hb.dh_part[1]);
    __syncthreads();
    if (threadIdx.x < 256 && hb.valid) {
        for (int g = 0; g < P.ngroups; g++) {
            double s = 0.0;
            for (int k = 0; k < 8; k++)
                if ((threadIdx.x >> k) & 1) s += hb.w[8 * g + k];
            hb.tab[g][threadIdx.x] = (T)s;
        }
    }
    __syncthreads();
}

// Enumerate row q of the current block.  The visitor gets diag(row, d) first
// and then add8(t, c): up to 8 off-diagonal (target row, coefficient) pairs
// at a time (t < 0 marks an unused slot), in the order high-high (up hops),
// low-low (down hops), mixed.  Handing over 8 independent targets at once lets
// the visitor issue 8 gathers before it consumes any of them.
constexpr int kChunk = 8;

template <typename T, class V>
__device__ __forceinline__ void visit_row(const HvTables &P, const HBlock<T> &hb, const T *coef_sm, uint32_t q,
                                          V &vis) {
    const uint32_t cp = hb.cp0 + q;
    uint32_t l;
    if (P.model == kSpin) l = __ldg(P.lstate + cp);
    else if (P.model == kSpinGC) l = q;
    else l = __ldg(P.states_dn + q);
    const int cnt = __ldg(P.ll_cnt + cp);
    T d = __ldg(((const T *)P.dlow) + cp) + hb.dh;
    for (int g = 0; g < P.ngroups; g++) d += hb.tab[g][(l >> (8 * g)) & 255u];
    const int64_t row = hb.base + q;
    vis.diag(row, d);
    int64_t t[kChunk];
    T c[kChunk];
    for (int k0 = 0; k0 < hb.nhh; k0 += kChunk) {
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            const int k = k0 + u;
            const bool ok = k < hb.nhh;
            t[u] = ok ? row + hb.hh_delta[k] : -1;
            c[u] = ok ? hb.hh_coef[k] : (T)0;
        }
        vis.add8(t, c);
    }
    for (int e0 = 0; e0 < cnt; e0 += kChunk) {
        uint32_t tg[kChunk];
        uint16_t cf[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            const int e = e0 + u;
            if (e < cnt) {
                const int64_t off = (int64_t)e * P.L + cp;
                tg[u] = __ldg(P.ll_tgt + off);
                cf[u] = __ldg(P.ll_cf + off);
            }
        }
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            const bool ok = e0 + u < cnt;
            t[u] = ok ? hb.base + tg[u] : -1;
            c[u] = ok ? coef_sm[cf[u]] : (T)0;
        }
        vis.add8(t, c);
    }
    for (int k0 = 0; k0 < hb.nlh; k0 += kChunk) {
        uint32_t tq[kChunk];
        bool ok[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            const int k = k0 + u;
            ok[u] = k < hb.nlh && ((l >> hb.lh_b[k]) & 1u) == hb.lh_need[k];
            if (ok[u]) tq[u] = __ldg(P.flipq + (int64_t)hb.lh_bi[k] * P.L + cp);
        }
#pragma unroll
        for (int u = 0; u < kChunk; u++) {
            t[u] = ok[u] ? hb.lh_base[k0 + u] + tq[u] : -1;
            c[u] = ok[u] ? hb.lh_coef[k0 + u] : (T)0;
        }
        vis.add8(t, c);
    }
}

}  // namespace hphi
