// Tiled two-pass block H*V for spin-1/2 models on the full 2^N space, 32 real
// columns in FP32 or FP64 (16 complex columns: the cTPQ block of Sec. 3.5.2 and the
// real-time evolution of Sec. 3.4).
//
// Row s (an N-bit spin string) holds 32 columns, 128 (FP32) or 256 (FP64)
// contiguous bytes.  An
// exchange bond (i, j) with Jxy != 0 couples s with s ^ (2^i | 2^j) where the
// two bits differ (Sec. 3.1.1).  The single-pass kernels gather about 20 such
// rows per row from all over the 8.6 GB block and move about 6x the
// algorithmic bytes from DRAM.
//
// Here the off-diagonal bonds are split over two passes.  Pass k works on a
// bit set S_k: it walks the rows tile by tile, a tile being the 2^|S_k| rows
// that share the bits outside S_k, every thread block on the same tile at a
// time, and applies only bonds with both sites in S_k, so every gather stays
// inside the current tile, which is sized to a fraction of L2 and comes from
// DRAM once.  The sets come from the bond graph: A and B disjoint site sets
// with no bond between them, S_1 = all sites but A, S_2 = all sites but B;
// a bond touching A lies in S_2, one touching B in S_1, the rest in both
// (split for balance).  So each pass reads x once and the pair moves
//   pass 1: x, diagonal (one value per row), t written;
//   pass 2: x, t, v (the gamma term), y written
// instead of x about 17 times.
//   pass 1:  t[s] = d[s] x[s] + sum_{bonds of pass 1} c_b x[s ^ m_b]
//   pass 2:  acc = t[s] + sum_{bonds of pass 2} c_b x[s ^ m_b],
//            y = alpha acc + beta y + gamma v  (pair swap, fused reductions)
// d is the diagonal, sum_b Jz_b S^z_i S^z_j, stored once per Hamiltonian and
// precision.  t lives in y when y's old value is not read (beta = 0 and
// v != y), else in a context buffer.  Lanes: 16 bytes each (FP32: 8 per row,
// 4 rows per warp; FP64: 16 per row, 2 rows per warp), tiles sized to the row
// bytes.  Every row sums its terms in a fixed order (ascending bond index):
// deterministic.
#include "hvcommon.cuh"

#include <algorithm>
#include <vector>

namespace hphi {

namespace {

constexpr int kTileThreads = 256;
constexpr int kTileItemBits = 5;  // at most 32 rows (8 warps x 4) per thread-block iteration
constexpr int kTileUnroll = 8;    // bonds tested and gathered per batch (4: 7 % slower in FP32)
constexpr int kTileMinB1 = 4;     // thread blocks per SM the registers of pass 1 are sized for

// Lane layout of a 32-column row: every lane moves 16 bytes (E columns), LPR
// lanes per row, RPW rows per warp, 2^IB rows per thread-block iteration
// (FP64: two rows per warp; one row per warp, a lane per column, was 10 %
// slower: the FP64 pipe is busy either way).
template <typename T>
struct TileShape {
    static constexpr int E = 16 / (int)sizeof(T);
    static constexpr int LPR = 32 / E;
    static constexpr int RPW = 32 / LPR;
    static constexpr int IB = RPW == 4 ? 5 : 4;
};

__device__ __forceinline__ void ld16(const float *p, float (&v)[4]) {
    asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
}
__device__ __forceinline__ void ld16(const double *p, double (&v)[2]) {
    asm("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p));
}
__device__ __forceinline__ void ldc16(const float *p, float (&v)[4]) {  // coherent: may alias y
    asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ldc16(const double *p, double (&v)[2]) {
    asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p) : "memory");
}
__device__ __forceinline__ void st16(float *p, const float (&v)[4]) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
}
__device__ __forceinline__ void st16(double *p, const double (&v)[2]) {
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
}

template <typename T>
__global__ void k_tile_diag(const DTerm *terms, int nt, int64_t D, T *d) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < D; s += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < nt; k++) {
            const DTerm &t = terms[k];
            if (t.kind != DT_SPIN) continue;
            v += (((s >> t.i) ^ (s >> t.j)) & 1) ? -0.25 * t.a : 0.25 * t.a;
        }
        d[s] = (T)v;
    }
}

// One pass.  PASS 1 writes t; PASS 2 reads t and applies the epilogue.
// LPR lanes per row, E columns (16 bytes) each; RPW rows per warp;
// kTileUnroll bonds (tested, their targets loaded) in flight.
template <typename T, int PASS, int RED>
__global__ void __launch_bounds__(kTileThreads, PASS == 1 ? kTileMinB1 : (RED == 0 ? 4 : 3))
    k_tile(const HvArgs<T> a, const TileArgs ta, const T *__restrict__ diag, T *tbuf) {
    using S = TileShape<T>;
    constexpr int E = S::E, LPR = S::LPR, RPW = S::RPW, IB = S::IB;
    __shared__ uint32_t pin[4][256], pout[4][256];
    __shared__ uint32_t bm[kTileMaxBonds];
    __shared__ T bc[kTileMaxBonds];
    constexpr int P = PASS - 1;
    const uint32_t *tab = ta.tab + (size_t)P * 8 * 256;
    for (int i = threadIdx.x; i < 4 * 256; i += kTileThreads) {
        pin[i >> 8][i & 255] = tab[i];
        pout[i >> 8][i & 255] = tab[4 * 256 + i];
    }
    const int nb = ta.nb[P];
    for (int i = threadIdx.x; i < nb; i += kTileThreads) {
        bm[i] = ta.m[P][i];
        bc[i] = (T)ta.c[P][i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % LPR, rsub = lane / LPR;
    const int nin = ta.nin[P];
    const int64_t per_tile = (int64_t)1 << (nin - IB);
    const int64_t items = per_tile << ta.nout[P];
    const T *__restrict__ X = a.x;
    T al[E], ga[E];
#pragma unroll
    for (int k = 0; k < E; k++) {
        al[k] = (T)(a.alpha_dev ? a.alpha_dev[E * gl + k] : a.alpha[E * gl + k]);
        ga[k] = (T)(a.gamma_dev ? a.gamma_dev[E * gl + k] : a.gamma[E * gl + k]);
    }
    const T be = (T)a.beta;
    const bool use_beta = a.beta != 0.0, use_v = a.v != nullptr;
    constexpr int NR = RED == 2 ? 3 : (RED ? 1 : 0);
    RedAcc<T> racc[NR > 0 ? NR : 1][E];
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const uint32_t t = (uint32_t)(w >> (nin - IB));
        const uint32_t inner = ((uint32_t)(w & (per_tile - 1)) << IB) | (uint32_t)(warp * RPW + rsub);
        const uint32_t s = pin[0][inner & 255] | pin[1][(inner >> 8) & 255] | pin[2][(inner >> 16) & 255] |
                           pin[3][inner >> 24] | pout[0][t & 255] | pout[1][(t >> 8) & 255] |
                           pout[2][(t >> 16) & 255] | pout[3][t >> 24];
        const uint64_t roff = (uint64_t)s * 32 + E * gl;
        T acc[E], xo[E];
        if constexpr (PASS == 1) {
            ld16(X + roff, xo);
            const T d = __ldg(diag + s);
#pragma unroll
            for (int k = 0; k < E; k++) acc[k] = d * xo[k];
        } else {
            ldc16(tbuf + roff, acc);
        }
        int k = 0;
        for (; k + kTileUnroll <= nb; k += kTileUnroll) {
            T v[kTileUnroll][E];
            bool ok[kTileUnroll];
#pragma unroll
            for (int u = 0; u < kTileUnroll; u++) {
                const uint32_t m = bm[k + u];
                ok[u] = __popc(s & m) == 1;
                if (ok[u]) ld16(X + (uint64_t)(s ^ m) * 32 + E * gl, v[u]);
            }
#pragma unroll
            for (int u = 0; u < kTileUnroll; u++)
                if (ok[u]) {
                    const T c = bc[k + u];
#pragma unroll
                    for (int j = 0; j < E; j++) acc[j] = fma(c, v[u][j], acc[j]);
                }
        }
        for (; k < nb; k++) {
            const uint32_t m = bm[k];
            if (__popc(s & m) == 1) {
                T v[E];
                ld16(X + (uint64_t)(s ^ m) * 32 + E * gl, v);
                const T c = bc[k];
#pragma unroll
                for (int j = 0; j < E; j++) acc[j] = fma(c, v[j], acc[j]);
            }
        }
        if constexpr (PASS == 1) {
            st16(tbuf + roff, acc);
        } else {
            T out[E];
#pragma unroll
            for (int j = 0; j < E; j++) out[j] = al[j] * (a.swap ? acc[j ^ 1] : acc[j]);
            T *yr = a.y + roff;
            if (use_beta) {
                T yo[E];
                ldc16(yr, yo);
#pragma unroll
                for (int j = 0; j < E; j++) out[j] = fma(be, yo[j], out[j]);
            }
            if (use_v) {
                T vo[E];
                ldc16(a.v + roff, vo);
#pragma unroll
                for (int j = 0; j < E; j++) out[j] = fma(ga[j], vo[j], out[j]);
            }
            st16(yr, out);
            if constexpr (RED == 1 || RED == 2) ld16(X + roff, xo);
#pragma unroll
            for (int j = 0; j < E; j++) {
                if constexpr (RED == 1) racc[0][j].add(xo[j], out[j]);
                if constexpr (RED == 2) {
                    racc[0][j].add(xo[j], acc[j]);
                    racc[1][j].add(acc[j], acc[j]);
                    racc[2][j].add(xo[j], xo[j]);
                }
                if constexpr (RED == 3) racc[0][j].add(out[j], out[j]);
            }
        }
    }
    if constexpr (PASS == 2 && RED != 0) {
        // lanes gl, gl + LPR, ... hold the same columns
        __shared__ double red_sm[kTileThreads / 32][3][32];
#pragma unroll
        for (int r = 0; r < NR; r++)
#pragma unroll
            for (int j = 0; j < E; j++) {
                double v = racc[r][j].value();
#pragma unroll
                for (int off = LPR; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (rsub == 0) red_sm[warp][r][E * gl + j] = v;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * 32; i += kTileThreads) {
            const int r = i / 32, c = i % 32;
            double sum = 0.0;
            if (r < NR)
                for (int w2 = 0; w2 < kTileThreads / 32; w2++) sum += red_sm[w2][r][c];
            a.partials[((int64_t)blockIdx.x * 3 + r) * a.ncol + c] = sum;
        }
    }
}

uint32_t pdep32(uint32_t v, uint32_t mask) {
    uint32_t out = 0;
    for (int b = 0; b < 32 && v; b++)
        if ((mask >> b) & 1u) {
            if (v & 1u) out |= 1u << b;
            v >>= 1;
        }
    return out;
}

// Two disjoint site sets A, B with no off-diagonal bond between them and
// N - |A|, N - |B| <= smax: A grown greedily from each start site by the
// neighbour that adds the fewest new neighbours, B taken from the sites
// neither in A nor next to it.  Returns false when no start site gives both
// sizes.
bool find_cover(int N, const std::vector<uint64_t> &adj, int smax, uint64_t *A_out, uint64_t *B_out) {
    const int need = N - smax;
    if (need <= 0) {
        *A_out = 0;
        *B_out = 0;
        return true;
    }
    const uint64_t all = N == 64 ? ~0ull : ((1ull << N) - 1);
    auto nbr = [&](uint64_t A) {
        uint64_t n = 0;
        for (int v = 0; v < N; v++)
            if ((A >> v) & 1) n |= adj[v];
        return n & ~A;
    };
    for (int st = 0; st < N; st++) {
        uint64_t A = 1ull << st;
        while (__builtin_popcountll(A) < need) {
            const uint64_t cand = nbr(A) ? nbr(A) : (all & ~A);
            int best = -1, bc = 1 << 30;
            for (int v = 0; v < N; v++) {
                if (!((cand >> v) & 1)) continue;
                const int c = __builtin_popcountll(nbr(A | (1ull << v)));
                if (c < bc) {
                    bc = c;
                    best = v;
                }
            }
            if (best < 0) break;
            A |= 1ull << best;
            const uint64_t R = all & ~(A | nbr(A));
            if (__builtin_popcountll(A) >= need && __builtin_popcountll(R) >= need) {
                // B: `need` sites of R (the fewest that bring pass 2 within smax;
                // the sites left out keep their bonds free for either pass)
                uint64_t B = 0;
                for (int v = 0; v < N && __builtin_popcountll(B) < need; v++)
                    if ((R >> v) & 1) B |= 1ull << v;
                *A_out = A;
                *B_out = B;
                return true;
            }
        }
    }
    return false;
}

template <typename T, int PASS>
int go_tile(hphi_ctx *ctx, const HvArgs<T> &a, const TileArgs &ta, const T *diag, T *tbuf, int red_mode, int grid) {
#define HPHI_TILE(R) k_tile<T, PASS, R><<<grid, kTileThreads, 0, ctx->stream>>>(a, ta, diag, tbuf)
    switch (red_mode) {
    case 0: HPHI_TILE(0); break;
    case 1: HPHI_TILE(1); break;
    case 2: HPHI_TILE(2); break;
    case 3: HPHI_TILE(3); break;
    default: return HPHI_E_INVAL;
    }
#undef HPHI_TILE
    HPHI_CUDA(ctx, cudaGetLastError());
    return HPHI_OK;
}

}  // namespace

// Bit sets, bond split and tables of the tiled kernel for a full-space spin
// Hamiltonian (built on the first launch that asks for it).  Leaves
// ham->tile[prec] null when the model is not eligible or no split fits L2.
// prec 0: FP32 rows (128 bytes), 1: FP64 rows (256 bytes).
int build_tile_tables(hphi_ctx *ctx, hphi_ham *H, int prec) {
    if (prec < 0 || prec > 1) return set_err(ctx, HPHI_E_INVAL, "tiled kernel tables: unknown precision");
    if (H->tile[prec] || H->tile_tried[prec]) return HPHI_OK;
    H->tile_tried[prec] = 1;
    const double row_bytes = prec ? 256.0 : 128.0;
    const size_t es = prec ? sizeof(double) : sizeof(float);
    if (H->model != HPHI_SPIN_HALF_GC) return HPHI_OK;
    const int N = H->basis->N;
    if (N < kTileItemBits || N > 32) return HPHI_OK;
    std::vector<uint64_t> adj(N, 0);
    struct Bd {
        int i, j;
        double c;
    };
    std::vector<Bd> bonds;
    for (const DTerm &t : H->dterms) {
        if (t.kind != DT_SPIN || t.b == 0.0) continue;
        adj[t.i] |= 1ull << t.j;
        adj[t.j] |= 1ull << t.i;
        bonds.push_back(Bd{t.i, t.j, 0.5 * t.b});
    }
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess || l2 <= 0) {
        cudaGetLastError();
        return HPHI_OK;
    }
    // a tile of 2^s rows within 30 % of L2
    int smax = kTileItemBits;
    while (smax < N && (row_bytes * (double)(2ull << smax)) <= 0.3 * (double)l2) smax++;
    uint64_t A = 0, B = 0;
    if (!find_cover(N, adj, smax, &A, &B)) return HPHI_OK;
    const uint64_t all = (N == 64) ? ~0ull : ((1ull << N) - 1);
    TileArgs ta{};
    const uint64_t S[2] = {all & ~A, all & ~B};
    std::vector<Bd> part[2];
    for (const Bd &b : bonds) {
        const uint64_t m = (1ull << b.i) | (1ull << b.j);
        const bool in1 = (m & A) == 0, in2 = (m & B) == 0;
        if (in1 && in2) part[part[0].size() <= part[1].size() ? 0 : 1].push_back(b);
        else if (in1) part[0].push_back(b);
        else part[1].push_back(b);
    }
    std::vector<uint32_t> tab(2 * 8 * 256);
    for (int p = 0; p < 2; p++) {
        if ((int)part[p].size() > kTileMaxBonds) return HPHI_OK;
        ta.nin[p] = __builtin_popcountll(S[p]);
        ta.nout[p] = N - ta.nin[p];
        if (ta.nin[p] < kTileItemBits) return HPHI_OK;
        ta.nb[p] = (int)part[p].size();
        for (size_t k = 0; k < part[p].size(); k++) {
            ta.m[p][k] = (1u << part[p][k].i) | (1u << part[p][k].j);
            ta.c[p][k] = part[p][k].c;
        }
        const uint32_t in_mask = (uint32_t)S[p], out_mask = (uint32_t)(all & ~S[p]);
        for (int byte = 0; byte < 4; byte++)
            for (uint32_t v = 0; v < 256; v++) {
                tab[(size_t)p * 2048 + byte * 256 + v] = pdep32(v << (8 * byte), in_mask);
                tab[(size_t)p * 2048 + 1024 + byte * 256 + v] = pdep32(v << (8 * byte), out_mask);
            }
    }
    const int64_t D = H->D;
    cudaError_t e = cudaMalloc((void **)&H->tile_tab[prec], tab.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(H->tile_tab[prec], tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&H->tile_diag[prec], (size_t)D * es);
    if (e != cudaSuccess) {
        cudaFree(H->tile_tab[prec]);
        H->tile_tab[prec] = nullptr;
        return cuda_err(ctx, e, "tiled kernel tables");
    }
    const int gd = (int)std::min<int64_t>((D + 255) / 256, (int64_t)ctx->sm_count * 16);
    if (prec)
        k_tile_diag<double><<<gd, 256, 0, ctx->stream>>>(H->dterms_d, (int)H->dterms.size(), D,
                                                         (double *)H->tile_diag[prec]);
    else
        k_tile_diag<float><<<gd, 256, 0, ctx->stream>>>(H->dterms_d, (int)H->dterms.size(), D,
                                                        (float *)H->tile_diag[prec]);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "tiled kernel diagonal");
    ta.tab = H->tile_tab[prec];
    H->tile[prec] = new (std::nothrow) TileArgs(ta);
    if (!H->tile[prec]) return set_err(ctx, HPHI_E_NOMEM, "tiled kernel tables");
    return HPHI_OK;
}

template <typename T>
int launch_tile(hphi_ctx *ctx, const hphi_ham *ham, HvArgs<T> &a, int red_mode, int *grid) {
    constexpr int prec = std::is_same<T, float>::value ? 0 : 1;
    if (!ham->tile[prec]) return set_err(ctx, HPHI_E_INVAL, "tiled H*V: not available for this Hamiltonian");
    const TileArgs &ta = *ham->tile[prec];
    const size_t need = (size_t)ham->D * 32 * sizeof(T);
    T *tbuf = nullptr;
    if (a.beta == 0.0 && (a.v == nullptr || a.v != a.y)) {
        tbuf = a.y;
    } else {
        if (ctx->seg_tmp_bytes < need) {
            HPHI_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(ctx->seg_tmp);
            ctx->seg_tmp = nullptr;
            ctx->seg_tmp_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->seg_tmp, need);
            if (e != cudaSuccess) return cuda_err(ctx, e, "tiled H*V buffer");
            ctx->seg_tmp_bytes = need;
        }
        tbuf = (T *)ctx->seg_tmp;
    }
    if (red_mode < 0 || red_mode > 3) return set_err(ctx, HPHI_E_INVAL, "tiled H*V: unknown reduction mode");
    static const void *const pass2[4] = {(const void *)k_tile<T, 2, 0>, (const void *)k_tile<T, 2, 1>,
                                         (const void *)k_tile<T, 2, 2>, (const void *)k_tile<T, 2, 3>};
    // no more thread blocks than the partials of an H*x launch hold (8 per SM)
    auto grid_of = [&](const void *f) {
        int occ = dyn_occupancy(ctx, f, kTileThreads, 0);
        occ = occ < 1 ? 1 : (occ < 8 ? occ : 8);
        int64_t g = (int64_t)occ * ctx->sm_count;
        if (g > ham->nh) g = ham->nh;
        return (int)(g < 1 ? 1 : g);
    };
    const int g1 = grid_of((const void *)k_tile<T, 1, 0>), g2 = grid_of(pass2[red_mode]);
    *grid = g2;
    const T *diag = (const T *)ham->tile_diag[prec];
    const int slot = prof_begin(ctx, PROF_HV);
    int st = go_tile<T, 1>(ctx, a, ta, diag, tbuf, 0, g1);
    if (!st) st = go_tile<T, 2>(ctx, a, ta, diag, tbuf, red_mode, g2);
    prof_end(ctx, slot);
    if (st) return st;
    snprintf(ctx->last_kernel, sizeof ctx->last_kernel, "k_tile<%s,RED%d>x2@" HPHI_SRC_TAG, tname<T>(), red_mode);
    return HPHI_OK;
}

template int launch_tile<float>(hphi_ctx *, const hphi_ham *, HvArgs<float> &, int, int *);
template int launch_tile<double>(hphi_ctx *, const hphi_ham *, HvArgs<double> &, int, int *);

}  // namespace hphi
