// Internal structures shared by the translation units of libhphi.
//
// Layout of the hot path.  Every model is handled as a two-level structure:
// a row is (h, q) where h indexes a "block" of consecutive rows and q the row
// inside it.
//   spin sector:  h = high half of the spin string (N_hi = floor(N/2) bits),
//                 the block holds the sector states with that high half in
//                 ascending order, q = rank of the low half among the N_lo-bit
//                 strings of its popcount (Lin's ja), block base = jb[h].
//   spin GC:      h = high half, q = low half, base = h << N_lo.
//   Hubbard:      h = rank of the up string, q = rank of the down string,
//                 base = h * D_dn.
// A low half (or down string) is addressed by its "class position"
// cp = cp0(h) + q, which indexes the per-low-half tables built once per
// Hamiltonian: the diagonal part that depends on the low half only, the
// low-low off-diagonal neighbours (ELL lists of target q' and coefficient
// index), and for spin models the rank of the low half with one bit flipped.
// Everything that depends on h only (high-high / up-hop neighbours as row
// offsets, the high-only diagonal part, byte tables of the mixed diagonal
// part) is prepared per block in shared memory by the thread block that owns
// the block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hphi.h"

namespace hphi {

constexpr int kMaxHH = 128;     // high-high / up-hop neighbours of one block
constexpr int kMaxLH = 64;      // mixed (low-high) spin bonds
constexpr int kMaxGroups = 4;   // byte groups of the low half (<= 32 bits)
constexpr int kMaxCoef = 512;   // coefficient table (ELL coefficient indices)
constexpr int kMaxBond = 256;   // bonds per class in the descriptor
constexpr int kMaxCols = 128;   // real columns of one H*x launch
constexpr int kPhRanges = 32;   // row ranges of a block in the bond-major kernel's list offsets
constexpr int kThreads = 256;   // threads per block of the H*x kernel

enum Model { kSpin = HPHI_SPIN_HALF, kSpinGC = HPHI_SPIN_HALF_GC, kHubbard = HPHI_HUBBARD };

// reductions a fused H*x launch can produce, per real column
enum Red { R_NONE = 0, R_XHX = 1, R_HXHX = 2, R_XX = 3, R_XO = 4, R_OO = 5 };

struct HHBond {   // spin bond with both sites in the high half
    int i, j;     // bit positions inside h
    double cz;    // -Jz/2: diagonal change when the two spins differ
    double cxy;   // Jxy/2: off-diagonal element
};
struct LHBond {   // spin bond between high bit a and low bit b
    int a, b, bi; // bi = row of the flip table for low bit b
    double cz, cxy;
};
struct LLBondD {  // spin bond with both sites in the low half
    int i, j;
    double cz, cxy;
};
struct VTerm {    // Hubbard V n_i n_j
    int i, j;
    double v;
};

// The merged interaction list in plain form (one entry per bond / hop / U / V),
// for the direct row evaluation of the small-problem solver.
enum DTermKind { DT_SPIN = 0, DT_HOP = 1, DT_U = 2, DT_V = 3 };
struct DTerm {
    int kind, i, j, s;  // s: species of a hop (0 up, 1 down)
    double a, b;        // spin: Jz, Jxy; hop: t; U: U; V: V
};

// Tiled two-pass block H*V (hv_tile.cu): per pass the bit set of the tile's
// rows (nin bits varied inside a tile, nout bits fixed per tile), its bonds
// (masks and Jxy/2), and the bit-deposit tables of both index parts.
constexpr int kTileMaxBonds = 64;
struct TileArgs {
    const uint32_t *tab;  // [2 passes][inner, outer][4 bytes][256]
    int nin[2], nout[2], nb[2];
    uint32_t m[2][kTileMaxBonds];
    double c[2][kTileMaxBonds];
};

// Per-Hamiltonian descriptor (device copy read by every block at set-up).
struct HamDesc {
    int model;
    int N, nlo, nhi;  // spin: bit split; Hubbard: N sites, nlo = N (down string bits)
    int n;            // up spins (spin sector); -1 otherwise
    int n_hh, n_lh, n_ncoef;
    int n_v;
    int ngroups;      // byte groups of the low half / down string
    int64_t ddn;      // Hubbard: D_dn
    HHBond hh[kMaxBond];
    LHBond lh[kMaxLH];
    LLBondD ll[kMaxBond];
    int n_ll;
    VTerm v[kMaxBond];
    double U[64];     // Hubbard on-site U per site
    double coef[kMaxCoef];
};

// High-high pass (hv_seg.cu): the low half split into its lowest n0 =
// min(8, N_lo) bits and the upper n1 = N_lo - n0 bits l1, and the segment
// offsets SO[p][l1] = number of class-p low halves whose upper part is below l1.
struct SegArgs {
    int n0, n1, nlo, nhi, n;
    const uint16_t *so;  // [(N_lo + 1) << n1]
};

// Lin tables of one species (spin string, or up / down fermion string).
struct Species {
    int N = 0, n = 0, nlo = 0, nhi = 0;
    int64_t dim = 0;
    uint32_t *ja = nullptr;      // [2^nlo] rank of l within its popcount class
    uint64_t *jb = nullptr;      // [2^nhi] sector rows below h, ~0 if h occurs in no state
    uint64_t *jbp = nullptr;     // [2^nhi + 1] the same count without the sentinel
    uint32_t *loff = nullptr;    // [nlo + 2] first class position of each popcount
    uint32_t *lstate = nullptr;  // [2^nlo] low halves ordered by (popcount, value)
    uint32_t *states = nullptr;  // [dim] explicit states (Hubbard species), else null
    std::vector<uint32_t> loff_h;
};

}  // namespace hphi

struct hphi_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    char last_kernel[96] = {0};  // the last H*x kernel launched (name and template arguments)
    // reduction scratch: per-block partials and the reduced values
    double *partials = nullptr;
    size_t partials_n = 0;
    double *dscal = nullptr;     // device scalars (reduced values, driver coefficients)
    size_t dscal_n = 0;
    double *hscal = nullptr;     // pinned host mirror of dscal
    // driver vectors (Lanczos / TPQ), grown on demand
    void *vec[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t vec_bytes = 0;
    int *dflag = nullptr;        // device status word of consistency checks
    // high-high pass: its partial products when y cannot hold them
    void *seg_tmp = nullptr;
    size_t seg_tmp_bytes = 0;
    // streaming H*x on host vectors: two x and two y device buffers, copy
    // streams (host to device, device to host) and their ordering events
    void *io[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t io_bytes = 0;
    cudaStream_t io_stream[2] = {nullptr, nullptr};
    cudaEvent_t io_ev[7] = {};
    // kernel timing: event pairs recorded around launches while profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

struct hphi_basis {
    int model = 0, N = 0, nup = 0, ndn = 0;
    int64_t D = 0;
    int device = 0;
    hphi::Species sp[2];
};

struct hphi_ham {
    const hphi_basis *basis = nullptr;
    int model = 0;
    int device = 0;
    int64_t D = 0;
    int64_t nh = 0;              // number of blocks
    int64_t L = 0;               // length of the per-class-position tables
    int nlo = 0;
    hphi::HamDesc host;          // host copy of the descriptor
    hphi::HamDesc *desc = nullptr;
    // per-class-position tables
    double *dlow_d = nullptr;
    float *dlow_f = nullptr;
    uint8_t *ll_cnt = nullptr;
    uint32_t *ll_tgt = nullptr;
    uint16_t *ll_cf = nullptr;
    int ll_w = 0;
    uint32_t *flipq = nullptr;   // [nlb][L]
    int nlb = 0;
    // Hubbard up-string tables (per h)
    uint8_t *up_cnt = nullptr;
    uint32_t *up_tgt = nullptr;
    uint16_t *up_cf = nullptr;
    int up_w = 0;
    double *aup = nullptr;       // diagonal part of the up string alone
    uint32_t *ll_pk = nullptr;   // packed low-low lists (target | coefficient index << 24)
    uint16_t *ja16 = nullptr;    // Lin's ja as 16-bit ranks (spin sector, N_lo <= 16)
    // per-class bond lists of the bond-major kernel (spin sector, N_lo <= 16):
    // entries q | q' << 16 (class positions), grouped by (popcount p, bond),
    // with offsets per group at kPhRanges + 1 row-range boundaries
    uint32_t *ph_ent = nullptr;
    int32_t *ph_off = nullptr;
    int64_t ph_mx0 = 0;          // first offset row of the mixed-bond groups
    int max_row_entries = 0;
    // high-high pass (spin S^z sector, N_lo <= 16): host copy of its
    // arguments (null when not available) and its device table
    hphi::SegArgs *seg = nullptr;
    uint16_t *seg_so = nullptr;
    // tiled block kernel (full space, 32 columns), per precision [0: FP32, 1: FP64]
    // (the tiles follow the row size): built on first use
    hphi::TileArgs *tile[2] = {nullptr, nullptr};
    int tile_tried[2] = {0, 0};
    uint32_t *tile_tab[2] = {nullptr, nullptr};
    void *tile_diag[2] = {nullptr, nullptr};  // the diagonal of H, one value per row in that precision
    // plain term list (host and device) and, for the S^z sector, the state of
    // every row (built on first use by the small-problem solver)
    std::vector<hphi::DTerm> dterms;
    std::vector<hphi_term> terms;  // the interaction list as given (term ids of the pattern export)
    hphi::DTerm *dterms_d = nullptr;
    uint32_t *rowstate = nullptr;
    // launch tuning (hphi_ham_set_tuning)
    int tune_inner = -1;
    int tune_split = 1;
    int tune_hints = 1;
    int tune_variant = -1;       // -1 automatic, 0 table-driven, 1 on-the-fly ranks, 2 staged, 3 bond-major
    int tune_coop = -1;          // wide rows: lanes of a row share the bond work (-1: FP32 only)
    int tune_staged_lists = -1;  // staged kernel: bit 0 lists, bit 1 one more block per SM (-1: by dtype)
};

namespace hphi {

// ---- error helpers (capi.cu) ----------------------------------------------
int set_err(hphi_ctx *ctx, int code, const char *fmt, ...);
int cuda_err(hphi_ctx *ctx, cudaError_t e, const char *what);
#define HPHI_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::hphi::cuda_err(ctx, _e, #call); \
    } while (0)

// ---- workspace (capi.cu) -------------------------------------------------------
int ensure_partials(hphi_ctx *ctx, size_t n);
int ensure_dscal(hphi_ctx *ctx, size_t n);
int ensure_vecs(hphi_ctx *ctx, size_t bytes);

// ---- dynamic shared memory (capi.cu) -------------------------------------------
// Occupancy (thread blocks per SM) of kernel fn with `threads` threads and
// `dyn` bytes of dynamic shared memory on the context's device.  The first
// call for a (kernel, device) raises the kernel's dynamic shared-memory limit
// to everything the device allows next to its static shared memory, so the
// limit never goes down and launches of one kernel with different sizes from
// several host threads cannot undercut one another.  Thread-safe.
int dyn_occupancy(hphi_ctx *ctx, const void *fn, int threads, size_t dyn);

// ---- kernel timing (capi.cu): returns a slot, -1 when not profiling ----------
int prof_begin(hphi_ctx *ctx, int kind);
void prof_end(hphi_ctx *ctx, int slot);
enum ProfKind { PROF_HV = 0, PROF_VEC = 1 };

// ---- basis (basis.cu) -----------------------------------------------------------
int build_species(hphi_ctx *ctx, Species &sp, int N, int n, bool want_states);
void free_species(Species &sp);

// ---- H*x launch description (hv.cu) ------------------------------------------------
struct HvLaunch {
    int dtype_real;          // HPHI_F64 or HPHI_F32 (complex data passed as 2x real columns)
    int ncol;                // real columns
    const void *x;
    int64_t ldx;             // in real elements
    void *y;
    int64_t ldy;
    const void *v;           // optional third vector (gamma term), may alias y
    int64_t ldv;
    double beta;
    const double *alpha_h;   // [ncol] host (nullptr: alpha_s for every column)
    const double *gamma_h;   // [ncol] host (nullptr: gamma_s)
    double alpha_s, gamma_s;
    const double *coef_dev;  // device [2*ncol]: alpha_c then gamma_c; overrides host values
    int swap;                // 1: y[c] = alpha_c (H x)[c ^ 1] + ... (ncol even); complex rotation
    int red[3];              // reductions (Red codes)
    double *partials;        // per column slice: [grid][3][nc], slices back to back
    int nslice;              // column slices launched (filled by the launcher)
    int sgrid[kMaxCols];     // grid of slice s
    int sc0[kMaxCols];       // first column of slice s
    int snc[kMaxCols];       // columns of slice s
};
int launch_hv(hphi_ctx *ctx, const hphi_ham *ham, HvLaunch &L);
// Upper bound of partials entries of one launch with ncol columns.
size_t hv_partials_size(hphi_ctx *ctx, const hphi_ham *ham, int ncol);
// Sums the partials of a finished launch: out_dev[r * ncol + c], r < 3.
int reduce_hv(hphi_ctx *ctx, const HvLaunch &L, double *out_dev);

// ---- reductions / vector kernels (vec.cu) ----------------------------------------------
// Sums partials[grid][nval] over grid in fixed order into out_dev[nval].
int reduce_partials(hphi_ctx *ctx, const double *partials, int grid, int nval, double *out_dev);
int launch_dot(hphi_ctx *ctx, int real_dtype, int cplx, int64_t n, int nr, const void *x, int64_t ldx,
               const void *y, int64_t ldy, double *out_dev /* nr (+ nr cross) */);
// out = a[c] x[c] + b[c] x[c^1] + g[c] y[c]   (real columns; coefficient arrays host or device)
struct LinComb {
    int real_dtype;
    int64_t n;
    int nr;
    const void *x;
    int64_t ldx;
    const void *y;
    int64_t ldy;
    void *out;
    int64_t ldo;
    const double *a_h, *b_h, *g_h;      // host [nr] (nullable -> 0)
    const double *coef_dev;             // device [3*nr] (a, b, g) overrides
    int red_oo;                          // also reduce sum out^2 per column
    double *partials;
    int grid;
};
int launch_lincomb(hphi_ctx *ctx, LinComb &L);
int launch_random(hphi_ctx *ctx, int real_dtype, int64_t n, int nr, uint64_t seed, void *x, int64_t ldx);
// c[j] = <V_j, w> for nv vectors stored back to back (V_j at V + j*n), into out_dev[nv]
int launch_mdot(hphi_ctx *ctx, int real_dtype, int64_t n, int nv, const void *V, const void *w, double *out_dev);
// w -= sum_j c_dev[j] V_j
int launch_maxpy(hphi_ctx *ctx, int real_dtype, int64_t n, int nv, const void *V, const double *c_dev, void *w);
int launch_copy(hphi_ctx *ctx, int real_dtype, int64_t n, int nr, const void *x, int64_t ldx, void *y,
                int64_t ldy);

// ---- tridiagonal helpers (drivers.cu) ------------------------------------------------
int tridiag_ql(int n, double *d, double *e, double *z);
// lowest eigenvalue of the Lanczos tridiagonal T_m (alpha[0..m-1], beta2[1..m-1])
// and |last component| of its normalised eigenvector
int lowest_ritz(int m, const double *alpha, const double *beta2, double *theta, double *ylast);
// the same with a warm start (an upper bound of the lowest eigenvalue, updated)
int lowest_ritz_warm(int m, const double *alpha, const double *beta2, double *warm, double *theta, double *ylast);

// ---- high-high pass table (hv_seg.cu) ------------------------------------------------
int build_seg_tables(hphi_ctx *ctx, hphi_ham *H);
// ---- tiled block kernel tables (hv_tile.cu) ------------------------------------------
int build_tile_tables(hphi_ctx *ctx, hphi_ham *H, int prec);

// ---- pattern (pattern.cu) --------------------------------------------------------
int dump_rows(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1, std::vector<int64_t> &cols,
              std::vector<double> &vals, std::vector<int32_t> &cnt, int &stride);

inline int real_of(int dtype) { return (dtype == HPHI_F64 || dtype == HPHI_C128) ? HPHI_F64 : HPHI_F32; }
inline int is_complex(int dtype) { return dtype == HPHI_C128 || dtype == HPHI_C64; }
inline size_t real_size(int real_dtype) { return real_dtype == HPHI_F64 ? 8 : 4; }
inline bool valid_dtype(int d) { return d >= HPHI_F64 && d <= HPHI_C64; }

}  // namespace hphi
