/*
 * hphi.h -- C ABI of the GB300 (sm_103a) library for the matrix-free
 * Hamiltonian-vector product of spin-1/2 and Hubbard models and the Krylov /
 * thermal-pure-quantum drivers built on it.
 *
 * What the library computes (arXiv 2307.13222, "Update of H-Phi"):
 *   - every iterative method of the paper reduces to repeated products of the
 *     Hamiltonian with a wave function (Sec. 1; Sec. 3.4; Sec. 3.5.1), done
 *     here matrix-free over a bit-encoded basis;
 *   - Lanczos ground states (Sec. 1, Table 1), canonical TPQ steps
 *     (Sec. 3.5.1, the equations of U_c and beta_k), and the vector kernels
 *     around them.
 * Hamiltonians (Sec. 3.1.1 Heisenberg example; Sec. 3.4 equation of
 * H_quench; Sec. 5 Eq. ham_general):
 *   spin-1/2  H = sum_b [ Jz_b S^z_i S^z_j + Jxy_b (S^x_i S^x_j + S^y_i S^y_j) ]
 *   Hubbard   H = - sum t (c^+_{i s} c_{j s} + h.c.) + U sum_i n_{i up} n_{i dn}
 *                 + sum V n_i n_j
 * Basis (the paper leaves it to its version-1 predecessor): bit i of a spin
 * string is site i (1 = up spin / occupied); sector states are in ascending
 * integer order and ranked with H. Q. Lin's two-table index
 *   rank(s) = ja[s & (2^N_lo - 1)] + jb[s >> N_lo],  N_lo = N - floor(N/2);
 * a Hubbard row is rank_up * D_dn + rank_dn, and a fermion state is
 *   prod_{i asc} c^+_{i up} prod_{i asc} c^+_{i dn} |0>, so a hop of species s
 *   between i and j carries (-1)^(# s-fermions strictly between i and j).
 *
 * Conventions for every call:
 *   - Status: 0 on success, a negative HPHI_E_* code otherwise; the message is
 *     in hphi_last_error(ctx).  No call aborts the process or throws.
 *   - Device vectors are caller-owned raw device pointers, row-major
 *     [D][nvec] with leading dimension ld (elements, >= nvec).  Complex
 *     dtypes store (re, im) pairs; ld counts complex elements.  The library
 *     never frees or keeps them after the call returns.
 *   - Host arrays (double *... "host") are caller-owned host memory.
 *   - Work is enqueued on the context's stream.  Calls that return host
 *     scalars (dot, nrm2, drivers) synchronise that stream before returning;
 *     hphi_apply_H, hphi_axpy, hphi_scal and hphi_random_vector are
 *     asynchronous.
 *   - Handles (ctx, basis, ham) are library-owned; destroy them with the
 *     matching call.  A basis or ham belongs to the device of the context it
 *     was built with.  A context is not thread-safe.
 */
#ifndef HPHI_H
#define HPHI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HPHI_API __attribute__((visibility("default")))
#else
#define HPHI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HPHI_OK 0
#define HPHI_E_INVAL (-1)        /* bad argument, size, alias or term        */
#define HPHI_E_NOMEM (-2)        /* device or host allocation failed         */
#define HPHI_E_CUDA (-3)         /* a CUDA runtime error (text in last_error) */
#define HPHI_E_NOTCONV (-4)      /* driver hit max_steps before tolerance    */
#define HPHI_E_NUMERIC (-5)      /* NaN/Inf or a non-positive norm           */
#define HPHI_E_DEVICE_CHECK (-6) /* a device-side consistency check failed   */
#define HPHI_E_TIMEOUT (-7)      /* a bounded device-side wait ran out       */

/* ---- models (Table 1 of the paper: Spin, SpinGC, Hubbard) --------------- */
#define HPHI_SPIN_HALF 0    /* spin-1/2, fixed number of up spins (S^z)     */
#define HPHI_SPIN_HALF_GC 1 /* spin-1/2, full 2^N space                     */
#define HPHI_HUBBARD 2      /* Hubbard, fixed N_up and N_dn                  */

/* ---- vector element types ----------------------------------------------- */
#define HPHI_F64 0
#define HPHI_F32 1
#define HPHI_C128 2 /* complex double, (re, im) pairs */
#define HPHI_C64 3  /* complex float,  (re, im) pairs */

/* ---- interaction terms (the paper's J / t / U / V terms) ----------------- */
#define HPHI_EXCHANGE 0  /* J S_i.S_j;                 v0 = J                 */
#define HPHI_XXZ 1       /* Jz SzSz + Jxy (SxSx+SySy);  v0 = Jz, v1 = Jxy      */
#define HPHI_HOP 2       /* -t (c+_{is} c_{js} + h.c.); v0 = t, spin 0 up,
                            1 down, -1 both                                  */
#define HPHI_HUBBARD_U 3 /* U n_{i up} n_{i dn};        v0 = U, j ignored      */
#define HPHI_DENS_DENS 4 /* V n_i n_j (n = n_up + n_dn); v0 = V               */

typedef struct hphi_term {
    int32_t kind, i, j, spin;
    double v0, v1;
} hphi_term;

typedef struct hphi_ctx hphi_ctx;
typedef struct hphi_basis hphi_basis;
typedef struct hphi_ham hphi_ham;

/* ---- context -------------------------------------------------------------
 * hphi_ctx_create: binds `device` and the CUDA stream `stream` (a
 * cudaStream_t, NULL = legacy default stream).  Errors: HPHI_E_INVAL (bad
 * device), HPHI_E_CUDA, HPHI_E_NOMEM.  The library allocates its own
 * workspace (reduction partials, driver vectors) lazily on the device. */
HPHI_API int hphi_ctx_create(int device, void *stream, hphi_ctx **out);
HPHI_API int hphi_ctx_set_stream(hphi_ctx *ctx, void *stream);
HPHI_API void hphi_ctx_destroy(hphi_ctx *ctx);
/* Message of the last failing call on this context ("" if none). */
HPHI_API const char *hphi_last_error(const hphi_ctx *ctx);
/* Name of the last H*x kernel this context launched, with the template
 * arguments that select its code path and a hash of the H*x kernel sources
 * (e.g. "k_hvp<f32,512,RED1,MINB2>@0123456789"); "" before the first
 * launch.  For matching profiles to launches: a profile taken on other
 * kernel sources carries another hash. */
HPHI_API const char *hphi_last_kernel(const hphi_ctx *ctx);
/* Number of SMs of the context's device (grid sizing information). */
HPHI_API int hphi_ctx_sm_count(const hphi_ctx *ctx);

/* ---- kernel timing ---------------------------------------------------------
 * hphi_ctx_profile(ctx, 1) records a CUDA event pair on the context's stream
 * around every launch of the H*x kernel (kind 0) and of the vector kernels
 * (kind 1: dot/nrm2 partials, axpy/scal/lincomb); 0 stops recording.
 * hphi_ctx_profile_read synchronises the stream and returns, for `kind`, the
 * number of launches and their summed device time (ms) since the previous
 * read of that kind, then resets that kind. */
HPHI_API int hphi_ctx_profile(hphi_ctx *ctx, int enable);
HPHI_API int hphi_ctx_profile_read(hphi_ctx *ctx, int kind, int64_t *launches, double *total_ms);

/* ---- basis (Sec. 3.5.1: "x may be the set of spin positions"; Table 1
 * sectors 2Sz / nelec) ------------------------------------------------------
 * hphi_build_basis: builds the two-table rank of the sector on the device.
 *   SPIN_HALF: n_sites <= 40 (tables of 2^ceil(N/2) entries), 0 <= n_up <= N.
 *   SPIN_HALF_GC: n_sites <= 36; n_up, n_dn ignored.
 *   HUBBARD: n_sites <= 32, 0 <= n_up, n_dn <= N, C(N, n) < 2^31 per species.
 * Errors: HPHI_E_INVAL for sizes outside these limits or an empty sector,
 * HPHI_E_NOMEM, HPHI_E_CUDA. */
HPHI_API int hphi_build_basis(hphi_ctx *ctx, int model, int n_sites, int n_up, int n_dn, hphi_basis **out);
HPHI_API void hphi_basis_destroy(hphi_basis *basis);
HPHI_API int64_t hphi_basis_dim(const hphi_basis *basis);
/* Sizes of the Lin tables of `species` (0: spins / up fermions, 1: down
 * fermions): n_ja = 2^N_lo, n_jb = 2^N_hi.  GC models have no tables (0). */
HPHI_API int hphi_basis_table_sizes(const hphi_basis *basis, int species, int64_t *n_ja, int64_t *n_jb);
/* Copies the tables to host arrays of the sizes above (for bit-exact checks).
 * jb holds ~0 for high halves that occur in no sector state. */
HPHI_API int hphi_basis_export(hphi_ctx *ctx, const hphi_basis *basis, int species, uint32_t *ja_host, uint64_t *jb_host);
/* Device: states of rows [row0, row0+n): su[k] (spin string / up string) and
 * sd[k] (down string, Hubbard only; may be NULL otherwise). */
HPHI_API int hphi_basis_states(hphi_ctx *ctx, const hphi_basis *basis, int64_t row0, int64_t n, uint64_t *su_dev,
                      uint64_t *sd_dev);
/* Device: rows of the n states (su, sd); -1 for a state outside the sector. */
HPHI_API int hphi_basis_rank(hphi_ctx *ctx, const hphi_basis *basis, const uint64_t *su_dev, const uint64_t *sd_dev,
                    int64_t n, int64_t *row_dev);

/* ---- Hamiltonian (interaction list; Expert-mode terms, Sec. 3.4 and 5) -----
 * Validates the terms (site bounds, i != j for pair terms, kind allowed for
 * the model: spin models take EXCHANGE/XXZ, Hubbard takes HOP/HUBBARD_U/
 * DENS_DENS) and builds the per-sector tables the kernels use.  Repeated pairs
 * are summed.  Errors: HPHI_E_INVAL, HPHI_E_NOMEM, HPHI_E_CUDA.  The ham keeps
 * a reference to `basis`, which must outlive it. */
HPHI_API int hphi_build_hamiltonian(hphi_ctx *ctx, const hphi_basis *basis, const hphi_term *terms, int n_terms,
                           hphi_ham **out);
HPHI_API void hphi_ham_destroy(hphi_ham *ham);
HPHI_API int64_t hphi_ham_dim(const hphi_ham *ham);

/* ---- launch tuning of a Hamiltonian ------------------------------------------
 * Knobs of the H*x kernel for this Hamiltonian (all launches that use it):
 *   HPHI_TUNE_INNER_BITS  high-half bits of the row-block traversal varied
 *                         first (an L2-resident subcube); -1 = automatic
 *   HPHI_TUNE_SPLIT       thread blocks that share one row block (1..8),
 *                         fewer row blocks in flight for the same occupancy
 *   HPHI_TUNE_L2_HINTS    1 = L2 eviction-priority hints on gathers/streams
 *   HPHI_TUNE_VARIANT     -1 = automatic (default); spin models: 1 = neighbour
 *                         ranks computed on the fly from Lin's ja table, 0 =
 *                         precomputed neighbour lists (also enables the
 *                         one-thread-per-row kernel for Hubbard), 2 = staged:
 *                         the row block's x in shared memory and low-half
 *                         ranks from shared tables (S^z sector, one column,
 *                         N_lo <= 16), 3 = bond-major: the staged block's H x
 *                         accumulated in shared memory one bond at a time over
 *                         precomputed lists of the rows the bond applies to
 *                         (same shapes as 2), 4 = a streaming pass for the
 *                         high-high bonds over L2-sized chunks of the low
 *                         half, then the bond-major kernel without them
 *                         (same shapes as 3, D < 2^31; on request), 5 =
 *                         tiled: full space, 32 columns (FP32 or FP64), the bonds split
 *                         over two passes that each gather only inside an
 *                         L2-resident tile of rows (automatic there when the
 *                         bond graph has such a split)
 *   HPHI_TUNE_COOP        32-column rows: 1-5 = the lanes of a row split the
 *                         bond evaluation and share targets (1: 8 targets per
 *                         batch, registers for 2 thread blocks per SM; 2: 4
 *                         targets, 3 blocks; 3: 4 targets, 4 blocks; 4: 4
 *                         targets, 5 blocks; 5: 2 targets, 6 blocks), 0 =
 *                         every lane evaluates every bond, -1 = 3 for FP32 and
 *                         0 for FP64 data (default)
 *   HPHI_TUNE_STAGED_LISTS staged kernel, two bits: bit 0 set = low-low
 *                         targets and flipped ranks from the per-low-half
 *                         lists, clear = from the shared rank tables; bit 1
 *                         set = registers sized for one more thread block per
 *                         SM; -1 = 3 for FP32 and 2 for FP64 data (default)
 * Results do not depend on the knobs except through summation order of the
 * reductions (still deterministic for fixed knobs).  HPHI_E_INVAL for an
 * unknown knob or value. */
/* hphi_ham_autotune: times every valid setting of the knobs below for
 * hphi_apply_H on this Hamiltonian with nvec columns of dtype (reps timed
 * launches each, after one warm-up; vectors allocated and freed here), keeps
 * the fastest on the Hamiltonian and reports its time per launch (*best_ms)
 * and the number of settings tried.  Later calls of any shape use the chosen
 * settings.  HPHI_E_NOMEM if two vectors of that shape do not fit. */
HPHI_API int hphi_ham_autotune(hphi_ctx *ctx, hphi_ham *ham, int dtype, int nvec, int reps, double *best_ms,
                               int *n_tried);
#define HPHI_TUNE_INNER_BITS 0
#define HPHI_TUNE_SPLIT 1
#define HPHI_TUNE_L2_HINTS 2
#define HPHI_TUNE_VARIANT 3
#define HPHI_TUNE_COOP 4
#define HPHI_TUNE_STAGED_LISTS 5
HPHI_API int hphi_ham_set_tuning(hphi_ham *ham, int knob, int value);
HPHI_API int hphi_ham_get_tuning(const hphi_ham *ham, int knob, int *value);

/* ---- H*x (the hot path) -------------------------------------------------
 * y <- alpha * H x + beta * y for nvec columns (1 <= nvec <= 128 real
 * columns; a complex column counts as two).  x and y are device arrays of
 * `dtype`, [D][nvec] with leading dimensions ldx, ldy >= nvec.  beta == 0
 * does not read y.  x and y must not overlap (HPHI_E_INVAL).  Asynchronous. */
HPHI_API int hphi_apply_H(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, const void *x, int64_t ldx, void *y,
                 int64_t ldy, double alpha, double beta);

/* ---- H*x on host vectors (streaming) -------------------------------------
 * y_b <- alpha * H x_b for nbatch independent vectors held in HOST memory:
 * x_host and y_host each hold nbatch arrays of [D][nvec] elements of dtype,
 * one after another (leading dimension nvec).  The library copies x_b to the
 * device, applies H (the same kernels as hphi_apply_H) and copies y_b back;
 * the copy of x_{b+1} to the device and of y_{b-1} to the host overlap the
 * product of b (two device buffers each for x and y, context-owned, 4 * D *
 * nvec * size bytes, grown on first use).  Pinned host memory (cudaHostAlloc,
 * cudaHostRegister) gives full copy speed; pageable memory works with
 * serialised copies.  Synchronous: returns once every y_b is on the host.
 * x and y must not overlap.  Errors as hphi_apply_H, and HPHI_E_CUDA when
 * the device buffers cannot be allocated. */
HPHI_API int hphi_apply_H_host(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, int64_t nbatch,
                               const void *x_host, void *y_host, double alpha);

/* ---- matrix pattern (debug; the paper's Matrix Market export, Sec. 3.1.2) --
 * hphi_dump_pattern: the off-diagonal entries of rows [row0, row1) of H, one
 * entry per term acting on the row's basis state (a HOP with spin = -1 gives
 * its up entry, then its down entry), ordered by row and then by term id:
 *   rows_host[k], cols_host[k]  the entry's row and column,
 *   signs_host[k]  the fermion sign of a hop, (-1)^(# occupied sites of the
 *                  hopping species strictly between i and j); +1 for a spin
 *                  flip,
 *   term_ids_host[k]  the index of the term in the list given to
 *                  hphi_build_hamiltonian.
 * The matrix element of the entry is sign * (-t) for a hop and Jxy/2 for a
 * spin flip (EXCHANGE: Jxy = J); terms with t = 0 or Jxy = 0 give no entry.
 * Duplicate or cancelling terms stay separate entries.  The diagonal is not
 * listed.  *count: in, the capacity of the four host arrays; out, the number
 * of entries.  With too small a capacity (or any array NULL) the call
 * returns HPHI_E_INVAL and sets *count to the number needed.  At most 2^22
 * rows per call.  HPHI_E_DEVICE_CHECK if a target falls outside the sector.
 *
 * hphi_dump_pattern_merged: the same rows with the entries of equal column
 * merged (summed), columns ascending, the diagonal always included, in CSR
 * form: rowptr_host has row1-row0+1 entries; cols_host / vals_host hold at
 * least *nnz_capacity entries.  On HPHI_E_INVAL because the capacity is too
 * small, *nnz_capacity is set to the needed count.  This is the matrix the
 * paper's Matrix Market file lists. */
HPHI_API int hphi_dump_pattern(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1, int64_t *rows_host,
                               int64_t *cols_host, int8_t *signs_host, int32_t *term_ids_host, int64_t *count);
HPHI_API int hphi_dump_pattern_merged(hphi_ctx *ctx, const hphi_ham *ham, int64_t row0, int64_t row1,
                                      int64_t *rowptr_host, int64_t *cols_host, double *vals_host,
                                      int64_t *nnz_capacity);

/* ---- vector kernels ---------------------------------------------------------
 * n rows, nvec columns, leading dimensions in elements of `dtype`.
 * Reductions are deterministic (fixed per-block partials, fixed-order sum)
 * and accumulate in FP64 (FP32 inputs: compensated float-float per thread).
 *   hphi_dot:  out_host[q] = <x_q|y_q> (complex: out_host[2q], [2q+1] = re, im
 *              of sum conj(x) y)
 *   hphi_nrm2: out_host[q] = |x_q|_2
 *   hphi_axpy: y_q += a_q x_q  (a_host: nvec reals, or nvec (re, im) pairs)
 *   hphi_scal: x_q *= a_q
 *   hphi_random_vector: x[r][c] = Gaussian of Philox4x32-10 stream element
 *              r * reals_per_row + c (reals_per_row = nvec, or 2*nvec for
 *              complex), key = seed; Box-Muller of two 53-bit uniforms. */
HPHI_API int hphi_dot(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const void *x, int64_t ldx, const void *y,
             int64_t ldy, double *out_host);
HPHI_API int hphi_nrm2(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const void *x, int64_t ldx, double *out_host);
HPHI_API int hphi_axpy(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const double *a_host, const void *x, int64_t ldx,
              void *y, int64_t ldy);
HPHI_API int hphi_scal(hphi_ctx *ctx, int dtype, int64_t n, int nvec, const double *a_host, void *x, int64_t ldx);
HPHI_API int hphi_random_vector(hphi_ctx *ctx, int dtype, int64_t n, int nvec, uint64_t seed, void *x, int64_t ldx);

/* ---- dot product without any device allocation ------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: a process that reserved its whole device
 * memory budget up front (for example a solver service holding every Krylov
 * vector resident), a host framework whose allocator must own every
 * allocation, or a latency-critical path on which cudaMalloc, which can
 * synchronise the device, is not acceptable.  Such callers cannot create an
 * hphi_ctx (its workspace is allocated), so this entry point takes the device
 * and stream directly.
 * It computes <x_q|y_q> for nvec columns of dtype on `device` with the
 * kernels of hphi_dot (same per-block partial sums, same fixed-order final
 * sum), enqueued on `stream` (a cudaStream_t, NULL = legacy default stream),
 * and waits for that stream.  Its grid is hphi_dot's (at most 8 blocks per
 * SM) capped at HPHI_DOT_STATIC_MAX_BLOCKS: on devices with at most
 * HPHI_DOT_STATIC_MAX_BLOCKS / 8 SMs (GB300 has 152) both calls sum in the
 * same order and return bitwise-equal results; on larger devices the block
 * partition of long vectors differs and the results agree to rounding.
 * x and y must be device memory of `device` (or managed memory); anything
 * else returns HPHI_E_INVAL.
 * Scratch: a file-scope device array of HPHI_DOT_STATIC_SCRATCH_BYTES
 * (about 2 MB) that every GPU which loads the library keeps until the
 * process exits; no cudaMalloc, cudaFree or allocating library routine is
 * called.  Every call looks up the array's device address with `device`
 * current (a host-side lookup that allocates nothing).  The first call on a
 * device may also load the library's device code onto it, so make that
 * first call before any stream capture.  Limits: at most
 * HPHI_DOT_STATIC_MAX_REAL real columns (a complex column counts two);
 * larger requests return HPHI_E_INVAL.  The calling thread's current device
 * is restored before returning.
 * Every call uses the same array, and nothing in it needs to start at zero
 * (each call writes every slot it reads before reading it).  Calls that
 * overlap on the GPU (other streams, other threads) race on the array: do not
 * overlap them. */
#define HPHI_DOT_STATIC_MAX_REAL 64
#define HPHI_DOT_STATIC_MAX_BLOCKS 2048
#define HPHI_DOT_STATIC_SCRATCH_BYTES (8 * (2 * HPHI_DOT_STATIC_MAX_BLOCKS * HPHI_DOT_STATIC_MAX_REAL + 2 * HPHI_DOT_STATIC_MAX_REAL))
HPHI_API int hphi_dot_static(int device, void *stream, int dtype, int64_t n, int nvec, const void *x, int64_t ldx,
                             const void *y, int64_t ldy, double *out_host);

/* ---- Lanczos ground state (Sec. 1, Table 1) ---------------------------------
 * Three-term Lanczos from v0 (device, length D, dtype F64 or F32: the storage
 * precision of the Krylov vectors; alpha/beta, the tridiagonal problem and
 * the reductions are FP64).  Stops when the residual estimate
 * beta_{m+1} |y_m| <= tol * max(1, |theta_0|) (tol <= 0: run max_steps), on
 * an invariant subspace, or at max_steps.  With gs_out != NULL (device,
 * length D, same dtype) a second pass rebuilds the Krylov vectors and returns
 * the normalised Ritz vector, and `resid` is the explicit |H x - theta x|.
 * alpha_host / beta_host (nullable) receive max_steps and max_steps+1
 * values.  Returns HPHI_OK, HPHI_E_NOTCONV (tol > 0 not reached; result
 * filled in), or an error. */
typedef struct hphi_lanczos_opts {
    int max_steps;
    double tol;
    int dtype;       /* HPHI_F64 or HPHI_F32 */
    int check_every; /* host convergence check period in steps (>= 1) */
    int reorth;      /* 0: three-term recurrence (two passes for the vector);
                        1: full reorthogonalisation, classical Gram-Schmidt
                        applied twice against every stored Krylov vector
                        (the library allocates (max_steps + 1) vectors) */
} hphi_lanczos_opts;

typedef struct hphi_lanczos_result {
    double e0;        /* lowest Ritz value */
    double resid_est; /* beta_{m+1} |y_m| */
    double resid;     /* |H x - e0 x| (only with gs_out), else -1 */
    int steps;
    int breakdown;    /* 1 if an invariant subspace ended the run */
    double e0_rq;     /* <x|H x> / <x|x> of the returned ground-state vector x
                         in FP64 arithmetic (an FP32 x is widened first), only
                         with gs_out, else NaN; NaN also when the two FP64
                         work vectors it needs (one for F64) cannot be
                         allocated.  For F32 storage this is the refined
                         energy: its error is quadratic in the error of x */
} hphi_lanczos_result;

HPHI_API int hphi_lanczos(hphi_ctx *ctx, const hphi_ham *ham, const hphi_lanczos_opts *opts, const void *v0, void *gs_out,
                 double *alpha_host, double *beta_host, hphi_lanczos_result *result);

/* ---- many small problems at once: the Lanczos driver in batched form -------------
 * hphi_lanczos_batch: the ground state of nprob independent problems (as
 * hphi_lanczos computes it: same recurrence, same stopping rule evaluated
 * after every step, two-pass ground-state vector; FP64, no
 * reorthogonalisation), one thread block per problem.  hams[p] (may repeat),
 * v0[p]: device FP64 start vector of length D_p; gs_out: null, or per
 * problem a device FP64 vector of length D_p or null.  opts->check_every is
 * the number of steps one launch runs (the stopping step does not depend on
 * it; larger values mean fewer launches and host checks).  Per problem:
 * results[p] (e0, resid_est, resid = |H gs - e0 gs| when gs_out[p] is given
 * else -1, steps, breakdown) and status[p] = HPHI_OK, HPHI_E_NOTCONV (tol > 0
 * not reached in max_steps), HPHI_E_NUMERIC or HPHI_E_INVAL (zero start
 * vector).  Returns HPHI_OK when every status is OK, otherwise an error code
 * from the statuses (errors before HPHI_E_NOTCONV).  A problem's results do
 * not depend on the rest of the batch (bit for bit).  Limits: D_p <= 2^26,
 * at most 256 merged terms, S^z sectors of at most 32 sites, nprob <= 65535.
 * Workspace: 3 D_p + 2 max_steps + 3 doubles per problem. */
HPHI_API int hphi_lanczos_batch(hphi_ctx *ctx, int nprob, hphi_ham *const *hams, const void *const *v0,
                                void *const *gs_out, const hphi_lanczos_opts *opts, hphi_lanczos_result *results,
                                int *status);

/* ---- serving loop: continuous batching of ground-state and spectrum requests -----
 * A server owns a device arena of opts->mem_budget bytes for the workspaces of
 * small problems (D <= small_max_dim, at most 256 merged terms), which run on
 * the batched block engine of hphi_lanczos_batch: every running recurrence is
 * one thread block, and hphi_server_step launches the next opts->chunk steps
 * of all of them at once, then evaluates each stopping rule after every step,
 * retires finished requests (freeing their memory at once) and admits queued
 * ones (FIFO) whose workspace fits and for which block slots are free.
 * Larger problems go to a second lane: worker threads that run the
 * grid-wide drivers, each on its own CUDA stream, concurrently.  A request's result
 * does not depend on the other requests (bit for bit).
 * Requests: HPHI_REQ_GROUND, the ground-state energy (hphi_lanczos' recurrence
 * and stopping rule, FP64, Philox start vector of `seed`, residual `tol`);
 * HPHI_REQ_SPECTRUM, in addition D(z_j) = <Phi|(z_j - H)^{-1}|Phi> for
 * Phi = sum_l e^{i q l} S^z_l Phi_0 and z_j = E0 + omega[j] + i eta (Sec. 3.2),
 * by the shifted-Krylov recurrences of Phi's real and imaginary parts, stopped
 * when every shift's relative residual is <= tol.  The Hamiltonian is the
 * caller's and must outlive the request; `omega` is copied at submission.
 * hphi_server_result: done = 1 once finished; the times are seconds on the
 * server's clock (hphi_server_clock); d_out (nullable, 2 nz doubles) receives
 * D(z_j) as re, im pairs.  Errors: HPHI_E_INVAL (bad options / request /
 * unknown id), HPHI_E_NOMEM, HPHI_E_CUDA; a request's own failure is in its
 * reply's status. */
typedef struct hphi_server hphi_server;
typedef struct hphi_server_opts {
    double mem_budget;     /* bytes of the device arena */
    int max_active;        /* recurrences (thread blocks) at once; 0: 2 x SMs */
    int chunk;             /* Lanczos steps per server step; 0: 16 */
    int64_t small_max_dim; /* larger problems use the grid lane; 0: 2^17 */
    int grid_workers;      /* grid-lane worker threads, each with its own stream; 0: 2 */
    int grid_dtype;        /* vector storage of the grid lane: HPHI_F64 (0, default) or
                              HPHI_F32 (scalars, reductions and the tridiagonal
                              problem stay FP64; the Lanczos recurrence runs to a
                              residual of max(tol, 1e-6), as FP32 vectors hold no
                              more; a ground-state request then also builds its
                              ground-state vector and reports the FP64 Rayleigh
                              quotient of it as e0, see e0_rq of
                              hphi_lanczos_result); the block lane is FP64 */
} hphi_server_opts;

#define HPHI_REQ_GROUND 0
#define HPHI_REQ_SPECTRUM 1

typedef struct hphi_request {
    int kind;
    hphi_ham *ham;
    uint64_t seed;
    int max_steps;
    double tol;
    double q, eta;        /* spectrum: wave number, broadening */
    int nz;               /* spectrum: number of shifts */
    const double *omega;  /* spectrum: [nz] frequencies above E0 */
} hphi_request;

typedef struct hphi_reply {
    int done, status, steps, krylov_steps, lane;
    double e0, max_resid;
    double t_submit, t_start, t_done;
} hphi_reply;

HPHI_API int hphi_server_create(hphi_ctx *ctx, const hphi_server_opts *opts, hphi_server **out);
HPHI_API void hphi_server_destroy(hphi_server *server);
HPHI_API double hphi_server_clock(const hphi_server *server);
HPHI_API int hphi_server_submit(hphi_server *server, const hphi_request *request, int64_t *id);
HPHI_API int hphi_server_step(hphi_server *server, int *n_running, int *n_queued);
HPHI_API int hphi_server_result(hphi_server *server, int64_t id, hphi_reply *reply, double *d_out);

/* Counters of a server: kernel launches of the block lane (steps, vector
 * passes, excitations, start vectors), requests finished per lane, requests
 * running per lane and queued, arena bytes in use and at most. */
typedef struct hphi_server_stats {
    int64_t block_launches, block_done, grid_done;
    int block_running, grid_running, queued;
    double arena_used, arena_peak;
} hphi_server_stats;
HPHI_API int hphi_server_get_stats(hphi_server *server, hphi_server_stats *stats);

/* ---- canonical TPQ step (Sec. 3.5.1) -----------------------------------------
 * One step Phi_{k+1} = U_c(dtau) Phi_k, U_c = sum_{n<=nmax} (-dtau H/2)^n / n!,
 * for nvec independent columns of V (device, dtype F64/F32/C128/C64, [D][nvec],
 * ld >= nvec), evaluated by Horner stages W <- sigma V + (-dtau/2)/j H W,
 * j = nmax .. 1, sigma = 1/sqrt(norm2_inout[q]).
 * In:  norm2_inout[q] = |V_q|^2 of the stored column (<= 0: computed here).
 * Out: e_host[q]  = <Phi_k|H|Phi_k> / <Phi_k|Phi_k>          (at beta_k)
 *      h2_host[q] = <H Phi_k|H Phi_k> / <Phi_k|Phi_k>
 *      logd_host[q] = log D_{k+1}, D_{k+1} = N_{k+1}/N_k (the relative squared
 *                     norm of the paper's Norm_n.dat)
 *      V_q <- Phi_{k+1} / |Phi_k| and norm2_inout[q] = |V_q|^2 = D_{k+1}.
 * The library holds two workspace blocks of V's size.  1 <= nmax <= 64. */
HPHI_API int hphi_tpq_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv, double dtau,
                  int nmax, double *norm2_inout, double *e_host, double *h2_host, double *logd_host);

/* ---- real-time evolution (Sec. 3.4) --------------------------------------------
 * One step Phi(t + dt) = sum_{n<=nmax} (-i dt H)^n / n! Phi(t) for nvec complex
 * columns of V (device, dtype C128 or C64, [D][nvec] complex, ld >= nvec),
 * evaluated by Horner stages W <- Phi + (-i dt / j) H W, j = nmax .. 1.
 * Out (host, per column, of the state before the step): norm2_host = <Phi|Phi>,
 * e_host = <Phi|H|Phi> / <Phi|Phi>, h2_host = <H Phi|H Phi> / <Phi|Phi>; and
 * norm2_new_host = <Phi(t + dt)|Phi(t + dt)> (the paper's accuracy check: it
 * stays equal to the old norm up to the truncation of the series).
 * V is overwritten with Phi(t + dt), not renormalised.  1 <= nmax <= 64,
 * 1 <= nvec <= 64.  The library holds two workspace blocks of V's size.
 * Errors: HPHI_E_INVAL, HPHI_E_NUMERIC (non-finite values), HPHI_E_CUDA. */
HPHI_API int hphi_time_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv, double dt,
                            int nmax, double *norm2_host, double *e_host, double *h2_host, double *norm2_new_host);

/* ---- dynamical correlation functions (Sec. 3.2) ------------------------------
 * D(z) = <Phi_ex| (z I - H)^{-1} |Phi_ex>, Phi_ex = O |Phi_0>; the spin
 * structure factor is S^zz(q, w) = -Im D(w + i eta) for O = sum_l e^{i q l} S^z_l.
 *
 * hphi_apply_sz_sum: y = sum_l A_l S^z_l x with complex weights
 * A_l = a_host[2l] + i a_host[2l+1] (l < n_sites; host array of 2 n_sites).
 * S^z_l = n_l - 1/2 for the spin models (bit l of the spin string) and
 * (n_{l up} - n_{l dn}) / 2 for Hubbard.  x: one real device vector (dtype
 * F64 or F32, element stride ldx >= 1); y: two real device columns of the
 * same dtype, y[r*ldy] = Re, y[r*ldy + 1] = Im (ldy >= 2; ldy = 2 is a complex
 * vector).  x and y must not overlap (HPHI_E_INVAL).  Asynchronous. */
HPHI_API int hphi_apply_sz_sum(hphi_ctx *ctx, const hphi_basis *basis, int dtype, const void *x, int64_t ldx, void *y,
                               int64_t ldy, const double *a_host);

/* hphi_shifted_krylov: D_c(z_j) = <b_c| (z_j I - H)^{-1} |b_c> for ncol real
 * right-hand sides b_c (device, [D][ldb], dtype F64 or F32, 1 <= ncol <= 64)
 * and nz complex shifts z_j = z_host[2j] + i z_host[2j+1], all from one
 * Krylov run per column (the columns share every launch).
 * Each column runs the Lanczos recurrence; the Galerkin solution of
 * (z - H) x = b on the m-step Krylov space gives
 *   D_c(z) = |b_c|^2 / (z - a_0 - b_1^2 / (z - a_1 - ... - b_{m-1}^2 / (z - a_{m-1})))
 * and the residual |b_c - (z - H) x| / |b_c| = prod_{k=1..m} b_k / |u_k(z)|,
 * u_1 = z - a_0, u_k = z - a_{k-1} - b_{k-1}^2 / u_{k-1}.  For real H and real
 * b_c this iterate is the shifted COCG iterate of the paper's CG method and
 * these residual norms are its convergence measure.  A complex excitation
 * Phi = a + i b is passed as the two real columns a and b: (z - H)^{-1} is
 * complex symmetric, so <Phi|G|Phi> = D_a + D_b.
 * The run stops when every (column, shift) residual is <= opts->tol
 * (checked every check_every steps), when every column has reached an
 * invariant subspace (beta_{k+1} <= 64 eps max_j(|a_j| + b_j + b_{j+1})), or
 * after max_steps.  Host outputs: g_host[2 (c nz + j) + {0, 1}] = Re, Im of
 * D_c(z_j); resid_host[c nz + j] (nullable); alpha_host[c max_steps + k] and
 * beta_host[c (max_steps + 1) + k] (nullable, zero past the column's steps;
 * beta[0] = |b_c|).  A zero column gives D = 0 and residual 0.
 * Returns HPHI_OK, HPHI_E_NOTCONV (tol > 0 not reached; outputs filled in),
 * HPHI_E_NUMERIC (non-finite scalars) or an error.  The library holds three
 * workspace blocks of D x ncol elements. */
typedef struct hphi_krylov_opts {
    int max_steps;
    double tol;      /* relative residual of every shift; <= 0 runs max_steps */
    int dtype;       /* HPHI_F64 or HPHI_F32 vectors (scalars are FP64) */
    int check_every; /* host residual checks every this many steps (>= 1) */
} hphi_krylov_opts;

typedef struct hphi_krylov_result {
    int steps;        /* Krylov steps taken */
    int converged;    /* 1 if the tolerance (or invariant subspaces) ended the run */
    double max_resid; /* largest relative residual over active columns and shifts */
} hphi_krylov_result;

HPHI_API int hphi_shifted_krylov(hphi_ctx *ctx, const hphi_ham *ham, const hphi_krylov_opts *opts, int ncol,
                                 const void *b, int64_t ldb, int nz, const double *z_host, double *g_host,
                                 double *resid_host, double *alpha_host, double *beta_host,
                                 hphi_krylov_result *result);

/* hphi_szz_spectrum: the spin structure factor of Sec. 3.2 for nq wave
 * numbers at once,
 *   D_q(z_j) = <Phi_q| (z_j I - H)^{-1} |Phi_q>,  Phi_q = sum_l e^{i q l} S^z_l Phi_0,
 *   S^zz(q, z_j) = -Im D_q(z_j),
 * with Phi_0 = gs (device, D elements of opts->dtype, F64 or F32, contiguous)
 * and the shifts z_j = z_host[2j] + i z_host[2j+1] (the caller adds E_0:
 * z = E_0 + omega + i eta).  Each Phi_q = a + i b is split into real columns
 * a and b (b is left out when sin(q l) vanishes for every site, |sin| <=
 * 1e-12), all columns share one hphi_shifted_krylov run (same opts, same
 * stopping rule), and D_q = D_a + D_b ((z - H)^{-1} is complex symmetric).
 * Host outputs: s_host[q nz + j] = S^zz; d_host (nullable) [q nz + j] as
 * (re, im) pairs; resid_host (nullable) [q nz + j] the larger relative
 * residual of the two columns; *result as hphi_shifted_krylov.
 * Limits: the columns (one or two per q) must number at most 64.  The
 * library allocates the excitation block (D x (columns + 1) elements) for the
 * call.  Returns HPHI_OK, HPHI_E_NOTCONV (outputs filled in) or an error. */
HPHI_API int hphi_szz_spectrum(hphi_ctx *ctx, const hphi_ham *ham, const hphi_krylov_opts *opts, const void *gs,
                               int nq, const double *q_host, int nz, const double *z_host, double *s_host,
                               double *d_host, double *resid_host, hphi_krylov_result *result);

/* ---- LOBPCG (Sec. 3.3) -------------------------------------------------------------
 * hphi_lobpcg: the m lowest eigenpairs (1 <= m <= 32) of H by the locally
 * optimal block conjugate gradient method (no preconditioner): each
 * iteration one block H*V of the residuals and a Rayleigh-Ritz step on
 * [R, Phi, P].  X: device FP64 [D][m] (leading dimension m), in: the start
 * block (full rank), out: the Ritz vectors (orthonormal columns).  Stops when
 * every residual |H x_n - e_n x_n| <= tol max(1, |e_n|), or after max_iter
 * iterations (HPHI_E_NOTCONV, outputs filled in).  Host outputs: evals_host[m]
 * ascending, resid_host[m], *iters.  Workspace: 9 D m doubles.
 * HPHI_E_NUMERIC if the Rayleigh-Ritz basis has rank below m (a rank-deficient
 * start block), HPHI_E_INVAL for D < 3 m. */
HPHI_API int hphi_lobpcg(hphi_ctx *ctx, const hphi_ham *ham, int m, void *X, int max_iter, double tol,
                         double *evals_host, double *resid_host, int *iters);

/* ---- microcanonical TPQ step (Sec. 3.5.1) ---------------------------------------
 * Phi_{k+1} = U_m Phi_k, U_m = 1 - (dtau/2) H with dtau = 2 / (l n_sites): the
 * cTPQ step above with nmax = 1 (same arguments, layout and outputs).  k is
 * the step index of the state the step starts from (Phi_0 = the random
 * start vector); beta_host (nullable, host, nvec) receives its inverse
 * temperature beta_k = k dtau / (1 - u_k / l), u_k = e_host[q] / n_sites.
 * l must exceed the largest eigenvalue of H / n_sites for U_m to be positive
 * on the spectrum.  HPHI_E_INVAL for l <= 0, n_sites < 1 or k < 0. */
HPHI_API int hphi_mtpq_step(hphi_ctx *ctx, const hphi_ham *ham, int dtype, int nvec, void *V, int64_t ldv, double l,
                            int n_sites, int k, double *norm2_inout, double *e_host, double *h2_host,
                            double *logd_host, double *beta_host);

/* ---- thermodynamics of TPQ samples: the bootstrap (Sec. 3.5.1) --------------------
 * From n_samples independent TPQ runs recorded at n_temps inverse
 * temperatures beta_k (host arrays, row-major [n_samples][n_temps]):
 *   e[n][k]  = <Phi|H|Phi> / <Phi|Phi> of sample n at beta_k,
 *   h2[n][k] = <Phi|H^2|Phi> / <Phi|Phi>,
 *   log_norm[n][k] = log <Phi|Phi> (any constant per k may be added: norms
 *            are taken relative to sample 0's, the paper's W(beta_k)),
 * M resamplings R_m of P sample indices each, drawn with replacement, give
 *   <A>_m = sum_{p} w_{R_m(p)} A_{R_m(p)} / sum_{p} w_{R_m(p)},
 *   w_n = exp(log_norm[n][k] - log_norm[0][k]),
 * and the outputs (host, n_temps each) are the mean over m and the standard
 * deviation sigma^2 = 1/(M-1) sum_m (x_m - mean)^2 (0 for M = 1) of
 *   E_m = <H>_m                         -> e_mean, e_sd
 *   C_m = beta_k^2 (<H^2>_m - <H>_m^2)  -> c_mean, c_sd (nullable pair; with
 *         beta NULL the factor beta_k^2 is left out).
 * picks (nullable, host, [M][P]) are the resamplings; with picks NULL they
 * are drawn from Philox4x32-10: pick e = m P + p is floor(U n_samples)
 * (at most n_samples - 1), U = (((w1 << 32) | w0) >> 11 + 0.5) 2^-53 of
 * output words w0, w1 for counter (e mod 2^32, e div 2^32, 0, 0) and key
 * (seed mod 2^32, seed div 2^32).  Host only; no GPU needed.
 * Errors: HPHI_E_INVAL (sizes < 1, a NULL input, a pick out of range),
 * HPHI_E_NUMERIC (non-finite weights or a zero weight sum). */
HPHI_API int hphi_tpq_bootstrap(int n_samples, int n_temps, const double *e, const double *h2,
                                const double *log_norm, const double *beta, int P, int M, const int32_t *picks,
                                uint64_t seed, double *e_mean, double *e_sd, double *c_mean, double *c_sd);

/* ---- host utility: symmetric tridiagonal eigenproblem ------------------------
 * All eigenvalues (ascending) of the n x n tridiagonal with diagonal a[0..n-1]
 * and off-diagonal b[1..n-1] (b[k] couples rows k-1 and k; b[0] unused), by the
 * implicit QL iteration with Wilkinson shifts; evecs (nullable, host n*n,
 * row-major) receives the eigenvectors as columns, each with a non-negative
 * first component.  This is the small problem of every Lanczos run (T_m of
 * alpha/beta).  Host memory only; no GPU needed.  HPHI_E_NUMERIC if the
 * iteration does not converge. */
HPHI_API int hphi_tridiag_eigen(int n, const double *a, const double *b, double *evals, double *evecs);

#ifdef __cplusplus
}
#endif
#endif /* HPHI_H */
