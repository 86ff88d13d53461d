/*
 * CPU oracle for the matrix-free Hamiltonian-vector product of spin-1/2 and
 * Hubbard models and for the Lanczos and canonical-TPQ drivers built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library itself never
 * does, and it shares no code, header, table or constant with the library.
 *
 * Everything is FP64 and every loop runs in the order the definitions are
 * written: no blocking, fusion or reordering.  The optional OpenMP pragma only
 * splits the independent row loop of H*x across threads (each row is still
 * summed in term order by one thread).
 *
 * Model definitions (the paper writes the Hamiltonians in Sec. 3.1.1, the
 * equation of H_quench in Sec. 3.4 and Eq. ham_general in Sec. 5):
 *   spin-1/2:  H = sum_b [ Jz_b S^z_i S^z_j + Jxy_b (S^x_i S^x_j + S^y_i S^y_j) ]
 *              (EXCHANGE is the isotropic case Jz = Jxy = J)
 *   Hubbard:   H = - sum t (c^+_{i s} c_{j s} + h.c.) + U sum_i n_{i up} n_{i dn}
 *                  + sum V n_i n_j
 * Basis encoding (the paper is silent; its ver.1 predecessor holds it):
 *   bit i of a spin string = site i (1 = up spin / occupied site); the states
 *   of a sector are in ascending integer order; a Hubbard state is the pair
 *   (s_up, s_dn) with row = rank_up * D_dn + rank_dn; a fermion state is
 *   prod_{i asc, up occupied} c^+_{i up}  prod_{i asc, dn occupied} c^+_{i dn} |0>.
 *
 * Parity pins for every function here are in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

enum { ORC_SPIN = 0, ORC_SPIN_GC = 1, ORC_HUBBARD = 2 };
enum { ORC_EXCHANGE = 0, ORC_XXZ = 1, ORC_HOP = 2, ORC_HUBBARD_U = 3, ORC_DENS_DENS = 4 };

typedef struct {
    int32_t kind, i, j, spin;
    double v0, v1;
} orc_term;

/* ------------------------------------------------------------------------- */
/* Small integer helpers.                                                     */
/* ------------------------------------------------------------------------- */

static int orc_popcount(uint64_t x)
{
    int c = 0;
    while (x) {
        c += (int)(x & 1u);
        x >>= 1;
    }
    return c;
}

static int64_t binom_table[65][65];
static int binom_ready = 0;

/* Threads the OpenMP row loop of orc_apply uses (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Pascal's triangle, C(n, k) for 0 <= k <= n <= 64 (C(64, 32) < 2^63). */
int64_t orc_binom(int n, int k)
{
    if (!binom_ready) {
        for (int a = 0; a <= 64; a++)
            for (int b = 0; b <= 64; b++)
                binom_table[a][b] = 0;
        for (int a = 0; a <= 64; a++) {
            binom_table[a][0] = 1;
            for (int b = 1; b <= a; b++)
                binom_table[a][b] = binom_table[a - 1][b - 1] + binom_table[a - 1][b];
        }
        binom_ready = 1;
    }
    if (n < 0 || k < 0 || k > n || n > 64)
        return 0;
    return binom_table[n][k];
}

/* Dimension of a sector: C(N, n_up) spins with fixed S^z (Sec. 3.5.1: "x may
 * be the set of spin positions"), 2^N without it, C(N,n_up) C(N,n_dn) Hubbard. */
int64_t orc_dim(int model, int N, int nup, int ndn)
{
    if (model == ORC_SPIN)
        return orc_binom(N, nup);
    if (model == ORC_SPIN_GC)
        return (N >= 0 && N <= 40) ? ((int64_t)1 << N) : 0;
    if (model == ORC_HUBBARD)
        return orc_binom(N, nup) * orc_binom(N, ndn);
    return 0;
}

/* All N-bit strings with n set bits, ascending: a plain loop over 0 .. 2^N-1. */
int64_t orc_enumerate(int N, int n, uint64_t *out, int64_t cap)
{
    if (N < 0 || N > 40)
        return ORC_EINVAL;
    int64_t cnt = 0;
    uint64_t top = (uint64_t)1 << N;
    for (uint64_t s = 0; s < top; s++) {
        if (orc_popcount(s) == n) {
            if (cnt < cap)
                out[cnt] = s;
            cnt++;
        }
    }
    return cnt;
}

/* Position of s in an ascending list, by binary search; -1 if absent. */
int64_t orc_rank_search(const uint64_t *list, int64_t len, uint64_t s)
{
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (list[mid] == s)
            return mid;
        if (list[mid] < s)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* Position of s among the strings with the same number of set bits, in
 * ascending order.  For a fixed popcount, ascending integer order is
 * co-lexicographic order of the set-bit positions p_1 < ... < p_n, whose rank
 * is the combinatorial number system: sum_k C(p_k, k).  (Pinned against the
 * enumeration + binary search above in the tests.) */
int64_t orc_rank_colex(uint64_t s)
{
    int64_t r = 0;
    int k = 0;
    for (int p = 0; p < 64; p++) {
        if ((s >> p) & 1u) {
            k++;
            r += orc_binom(p, k);
        }
    }
    return r;
}

/* Inverse of orc_rank_colex for strings with n set bits. */
uint64_t orc_unrank_colex(int64_t r, int n)
{
    uint64_t s = 0;
    for (int k = n; k >= 1; k--) {
        int p = 63;
        while (orc_binom(p, k) > r)
            p--;
        s |= (uint64_t)1 << p;
        r -= orc_binom(p, k);
    }
    return s;
}

/* The two-table (Lin) index of a sector, written from its definition by
 * counting.  Low half: N_lo = N - floor(N/2) bits, high half floor(N/2) bits.
 *   ja[l] = #{ l' < l : popcount(l') == popcount(l) }
 *   jb[h] = #{ sector states s : (s >> N_lo) < h }, or all-ones if no sector
 *           state has high half h.
 * Then rank(s) = ja[s & (2^N_lo - 1)] + jb[s >> N_lo].  H. Q. Lin, Phys. Rev.
 * B 42, 6561 (1990); the paper leaves the encoding to its ver.1 predecessor. */
int orc_lin_tables(int N, int n, uint32_t *ja, uint64_t *jb)
{
    if (N < 2 || N > 40 || n < 0 || n > N)
        return ORC_EINVAL;
    int nlo = N - N / 2, nhi = N / 2;
    uint64_t Llo = (uint64_t)1 << nlo, Lhi = (uint64_t)1 << nhi;
    /* running count of the strings seen so far, per popcount */
    uint32_t seen[65];
    for (int p = 0; p <= 64; p++)
        seen[p] = 0;
    for (uint64_t l = 0; l < Llo; l++) {
        int p = orc_popcount(l);
        ja[l] = seen[p];
        seen[p]++;
    }
    /* running count of sector states whose high half is below h: a high half
     * h2 pairs with every low half of popcount n - popcount(h2) */
    uint64_t below = 0;
    for (uint64_t h = 0; h < Lhi; h++) {
        int need = n - orc_popcount(h);
        int valid = need >= 0 && need <= nlo;
        jb[h] = valid ? below : ~(uint64_t)0;
        if (valid)
            below += seen[need]; /* after the loop above: all low halves of that popcount */
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Model: sector + interaction list.                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int model, N, nup, ndn;
    int64_t D, Dup, Ddn;
    int nterms;
    orc_term *terms;
    /* optional ascending state lists; when present, ranks use binary search */
    uint64_t *list_up, *list_dn;
} orc_model;

static int term_ok(const orc_model *m, const orc_term *t)
{
    if (t->i < 0 || t->i >= m->N)
        return 0;
    switch (t->kind) {
    case ORC_EXCHANGE:
    case ORC_XXZ:
        return m->model != ORC_HUBBARD && t->j >= 0 && t->j < m->N && t->j != t->i;
    case ORC_HOP:
        return m->model == ORC_HUBBARD && t->j >= 0 && t->j < m->N && t->j != t->i &&
               (t->spin == 0 || t->spin == 1 || t->spin == -1);
    case ORC_HUBBARD_U:
        return m->model == ORC_HUBBARD;
    case ORC_DENS_DENS:
        return m->model == ORC_HUBBARD && t->j >= 0 && t->j < m->N && t->j != t->i;
    default:
        return 0;
    }
}

/* Create a model.  use_lists != 0 enumerates the sector and ranks by binary
 * search (small N); otherwise ranks use the combinatorial number system. */
orc_model *orc_model_create(int model, int N, int nup, int ndn, const orc_term *terms, int nterms,
                            int use_lists, int *status)
{
    *status = ORC_EINVAL;
    if (model < ORC_SPIN || model > ORC_HUBBARD || N < 1 || N > 64 || nterms < 0)
        return NULL;
    if (model == ORC_SPIN_GC && N > 40)
        return NULL;
    if (model == ORC_SPIN && (nup < 0 || nup > N))
        return NULL;
    if (model == ORC_HUBBARD && (nup < 0 || nup > N || ndn < 0 || ndn > N))
        return NULL;
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    if (!m) {
        *status = ORC_ENOMEM;
        return NULL;
    }
    m->model = model;
    m->N = N;
    m->nup = nup;
    m->ndn = ndn;
    m->D = orc_dim(model, N, nup, ndn);
    m->Dup = model == ORC_HUBBARD ? orc_binom(N, nup) : m->D;
    m->Ddn = model == ORC_HUBBARD ? orc_binom(N, ndn) : 1;
    m->nterms = nterms;
    m->terms = (orc_term *)malloc(sizeof(orc_term) * (size_t)(nterms > 0 ? nterms : 1));
    if (!m->terms) {
        free(m);
        *status = ORC_ENOMEM;
        return NULL;
    }
    memcpy(m->terms, terms, sizeof(orc_term) * (size_t)nterms);
    for (int k = 0; k < nterms; k++) {
        if (!term_ok(m, &m->terms[k])) {
            free(m->terms);
            free(m);
            return NULL;
        }
    }
    if (use_lists && model != ORC_SPIN_GC) {
        if (N > 30) {
            free(m->terms);
            free(m);
            return NULL;
        }
        m->list_up = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m->Dup);
        if (model == ORC_HUBBARD)
            m->list_dn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m->Ddn);
        if (!m->list_up || (model == ORC_HUBBARD && !m->list_dn)) {
            free(m->list_up);
            free(m->list_dn);
            free(m->terms);
            free(m);
            *status = ORC_ENOMEM;
            return NULL;
        }
        orc_enumerate(N, nup, m->list_up, m->Dup);
        if (model == ORC_HUBBARD)
            orc_enumerate(N, ndn, m->list_dn, m->Ddn);
    }
    *status = ORC_OK;
    return m;
}

void orc_model_free(orc_model *m)
{
    if (!m)
        return;
    free(m->list_up);
    free(m->list_dn);
    free(m->terms);
    free(m);
}

int64_t orc_model_dim(const orc_model *m) { return m->D; }

static uint64_t species_state(const orc_model *m, int species, int64_t r)
{
    const uint64_t *list = species ? m->list_dn : m->list_up;
    int n = species ? m->ndn : m->nup;
    if (list)
        return list[r];
    return orc_unrank_colex(r, n);
}

static int64_t species_rank(const orc_model *m, int species, uint64_t s)
{
    const uint64_t *list = species ? m->list_dn : m->list_up;
    if (list)
        return orc_rank_search(list, species ? m->Ddn : m->Dup, s);
    return orc_rank_colex(s);
}

/* Row -> basis state (s_up, s_dn); spin models use s_up only. */
void orc_row_state(const orc_model *m, int64_t r, uint64_t *su, uint64_t *sd)
{
    if (m->model == ORC_SPIN_GC) {
        *su = (uint64_t)r;
        *sd = 0;
    } else if (m->model == ORC_SPIN) {
        *su = species_state(m, 0, r);
        *sd = 0;
    } else {
        *su = species_state(m, 0, r / m->Ddn);
        *sd = species_state(m, 1, r % m->Ddn);
    }
}

/* Basis state -> row (-1 if the state is outside the sector). */
int64_t orc_state_row(const orc_model *m, uint64_t su, uint64_t sd)
{
    if (m->model == ORC_SPIN_GC)
        return (int64_t)su;
    if (m->model == ORC_SPIN) {
        if (orc_popcount(su) != m->nup)
            return -1;
        return species_rank(m, 0, su);
    }
    if (orc_popcount(su) != m->nup || orc_popcount(sd) != m->ndn)
        return -1;
    int64_t a = species_rank(m, 0, su), b = species_rank(m, 1, sd);
    if (a < 0 || b < 0)
        return -1;
    return a * m->Ddn + b;
}

static int bit(uint64_t s, int i) { return (int)((s >> i) & 1u); }

/* Sign of moving one fermion of a species between sites i and j with the
 * operator ordering above: (-1)^(number of occupied sites strictly between). */
static double hop_sign(uint64_t s, int i, int j)
{
    int lo = i < j ? i : j, hi = i < j ? j : i;
    int c = 0;
    for (int k = lo + 1; k < hi; k++)
        c += bit(s, k);
    return (c & 1) ? -1.0 : 1.0;
}

/* All matrix elements H[r][col] of row r, in term order: entry 0 is the
 * diagonal (sum of the diagonal parts of every term, term id -1); each
 * off-diagonal entry comes from one term acting on the row's state (a HOP on
 * both species gives its up entry, then its down entry).  signs (nullable)
 * receives the fermion sign of each entry: (-1)^(# occupied sites strictly
 * between i and j) for a hop, +1 for spin flips and the diagonal.  Returns
 * the count, or a negative status (a target outside the sector is an error). */
int orc_row_entries(const orc_model *m, int64_t r, int64_t *cols, double *vals, int32_t *tids, int8_t *signs,
                    int cap)
{
    uint64_t su, sd;
    orc_row_state(m, r, &su, &sd);
    int cnt = 1;
    double diag = 0.0;
    if (cap < 1)
        return ORC_EINVAL;
    for (int k = 0; k < m->nterms; k++) {
        const orc_term *t = &m->terms[k];
        int i = t->i, j = t->j;
        if (t->kind == ORC_EXCHANGE || t->kind == ORC_XXZ) {
            double Jz = t->v0;
            double Jxy = t->kind == ORC_EXCHANGE ? t->v0 : t->v1;
            /* S^z_i S^z_j = +1/4 for parallel, -1/4 for antiparallel spins */
            diag += bit(su, i) == bit(su, j) ? 0.25 * Jz : -0.25 * Jz;
            /* (S^+_i S^-_j + S^-_i S^+_j)/2 flips an antiparallel pair */
            if (bit(su, i) != bit(su, j) && Jxy != 0.0) {
                uint64_t s2 = su ^ (((uint64_t)1 << i) | ((uint64_t)1 << j));
                int64_t c = orc_state_row(m, s2, 0);
                if (c < 0)
                    return ORC_EINVAL;
                if (cnt >= cap)
                    return ORC_EINVAL;
                cols[cnt] = c;
                vals[cnt] = 0.5 * Jxy;
                tids[cnt] = k;
                if (signs)
                    signs[cnt] = 1;
                cnt++;
            }
        } else if (t->kind == ORC_HOP) {
            for (int sp = 0; sp < 2; sp++) {
                if (t->spin != -1 && t->spin != sp)
                    continue;
                uint64_t s = sp ? sd : su;
                /* c^+_i c_j + c^+_j c_i: nonzero iff exactly one of i, j occupied */
                if (bit(s, i) == bit(s, j) || t->v0 == 0.0)
                    continue;
                uint64_t s2 = s ^ (((uint64_t)1 << i) | ((uint64_t)1 << j));
                int64_t c = sp ? orc_state_row(m, su, s2) : orc_state_row(m, s2, sd);
                if (c < 0)
                    return ORC_EINVAL;
                if (cnt >= cap)
                    return ORC_EINVAL;
                double sg = hop_sign(s, i, j);
                cols[cnt] = c;
                vals[cnt] = -t->v0 * sg;
                tids[cnt] = k;
                if (signs)
                    signs[cnt] = sg < 0.0 ? -1 : 1;
                cnt++;
            }
        } else if (t->kind == ORC_HUBBARD_U) {
            diag += t->v0 * (double)(bit(su, i) * bit(sd, i));
        } else if (t->kind == ORC_DENS_DENS) {
            diag += t->v0 * (double)((bit(su, i) + bit(sd, i)) * (bit(su, j) + bit(sd, j)));
        }
    }
    cols[0] = r;
    vals[0] = diag;
    tids[0] = -1;
    if (signs)
        signs[0] = 1;
    return cnt;
}

/* Upper bound on entries per row. */
int orc_max_row_entries(const orc_model *m) { return 1 + 2 * m->nterms; }

/* The matrix pattern of rows [r0, r1) with entries of equal column merged
 * (summed) and sorted by column; the diagonal is always present.  rowptr has
 * r1-r0+1 entries.  Returns the total count or a negative status. */
int64_t orc_pattern(const orc_model *m, int64_t r0, int64_t r1, int64_t *rowptr, int64_t *cols, double *vals,
                    int64_t cap)
{
    int mx = orc_max_row_entries(m);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * (size_t)mx);
    double *v = (double *)malloc(sizeof(double) * (size_t)mx);
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)mx);
    if (!c || !v || !t) {
        free(c);
        free(v);
        free(t);
        return ORC_ENOMEM;
    }
    int64_t pos = 0;
    for (int64_t r = r0; r < r1; r++) {
        rowptr[r - r0] = pos;
        int n = orc_row_entries(m, r, c, v, t, NULL, mx);
        if (n < 0) {
            pos = n;
            break;
        }
        /* insertion sort by column (stable: term order kept among equals) */
        for (int a = 1; a < n; a++) {
            int64_t cc = c[a];
            double vv = v[a];
            int b = a - 1;
            while (b >= 0 && c[b] > cc) {
                c[b + 1] = c[b];
                v[b + 1] = v[b];
                b--;
            }
            c[b + 1] = cc;
            v[b + 1] = vv;
        }
        for (int a = 0; a < n; a++) {
            if (pos > rowptr[r - r0] && cols[pos - 1] == c[a]) {
                vals[pos - 1] += v[a];
                continue;
            }
            if (pos >= cap) {
                pos = ORC_EINVAL;
                goto done;
            }
            cols[pos] = c[a];
            vals[pos] = v[a];
            pos++;
        }
    }
    if (pos >= 0)
        rowptr[r1 - r0] = pos;
done:
    free(c);
    free(v);
    free(t);
    return pos;
}

/* y[r][:] = alpha * sum_col H[r][col] x[col][:] + beta * y[r][:] for rows
 * [r0, r1), pull form.  x and y are row-major [D][nvec] with leading
 * dimensions ldx, ldy.  beta == 0 overwrites y without reading it.  Each row's
 * sum runs in the entry order of orc_row_entries (diagonal first). */
int orc_apply(const orc_model *m, int nvec, const double *x, int64_t ldx, double *y, int64_t ldy, double alpha,
              double beta, int64_t r0, int64_t r1)
{
    int mx = orc_max_row_entries(m);
    int bad = 0;
#pragma omp parallel
    {
        int64_t *c = (int64_t *)malloc(sizeof(int64_t) * (size_t)mx);
        double *v = (double *)malloc(sizeof(double) * (size_t)mx);
        int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)mx);
        double *acc = (double *)malloc(sizeof(double) * (size_t)(nvec > 0 ? nvec : 1));
        if (!c || !v || !t || !acc) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t r = r0; r < r1; r++) {
                int n = orc_row_entries(m, r, c, v, t, NULL, mx);
                if (n < 0) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (int q = 0; q < nvec; q++)
                    acc[q] = 0.0;
                for (int a = 0; a < n; a++)
                    for (int q = 0; q < nvec; q++)
                        acc[q] += v[a] * x[c[a] * ldx + q];
                for (int q = 0; q < nvec; q++) {
                    double o = alpha * acc[q];
                    if (beta != 0.0)
                        o += beta * y[r * ldy + q];
                    y[r * ldy + q] = o;
                }
            }
        }
        free(c);
        free(v);
        free(t);
        free(acc);
    }
    return bad ? ORC_EINVAL : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Vector helpers (plain loops).                                              */
/* ------------------------------------------------------------------------- */

static double vdot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------- */
/* Symmetric tridiagonal eigenproblem: Sturm-sequence bisection + inverse     */
/* iteration (a textbook method; the GPU driver uses a different one).        */
/* T has diagonal a[0..m-1] and off-diagonal b[1..m-1] (b[k] couples k-1, k). */
/* ------------------------------------------------------------------------- */

/* Number of eigenvalues of T strictly below x (Sylvester inertia of T - x). */
int orc_sturm_count(int m, const double *a, const double *b, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (int k = 0; k < m; k++) {
        double bb = k > 0 ? b[k] * b[k] : 0.0;
        q = (a[k] - x) - (k > 0 ? bb / q : 0.0);
        if (q == 0.0)
            q = -1e-300; /* perturb an exact zero pivot */
        if (q < 0.0)
            cnt++;
    }
    return cnt;
}

/* The k-th smallest eigenvalue (k = 0, 1, ...) by bisection. */
double orc_tridiag_eig(int m, const double *a, const double *b, int k)
{
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; i++) {
        double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
        if (a[i] - r < lo)
            lo = a[i] - r;
        if (a[i] + r > hi)
            hi = a[i] + r;
    }
    double w = hi - lo;
    lo -= 1e-3 * w + 1e-300;
    hi += 1e-3 * w + 1e-300;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        if (orc_sturm_count(m, a, b, mid) > k)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* Unit eigenvector y of T for eigenvalue theta by inverse iteration with the
 * tridiagonal (Thomas) solve of (T - theta' I) z = y, theta' a hair off theta. */
int orc_tridiag_vec(int m, const double *a, const double *b, double theta, double *y)
{
    double *cp = (double *)malloc(sizeof(double) * (size_t)m);
    double *dp = (double *)malloc(sizeof(double) * (size_t)m);
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    if (!cp || !dp || !z) {
        free(cp);
        free(dp);
        free(z);
        return ORC_ENOMEM;
    }
    double scale = fabs(theta) + 1.0;
    double sh = theta - 1e-13 * scale;
    for (int i = 0; i < m; i++)
        y[i] = 1.0 / sqrt((double)m) * (1.0 + 0.01 * (double)(i % 7));
    for (int it = 0; it < 4; it++) {
        /* forward elimination (no pivoting) */
        for (int i = 0; i < m; i++) {
            double diag = a[i] - sh;
            double sub = i > 0 ? b[i] : 0.0;
            double denom = diag - (i > 0 ? sub * cp[i - 1] : 0.0);
            if (denom == 0.0)
                denom = 1e-300;
            cp[i] = (i + 1 < m ? b[i + 1] : 0.0) / denom;
            dp[i] = (y[i] - (i > 0 ? sub * dp[i - 1] : 0.0)) / denom;
        }
        z[m - 1] = dp[m - 1];
        for (int i = m - 2; i >= 0; i--)
            z[i] = dp[i] - cp[i] * z[i + 1];
        double nz = sqrt(vdot(m, z, z));
        for (int i = 0; i < m; i++)
            y[i] = z[i] / nz;
    }
    if (y[0] < 0.0)
        for (int i = 0; i < m; i++)
            y[i] = -y[i];
    free(cp);
    free(dp);
    free(z);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Lanczos (the paper's ground-state method, Sec. 1 and Table 1).             */
/* ------------------------------------------------------------------------- */

/* Textbook three-term Lanczos on the real symmetric H:
 *   v_0 = v0/|v0|, beta_0 = 0
 *   w = H v_k - beta_k v_{k-1};  alpha_k = <v_k, w>;  w -= alpha_k v_k
 *   beta_{k+1} = |w|;  v_{k+1} = w / beta_{k+1}
 * After every step (k+1 >= 2) the lowest eigenvalue theta of T_{k+1} and its
 * eigenvector y give the residual estimate beta_{k+1} |y_k|; the run stops when
 * it is <= tol * max(1, |theta|), when beta_{k+1} <= 64 eps max_j(|alpha_j| +
 * beta_j + beta_{j+1}) (an invariant subspace; the paper gives no rule),
 * or after max_steps.  tol <= 0 runs exactly max_steps steps.
 * If gs != NULL, a second pass regenerates v_k from v0 with the stored
 * alpha/beta and accumulates gs = sum_k y_k v_k (normalised).
 * Outputs alpha[0..steps-1], beta[0..steps] (beta[0] = 0).
 * Returns 0 converged, 1 max_steps reached, 2 invariant subspace, <0 error. */
int orc_lanczos(const orc_model *m, const double *v0, int max_steps, double tol, double *alpha, double *beta,
                int *steps_out, double *e0_out, double *resid_out, double *gs)
{
    int64_t D = m->D;
    double *vp = (double *)calloc((size_t)D, sizeof(double));
    double *vc = (double *)malloc(sizeof(double) * (size_t)D);
    double *w = (double *)malloc(sizeof(double) * (size_t)D);
    double *y = (double *)malloc(sizeof(double) * (size_t)(max_steps + 1));
    if (!vp || !vc || !w || !y) {
        free(vp);
        free(vc);
        free(w);
        free(y);
        return ORC_ENOMEM;
    }
    double n0 = sqrt(vdot(D, v0, v0));
    for (int64_t i = 0; i < D; i++)
        vc[i] = v0[i] / n0;
    beta[0] = 0.0;
    int status = 1, k;
    double theta = 0.0, resid = 0.0;
    for (k = 0; k < max_steps; k++) {
        if (orc_apply(m, 1, vc, 1, w, 1, 1.0, 0.0, 0, D) != ORC_OK) {
            status = ORC_EINVAL;
            break;
        }
        for (int64_t i = 0; i < D; i++)
            w[i] -= beta[k] * vp[i];
        alpha[k] = vdot(D, vc, w);
        for (int64_t i = 0; i < D; i++)
            w[i] -= alpha[k] * vc[i];
        beta[k + 1] = sqrt(vdot(D, w, w));
        int mm = k + 1;
        theta = orc_tridiag_eig(mm, alpha, beta, 0);
        orc_tridiag_vec(mm, alpha, beta, theta, y);
        resid = beta[k + 1] * fabs(y[mm - 1]);
        /* invariant subspace: beta below a few ulps of the scale of T */
        double tnorm = 0.0;
        for (int q = 0; q <= k; q++) {
            double r = fabs(alpha[q]) + beta[q] + beta[q + 1];
            if (r > tnorm)
                tnorm = r;
        }
        if (beta[k + 1] <= 64.0 * 2.220446049250313e-16 * tnorm) {
            status = 2;
            k++;
            break;
        }
        if (tol > 0.0 && mm >= 2 && resid <= tol * (fabs(theta) > 1.0 ? fabs(theta) : 1.0)) {
            status = 0;
            k++;
            break;
        }
        for (int64_t i = 0; i < D; i++) {
            vp[i] = vc[i];
            vc[i] = w[i] / beta[k + 1];
        }
    }
    if (status < 0) {
        free(vp);
        free(vc);
        free(w);
        free(y);
        return status;
    }
    int steps = k;
    *steps_out = steps;
    *e0_out = theta;
    *resid_out = resid;
    if (gs) {
        /* second pass: regenerate the Krylov vectors and accumulate */
        for (int64_t i = 0; i < D; i++) {
            vp[i] = 0.0;
            vc[i] = v0[i] / n0;
            gs[i] = 0.0;
        }
        for (int q = 0; q < steps; q++) {
            for (int64_t i = 0; i < D; i++)
                gs[i] += y[q] * vc[i];
            if (q + 1 == steps)
                break;
            orc_apply(m, 1, vc, 1, w, 1, 1.0, 0.0, 0, D);
            for (int64_t i = 0; i < D; i++) {
                double nv = (w[i] - alpha[q] * vc[i] - beta[q] * vp[i]) / beta[q + 1];
                vp[i] = vc[i];
                vc[i] = nv;
            }
        }
        double ng = sqrt(vdot(D, gs, gs));
        for (int64_t i = 0; i < D; i++)
            gs[i] /= ng;
    }
    free(vp);
    free(vc);
    free(w);
    free(y);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Canonical TPQ step (Sec. 3.5.1): U_c = sum_{n<=nmax} (-dtau H / 2)^n / n!  */
/* ------------------------------------------------------------------------- */

/* One cTPQ step for nvec independent columns of V.  A column has ncomp real
 * components (1: real vector, 2: complex vector stored re, im), so V is the
 * row-major real array [D][nvec * ncomp].  H is real, so it acts on each
 * component alike, and <a|b> below is the real inner product of the
 * component arrays (for complex vectors: Re<a|b>, which is the whole of
 * <Phi|H|Phi> for Hermitian H).  For each column Phi:
 *   e[q]  = <Phi|H|Phi> / <Phi|Phi>          (at the current beta_k)
 *   h2[q] = <H Phi|H Phi> / <Phi|Phi>
 *   Phi'  = sum_{n=0}^{nmax} (1/n!) (-dtau/2 H)^n Phi, term by term:
 *           T_0 = Phi, T_n = (-dtau/2)/n * H T_{n-1}, Phi' = sum_n T_n
 *   d[q]  = <Phi'|Phi'> / <Phi|Phi>          (relative squared norm D_{k+1})
 * and V[:, q] <- Phi' / |Phi'|.  Returns a status. */
int orc_tpq_step(const orc_model *m, int nvec, int ncomp, double *V, double dtau, int nmax, double *e, double *h2,
                 double *d)
{
    int64_t D = m->D;
    int64_t L = D * ncomp, ld = (int64_t)nvec * ncomp;
    double *phi = (double *)malloc(sizeof(double) * (size_t)L);
    double *term = (double *)malloc(sizeof(double) * (size_t)L);
    double *hterm = (double *)malloc(sizeof(double) * (size_t)L);
    double *acc = (double *)malloc(sizeof(double) * (size_t)L);
    if (!phi || !term || !hterm || !acc) {
        free(phi);
        free(term);
        free(hterm);
        free(acc);
        return ORC_ENOMEM;
    }
    int st = ORC_OK;
    for (int q = 0; q < nvec && st == ORC_OK; q++) {
        for (int64_t i = 0; i < D; i++)
            for (int c = 0; c < ncomp; c++)
                phi[i * ncomp + c] = V[i * ld + q * ncomp + c];
        double nn = vdot(L, phi, phi);
        st = orc_apply(m, ncomp, phi, ncomp, hterm, ncomp, 1.0, 0.0, 0, D);
        e[q] = vdot(L, phi, hterm) / nn;
        h2[q] = vdot(L, hterm, hterm) / nn;
        for (int64_t i = 0; i < L; i++) {
            term[i] = phi[i];
            acc[i] = phi[i];
        }
        for (int n = 1; n <= nmax && st == ORC_OK; n++) {
            st = orc_apply(m, ncomp, term, ncomp, hterm, ncomp, 1.0, 0.0, 0, D);
            double c = (-0.5 * dtau) / (double)n;
            for (int64_t i = 0; i < L; i++) {
                term[i] = c * hterm[i];
                acc[i] += term[i];
            }
        }
        double na = vdot(L, acc, acc);
        d[q] = na / nn;
        double inv = 1.0 / sqrt(na);
        for (int64_t i = 0; i < D; i++)
            for (int c = 0; c < ncomp; c++)
                V[i * ld + q * ncomp + c] = acc[i * ncomp + c] * inv;
    }
    free(phi);
    free(term);
    free(hterm);
    free(acc);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Excitation operator of the dynamical structure factor (Sec. 3.2):         */
/*   y = sum_l A_l S^z_l x,  A_l complex (A_l = e^{i q l} is the paper's      */
/* O_spin at wave number q).  S^z_l = n_l - 1/2 for spin-1/2 (bit l of the    */
/* spin string) and (n_{l up} - n_{l dn}) / 2 for Hubbard.  Rows [r0, r1)    */
/* only: x[r - r0] is the input of row r and y_re + i y_im its output.        */
/* ------------------------------------------------------------------------- */
int orc_apply_sz_sum(const orc_model *m, const double *a_re, const double *a_im, const double *x, double *y_re,
                     double *y_im, int64_t r0, int64_t r1)
{
    if (r0 < 0 || r1 > m->D || r0 > r1)
        return ORC_EINVAL;
    for (int64_t r = r0; r < r1; r++) {
        uint64_t su, sd;
        orc_row_state(m, r, &su, &sd);
        double f_re = 0.0, f_im = 0.0;
        for (int l = 0; l < m->N; l++) {
            double sz;
            if (m->model == ORC_HUBBARD)
                sz = 0.5 * ((double)((su >> l) & 1u) - (double)((sd >> l) & 1u));
            else
                sz = (double)((su >> l) & 1u) - 0.5;
            f_re += a_re[l] * sz;
            f_im += a_im[l] * sz;
        }
        y_re[r - r0] = f_re * x[r - r0];
        y_im[r - r0] = f_im * x[r - r0];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Real-time evolution (Sec. 3.4): Phi(t + dt) = sum_{n<=nmax} (-i dt H)^n / n! Phi(t). */
/* ------------------------------------------------------------------------- */

/* One step for nvec complex columns of V (row-major [D][nvec] complex, stored
 * re, im).  Term by term in complex arithmetic, H real:
 *   T_0 = Phi,  T_n = (-i dt / n) H T_{n-1},  Phi' = sum_{n=0}^{nmax} T_n,
 * where (-i c)(a + i b) = c b - i c a.  Outputs per column, for the state
 * before the step: norm2[q] = <Phi|Phi>, e[q] = <Phi|H|Phi> / <Phi|Phi>, and
 * norm2_new[q] = <Phi'|Phi'>.  V <- Phi' (not renormalised: the evolution is
 * unitary up to the truncation of the series). */
int orc_time_step(const orc_model *m, int nvec, double *V, double dt, int nmax, double *norm2, double *e,
                  double *norm2_new)
{
    int64_t D = m->D, ld = 2 * (int64_t)nvec;
    double *re = (double *)malloc(sizeof(double) * (size_t)D * 6);
    if (!re)
        return ORC_ENOMEM;
    double *im = re + D, *hre = re + 2 * D, *him = re + 3 * D, *are = re + 4 * D, *aim = re + 5 * D;
    int st = ORC_OK;
    for (int q = 0; q < nvec && st == ORC_OK; q++) {
        for (int64_t i = 0; i < D; i++) {
            re[i] = V[i * ld + 2 * q];
            im[i] = V[i * ld + 2 * q + 1];
            are[i] = re[i];
            aim[i] = im[i];
        }
        double nn = vdot(D, re, re) + vdot(D, im, im);
        st = orc_apply(m, 1, re, 1, hre, 1, 1.0, 0.0, 0, D);
        if (st == ORC_OK)
            st = orc_apply(m, 1, im, 1, him, 1, 1.0, 0.0, 0, D);
        norm2[q] = nn;
        e[q] = (vdot(D, re, hre) + vdot(D, im, him)) / nn;
        for (int n = 1; n <= nmax && st == ORC_OK; n++) {
            st = orc_apply(m, 1, re, 1, hre, 1, 1.0, 0.0, 0, D);
            if (st == ORC_OK)
                st = orc_apply(m, 1, im, 1, him, 1, 1.0, 0.0, 0, D);
            double c = dt / (double)n;
            for (int64_t i = 0; i < D; i++) {
                re[i] = c * him[i];
                im[i] = -c * hre[i];
                are[i] += re[i];
                aim[i] += im[i];
            }
        }
        norm2_new[q] = vdot(D, are, are) + vdot(D, aim, aim);
        for (int64_t i = 0; i < D; i++) {
            V[i * ld + 2 * q] = are[i];
            V[i * ld + 2 * q + 1] = aim[i];
        }
    }
    free(re);
    return st;
}
