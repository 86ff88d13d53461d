// Batched small-problem Lanczos (batch.cu): the per-problem descriptor and the
// launchers that the batch entry point and the serving loop share.
#pragma once

#include "hphi_internal.cuh"

namespace hphi {

constexpr int kBatchThreads = 1024;          // threads per problem
constexpr int kBatchMaxTerms = 256;          // merged terms of one problem
constexpr size_t kBatchSmemBudget = 160 * 1024;

struct BProb {
    int model, nterms;
    int nlo_u, nlo_d;
    int nbits[2];              // bits of the up / down (spin: the only) string
    int64_t D, ddn;
    const uint32_t *ja_u, *ja_d;
    const uint64_t *jb_u, *jb_d;
    const uint32_t *rowstate;  // S^z sector: state of every row
    const uint32_t *st_u, *st_d;
    const DTerm *terms;
    const double *v0;
    int64_t v0_stride;         // element stride of the start vector (1: contiguous)
    double *diag;              // D: the diagonal of H (computed at step 0)
    int stage_x;               // x of the step staged in shared memory
    int stage_tab;             // rank tables (and Hubbard state lists) in shared memory
    double *w;                 // 3 D: the rotating Krylov vectors
    double *alpha, *beta2;     // alpha[k * stride], beta2[k * stride] (step-major over the batch)
    int stride;
    double *scal;              // [0] running max of |alpha_j| + beta_j + beta_{j+1}
    int *state;                // [0]: 0 running, 1 invariant subspace, 2 non-finite, 3 zero start; [1] steps
    int k0, nsteps;            // steps k0 .. k0 + nsteps - 1 in this launch
    // ground-state pass
    const double *y;           // Ritz vector of T_m
    int m;
    double theta;
    double *gs;
    double *resid;             // |H gs - theta gs|
    // optional per-launch staging (one read-back for every problem of a launch):
    // [0] beta_{k0}^2, [1 + 2s] alpha_{k0+s}, [2 + 2s] beta_{k0+s+1}^2, then the state pair
    double *stage;
};


// Fills the model-dependent fields (tables, terms, sizes, shared-memory
// staging) of a descriptor; returns the dynamic shared memory it needs.
size_t batch_fill(const hphi_ham *h, BProb &P);
// The S^z sector's row -> state table of a Hamiltonian (built on first use).
int ensure_rowstate(hphi_ctx *ctx, hphi_ham *ham);
// nsteps Lanczos steps of every descriptor (one thread block each).
int batch_launch_steps(hphi_ctx *ctx, const BProb *dprob, int n, size_t dyn);
// Ground-state pass of every descriptor with m > 0 and gs set.
int batch_launch_gs(hphi_ctx *ctx, const BProb *dprob, int n, size_t dyn);

}  // namespace hphi
