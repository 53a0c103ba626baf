// scqr3_internal.cuh -- shared definitions of the sm_103a kernels.
//
// Storage of the small n x n matrices (Gram A, per-pass factor R_k, product
// R): "packed upper, row-major" over the padded size NP. Row j holds entries
// (j, j), (j, j+1), ..., (j, NP-1); its start is pk_row(NP, j).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/scqr3.h"

namespace scqr3 {

__host__ __device__ constexpr int pk_size(int np) { return np * (np + 1) / 2; }
__host__ __device__ constexpr int pk_row(int np, int j) { return j * np - (j * (j - 1)) / 2; }
__host__ __device__ constexpr int pk_idx(int np, int j, int k) { return pk_row(np, j) + (k - j); }

// Device-side control block of one factorization. It lives at the start of
// the workspace; the public scqr3_info mirrors the user-visible fields.
struct DevState {
  int status;          // SCQR3_OK or a failure code (first failure wins)
  int passes;          // factors R_k computed so far
  int plain_in_a_row;  // consecutive unshifted passes ending at the last one
  int pad0;
  int run_trsm[SCQR3_MAX_PASSES];    // pass k's solve Q := Q R_k^{-1} runs
  int gram_after[SCQR3_MAX_PASSES];  // ...and accumulates the next Gram
  double normb;                      // ||B||_2 (or its bound) for the shift
  double normb_bits_max;             // scratch for the device max of ||B_j||_F
};

// Parameters of a factorization that every kernel needs (passed by value).
struct Params {
  int64_t m;
  int n;
  int np;            // padded n: 16, 32, 64, 128 or 256
  int max_passes;
  int bs;            // 0: B = I; else block size of B
  double norm_x2;    // opts.norm_x2
  double normb_in;   // B->norm2 (<= 0: compute)
  double shift_scale;  // opts.shift_scale (<= 0: Eq. (finds2)/(finds2B) only)
  int algorithm;       // 2 (Alg. 2) or 3 (Alg. 3)
  double tol;          // Alg. 2 stopping tolerance (resolved on the host, > 0)
  int csr;             // 1: B in CSR form (csr_gram_kernel forms Q^T B Q)
  int tc;              // 1: Gram matrices on the tensor cores (tc_gram_kernel)
  int solve_only;      // 1: the pass kernel only solves; a separate kernel forms the Gram
  long long wait_ns;       // limit (ns) of the hand-off waits in the tensor-core substitution kernels
  long long wait_ns_gram;  // ... and in the tensor-core Gram kernel
};

// The factorization uses an oblique inner product (block-diagonal or CSR B).
__host__ __device__ inline bool is_oblique(const Params& P) { return P.bs > 0 || P.csr != 0; }

// Params fields set from the options (shared by the single and batched paths).
void set_options(Params* P, const scqr3_opts* opts);

// Workspace carve-up (byte offsets from the base, each 256-aligned).
struct Layout {
  size_t state, gram, rstack, racc, chol, lt, partials, total;
  size_t rdev, infodev;  // host-buffer entry point: R and info on the device
  int n_partials;    // partial Gram slots used by this call (grid CTAs x groups)
  int csr_grid;      // CTAs of csr_gram_kernel (CSR form only)
  int tc_grid;       // CTAs of tc_gram_kernel (tensor-core Gram only)
  size_t colmax;     // tensor-core Gram: per-column max |q_ij| (128 words)
  size_t tcr;        // tensor-core substitution: the diagonal blocks of R_k packed 32 x 32 (8 x 528 doubles)
  int part_stride;   // doubles per partial slot: pk_size(np) + 1 (||.||_F^2)
};

constexpr int kThreads = 256;   // threads of the pass kernel

// Launch geometry of the FP64 pass kernel for a padded size.
struct PassGeom {
  int np, pr, groups, group_threads, h, c;
  size_t smem;
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace scqr3
