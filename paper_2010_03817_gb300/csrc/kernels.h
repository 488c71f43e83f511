// Internal interface between the C ABI (abi.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spg {

// per-chain / per-item status words (mirrored by SP_ST_* in spectra_gb.h)
enum ChainStatus : int {
  kOk = 0,
  kNotPD = 1,
  kUnbounded = 2,
  kNoConv = 3,
  kRho = 4,
  kDegenerate = 5,
};

// per-chain statistics slots (int64 each)
enum StatSlot : int {
  kStatSegments = 0,     // boundary-oracle calls
  kStatReflections = 1,  // reflections
  kStatBadSteps = 2,     // steps rejected (status != OK), point kept
  kStatLanczos = 3,      // Lanczos iterations
  kStatShiftRetry = 4,   // shifted factorisations that failed and were redone unshifted
  kStatNoConv = 5,       // eigen-solves that hit the iteration cap
  kNumStats = 8,
};

struct DevSpec {
  int n, m;
  long long P;             // m(m+1)/2
  const double* A;         // (n+1) x P, packed lower triangles of A_0..A_n
  const uint32_t* pidx;    // P entries: (i << 16) | k
};

struct DevWork {
  double* Vfull;  // per CTA: m*m
  double* Fg;     // per CTA: P
  double* Q;      // per CTA: kmax*m
  double* Lg;     // per CTA: P (only when the factor does not fit in shared memory)
  int kmax;
  double tol;     // Lanczos relative residual target
  int l_in_smem;
  int ctas;
};

struct WalkParams {
  int kind;          // 0 billiard, 1 hit-and-run, 2 cdhr
  int C;             // chains
  int steps;
  uint32_t step0;    // first step number (Philox counter)
  uint32_t chain0;   // Philox chain offset
  uint64_t seed;
  double tau, kappa, sigma_frac;
  int rho;
  double* X;         // C x n
  int* status;       // C
  long long* stats;  // C x kNumStats
};

struct PrimParams {
  int op;            // 0 intersect, 1 reflect, 2 membership
  int count;
  const double* x;   // count x n
  const double* v;   // count x n
  double* t_minus;   // count (intersect)
  double* t_plus;    // count
  double* u;         // count x m (intersect, optional)
  double* w_hat;     // count x n (reflect)
  double* s;         // count x n (reflect)
  int* status;       // count
  int* inside;       // count (membership)
};

size_t fp64_smem_bytes(int n, int m, bool l_in_smem);
cudaError_t launch_walk_fp64(const DevSpec& sp, const DevWork& wk, const WalkParams& wp,
                             cudaStream_t st);
cudaError_t launch_prim_fp64(const DevSpec& sp, const DevWork& wk, const PrimParams& pp,
                             cudaStream_t st);

}  // namespace spg
