// Internal interface between the C ABI (abi.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct sp_spec;
struct sp_chains;

struct sp_mlp;
// forward pass of the warm-start network on B rows of device features X;
// *Y receives the device output (B rows, leading dimension *ld)
int spg_mlp_infer(sp_mlp* q, int B, const float* X, cudaStream_t st, const float** Y, int* ld);
int spg_mlp_io(const sp_mlp* q, int* din, int* dout);

namespace spg {

// per-chain / per-item status words (mirrored by SP_ST_* in spectra_gb.h)
enum ChainStatus : int {
  kOk = 0,
  kNotPD = 1,
  kUnbounded = 2,
  kNoConv = 3,
  kRho = 4,
  kDegenerate = 5,
  kInvalid = 6,
};

// per-chain statistics slots (int64 each)
enum StatSlot : int {
  kStatSegments = 0,     // boundary-oracle calls
  kStatReflections = 1,  // reflections
  kStatBadSteps = 2,     // steps rejected (status != OK), point kept
  kStatLanczos = 3,      // Lanczos iterations
  kStatShiftRetry = 4,   // shifted factorisations that failed and were redone unshifted
  kStatNoConv = 5,       // eigen-solves that hit the iteration cap
  kStatFallback = 6,     // mixed path: FP64 Lanczos fallbacks
  kStatPower = 7,        // mixed path: power iterations next to the boundary
  kStatLearnedOk = 8,    // learned path: warm starts accepted by the certificate
  kStatLearnedMiss = 9,  // learned path: warm starts rejected (plain stage 1 instead)
  kNumStats = 12,
};

// Sampled record of the boundary-oracle calls of a walk (sp_record_segments):
// the k-th segment any chain completes (arrival order, one atomic ticket per
// segment) is written to slot k / every when k % every == 0 and k / every <
// cap.  Slot layout (3n + 8 doubles): p[n] (start of the segment), v[n]
// (direction), w_hat[n] (unit normal, zero unless the segment reflected),
// t_plus, t_minus (-inf unless computed), status, reflected (0 / 1), the
// chain's Philox index, the step number, the segment's index in its step
// and the solver path flags (kSegFlag*).
struct SegLog {
  double* buf;  // cap x (3n + 8), or null: no recording
  int cap;
  int every;
  int* count;   // segments seen so far (device)
};
constexpr int kSegExtra = 8;
enum SegFlag : int {
  kSegShiftRetry = 1,     // the shifted factorisation failed: a smaller shift was used
  kSegFallback = 2,       // mixed path: stage 2 fell back to FP64
  kSegLearnedOk = 4,      // learned path: the warm start was accepted
  kSegLearnedMiss = 8,    // learned path: the warm start was rejected
  kSegNoConv = 16,        // an eigen-solve hit its iteration cap
  kSegRefined = 32,       // a shift-invert refinement next to the boundary ran
};

struct DevSpec {
  int n, m;
  long long P;             // m(m+1)/2
  const double* A;         // (n+1) x P, packed lower triangles of A_0..A_n
  const uint32_t* pidx;    // P entries: (i << 16) | k
};

struct DevWork {
  double* Vfull;  // per CTA: m*m
  double* Fg;     // per CTA: P, Y = sum_{j>=1} p_j A_j of the current point (F = A_0 + Y)
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
  SegLog seg;
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
  // mixed reflect with the tensor-core normals: null vectors out (count x m,
  // zero rows where the oracle failed), then partial sums of w_j in
  double* Ubuf;
  const double* Wpart;
  int wtiles;
  // learned warm start (reflect): the network's (log(t+ / t_scale), u) per line
  const float* pred;
  int ld_pred;
  double t_scale, margin;
  int* learned_ok;  // optional device pair: warm starts accepted / rejected
};

size_t fp64_smem_bytes(int n, int m, bool l_in_smem);

// ---- mixed-precision path ----------------------------------------------------
struct MixWork {
  const float2* Ahl;        // (n+1) x P: the A stack as FP32 (hi, lo) pairs
  float* Q32;               // per CTA: kmax32 * m (FP32 Lanczos basis)
  double* Q64;              // per CTA: kmax64 * m (FP64 fallback basis)
  uint8_t* region_global;   // per CTA work region when it does not fit in shared memory
  float2* vdf;              // per CTA: P double-float entries of stage 2's V
  size_t region_bytes;
  int kmax32, kmax64, power_iters, learned_iters;
  double tol32, tol64, delta1, sigma_frac;
  int ctas;
  long long* prof;  // optional: per-CTA clock64 sums per stage (kProfSlots each)
};
constexpr int kProfSlots = 16;  // 0-6: stages, 8-11: Lanczos, 12-15: stage-2 iteration parts

struct MixWave {
  int kind, C, steps, rho;
  uint32_t step0, chain0;
  uint64_t seed;
  double tau, kappa;
  double* X;        // C x n current points
  double* Xstart;   // C x n start of the current step
  double* F;        // C x P carried F(x) (FP64 packed)
  const double* Vrows;  // count x P: V of the listed chains (FP64 packed)
  double* ell;      // C remaining Billiard length
  double* tprev;    // C previous t+ (0 at a step start)
  int* nrefl;       // C reflections in the current step
  int* done;        // C steps completed in this call
  int* id_cur;      // active chains of this wave
  double* dir_cur;  // their directions (count x n)
  int* count_cur;
  int* id_next;
  double* dir_next;
  int* count_next;
  int* status;
  long long* stats;
  // learned warm start: predictions for the listed chains (row r: log(t/t_scale), u)
  const float* pred;
  int ld_pred;
  double t_scale, margin;
  // recording of (features, targets) tuples for training
  float* rec_x;     // cap x 2n: (x * x_scale, v)
  float* rec_y;     // cap x (1 + m): (log(t+ / t_scale), u)
  int* rec_count;
  int rec_cap;
  double x_scale;
  // deferred normals (tensor-core contraction of the whole wave): per slot
  // the null vector (count x m), t+ and a pending flag; null: in-kernel
  double* Ubuf;
  double* Tbuf;
  int* pend;
  const double* Wpart;  // slot x (n+1) x wtiles partial sums of w_j
  int wtiles;
  SegLog seg;
  // F refresh: a chain whose carried F has taken kFRefresh updates (or whose
  // step was rejected) is listed for a fresh formation before the next wave
  int* fage;        // C updates since the last fresh formation
  int* ref_ids;     // chains listed for the next wave's formation of F
  int* ref_count;
  int* ticket;  // the wave's line counter (zero at launch): lines are taken in order, one per CTA at a time
};
// updates of a carried F between fresh formations: Billiard and Hit-and-Run,
// CDHR (whose update F + t A_j the paper prescribes)
constexpr int kFRefresh = 16, kFRefreshCdhr = 64;

size_t mixed_region_bytes(int n, int m);
cudaError_t launch_learned_features(const double* X, const double* dir, const int* id, int count,
                                    int n, double x_scale, float* feats, cudaStream_t st);
size_t mixed_smem_bytes(int n, int m, bool region_in_smem);
cudaError_t launch_mixed_begin(const DevSpec& sp, const MixWave& wv, cudaStream_t st);
cudaError_t launch_mixed_reflect(const DevSpec& sp, const MixWave& wv, int count, int ctas,
                                 cudaStream_t st);
cudaError_t launch_prim_reflect_finish(const DevSpec& sp, const PrimParams& pp, int ctas,
                                       cudaStream_t st);
cudaError_t launch_mixed_wave(const DevSpec& sp, const MixWork& mw, const MixWave& wv,
                              cudaStream_t st);
cudaError_t launch_prim_mixed(const DevSpec& sp, const MixWork& mw, const PrimParams& pp,
                              const double* Frows, const double* Vrows, cudaStream_t st);

// pencil formation: Y[r, :] = lead * A_0 + sum_j vec[r, j] A_{j+1} (packed)
cudaError_t launch_form64(const double* A, long long P, int n, const double* vec, int R,
                          double lead, double* Y, long long ldy, cudaStream_t st);
// the same on the BF16 tensor cores with the exact digit splitting
int ozaki_kp(int n);
size_t ozaki_b_bytes(long long P, int n);
size_t ozaki_row_bytes(int R, int n);
void ozaki_slice_stack(const double* packed, int n, long long P, uint16_t* Bsl, int* ecol);
// rows (optional): coefficient row r is vec[rows[r]] and its result goes to
// Y[rows[r]]; count_dev (optional, device): only rows r < *count_dev
cudaError_t launch_ozaki_form(const double* vec, int R, int n, double lead, const double* A0,
                              const uint16_t* Bsl, const int* ecol, long long P, void* row_digits,
                              int* erow, double* Y, long long ldy, int* err, cudaStream_t st,
                              const int* rows = nullptr, const int* count_dev = nullptr);
constexpr int kOzakiMaxK = 224;  // n limit of the tensor-core formation (m for the contraction)
// the normal forms w_j = u^T A_j u of R null vectors on the tensor cores:
// (A_j u)_i by the same digit-split GEMM over the rows (j, i) of the full
// matrices (K = m), folded with u_i into per-tile partial sums
// Wpart[(r (n+1) + j) (ozaki_mpad(m) / 32) + tile]
int ozaki_mpad(int m);
size_t ozaki_contract_bytes(int n, int m);
cudaError_t launch_ozaki_slice_full(const double* A, int n, int m, long long P, uint16_t* Bc,
                                    int* ecolc, cudaStream_t st);
cudaError_t launch_ozaki_contract(const double* U, int R, int n, int m, const uint16_t* Bc,
                                  const int* ecolc, void* row_digits, int* erow, double* Wpart,
                                  int* err, cudaStream_t st);

// BF16 GEMM on tcgen05: C = A B^T (+ bias) (ReLU); FP32 and / or BF16 output
cudaError_t launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                             const float* bias, int relu, float* C32, int ldc32, void* C16,
                             int ldc16, int* err, cudaStream_t st);
// MLP helpers (mlp.cu)
cudaError_t launch_f32_to_bf16(const float* in, void* out, long long n, cudaStream_t st);
cudaError_t launch_f32_to_bf16_pad(const float* in, int B, int din, int dinp, void* out,
                                   cudaStream_t st);
cudaError_t launch_transpose_bf16(const void* in, int R, int C, int ldi, void* out, int ldo,
                                  cudaStream_t st);
cudaError_t launch_loss_grad(const float* Y, const float* T, int B, int D, int ld, void* dY16,
                             float* loss_acc, cudaStream_t st);
cudaError_t launch_relu_back(void* dH, const void* H, long long n, cudaStream_t st);
cudaError_t launch_col_sum(const void* dZ, int R, int C, int ld, float* g, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, long long n, float lr,
                        float b1, float b2, float c1, float c2, float eps, void* p16, void* pt16,
                        int rows, int cols, cudaStream_t st);
cudaError_t launch_walk_fp64(const DevSpec& sp, const DevWork& wk, const WalkParams& wp,
                             cudaStream_t st);
cudaError_t launch_prim_fp64(const DevSpec& sp, const DevWork& wk, const PrimParams& pp,
                             cudaStream_t st);

// ---- a batch of spectrahedra in one persistent launch (FP64 path) ----------
struct BatchBody {
  DevSpec sp;
  int l_in_smem;   // 1: the factor fits in shared memory
  int panel;       // Cholesky panel width of this body (4, 8 or 16)
  double tau;      // Billiard length scale
  long long xoff;  // first double of the body's chain points in X
  int c0;          // first global chain index (Philox chain, status, stats)
  int C;           // chains of the body
};
struct BatchParams {
  const BatchBody* bodies;
  const int2* items;  // (body, chain within the body) in the order they are handed out
  int total;
  int* next;          // work-queue ticket (zero before the launch)
  int steps;
  uint32_t step0;
  uint64_t seed;
  double kappa, sigma_frac;
  int rho;
  double* X;          // all chains' points, body by body
  int* status;        // total
  long long* stats;   // total x kNumStats
  // per-CTA work space sized for the largest body
  double* Vfull;
  double* Fg;
  double* Q;
  double* Lg;
  long long max_mm, max_P;
  int max_m, kmax;
  double tol;
};
size_t batch_smem_bytes(int n, int m, bool l_in_smem);
cudaError_t launch_batch_fp64(const BatchParams& bp, int ctas, size_t smem, cudaStream_t st);
// REFLECTION of `count` lines with the Cholesky panel width `panel`, for the
// panel tuner (FP64 path)
cudaError_t launch_prim_fp64_panel(const DevSpec& sp, const DevWork& wk, const PrimParams& pp,
                                   int panel, cudaStream_t st);
DevSpec spec_dev(const sp_spec* s);
// a chain set's device state for walk drivers outside abi.cu
struct ChainState {
  double* X;
  int* status;
  long long* stats;
  int C;
  uint64_t seed;
  uint32_t chain0, step;
  sp_spec* spec;
};
ChainState chain_state(sp_chains* ch);
void chain_advance(sp_chains* ch, uint32_t steps);  // the step counter moves on

// ---- HMC with reflections on the degree-2 Boltzmann trajectory (hmc.cu) ----
struct CurveParams {
  int op;            // 0 reflect lines (primitive), 1 walk
  int count;         // lines (op 0) or chains (op 1)
  const double* x;   // op 0: count x n start points
  const double* v;   // op 0: count x n initial velocities
  const double* c;   // n: the Boltzmann density's linear coefficient
  const double* Cp;  // P: packed C = -(1/(2T)) sum c_j A_j
  double T;
  double* t_plus;    // op 0
  double* w_hat;     // op 0: count x n
  double* s;         // op 0: count x n
  int* status;       // count
  // walk (op 1)
  double* X;
  long long* stats;
  int steps;
  uint32_t step0, chain0;
  uint64_t seed;
  double tau, kappa;
  int rho;
};
size_t curve_smem_bytes(int n, int m);
cudaError_t launch_curve(const DevSpec& sp, const CurveParams& cp, int ctas, cudaStream_t st);
constexpr int kCurveMaxM = 64;  // the companion matrix (2m x 2m) lives in shared memory

// library internals for the host drivers (abi.cu): the packed LMI stack
// ((n+1) x P doubles) copied to the host, and the device array of a chain
// set's points (C x n)
int spec_copy_stack(const sp_spec* s, double* packed_host);
const double* chain_points(const sp_chains* ch);
const double* chain_points(const sp_chains* ch, int* C, int* n);

}  // namespace spg
