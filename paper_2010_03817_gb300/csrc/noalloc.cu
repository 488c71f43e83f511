// Allocation-free INTERSECTION entry point.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or under a strict allocator policy, real-time loops
// that must not touch the driver's allocator, and plug-ins whose host process
// owns every device allocation.  For them sp_intersect_noalloc computes the
// same t-/t+ as sp_intersect without any allocation of its own: the caller
// passes the packed LMI stack, the lines and the outputs, and the kernel's
// working memory is a fixed file-scope device array of this library.
//
// That array (kScratchDoubles doubles, 8 MiB) exists on every GPU that loads
// the library, for as long as the library stays loaded.  Its device address
// is looked up once per device, on the first call made with that device
// current; make that first call before any stream capture.  Every call
// shares the one array and it keeps the previous call's contents: the
// kernel writes everything it reads, and calls that overlap on the GPU (two
// streams, two host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/spectra_gb.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 20;  // 8 MiB
__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// (i << 16) | k for every packed element, written into the scratch each call
__global__ void fill_pair_index(uint32_t* pidx, int m) {
  for (int i = blockIdx.x; i < m; i += gridDim.x)
    for (int k = threadIdx.x; k <= i; k += blockDim.x)
      pidx[spg::tri(i, k)] = ((uint32_t)i << 16) | (uint32_t)k;
}

}  // namespace

extern "C" int spg_set_error(int code, const char* msg);  // defined in abi.cu

extern "C" int sp_intersect_noalloc(int n, int m, const double* A_packed, int count,
                                    const double* x, const double* v, double* t_minus,
                                    double* t_plus, int* status, void* stream) {
  if (n < 1 || m < 1 || m > 4096 || count < 0)
    return spg_set_error(SP_EINVAL, "sp_intersect_noalloc: bad n, m or count");
  if (count == 0) return SP_OK;
  if (!A_packed || !x || !v || !t_minus || !t_plus || !status)
    return spg_set_error(SP_EINVAL, "sp_intersect_noalloc: null argument");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return spg_set_error(SP_ECUDA, "sp_intersect_noalloc: no current device");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return spg_set_error(SP_ECUDA, "sp_intersect_noalloc: scratch address lookup failed");
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    base = g_scratch_addr[dev];
  }
  // the factor must fit in shared memory (no global factor buffer here)
  int optin = 0, sms = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (spg::fp64_smem_bytes(n, m, true) > (size_t)optin)
    return spg_set_error(SP_EINVAL, "sp_intersect_noalloc: m too large for this entry point");
  const long long P = (long long)m * (m + 1) / 2;
  const int kmax = 96;
  const size_t pidx_doubles = (size_t)(P + 1) / 2;
  const size_t per_cta = (size_t)m * m + (size_t)P + (size_t)kmax * m;
  if (pidx_doubles + per_cta > kScratchDoubles)
    return spg_set_error(SP_EINVAL,
                            "sp_intersect_noalloc: problem exceeds the 8 MiB static scratch");
  int ctas = (int)((kScratchDoubles - pidx_doubles) / per_cta);
  if (ctas > sms) ctas = sms;
  if (ctas > count) ctas = count;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* pidx = reinterpret_cast<uint32_t*>(base);
  double* ws = base + pidx_doubles;
  fill_pair_index<<<m < 1024 ? m : 1024, 128, 0, st>>>(pidx, m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return spg_set_error(SP_ECUDA, "sp_intersect_noalloc: index kernel launch failed");
  spg::DevSpec sp;
  sp.n = n;
  sp.m = m;
  sp.P = P;
  sp.A = A_packed;
  sp.pidx = pidx;
  spg::DevWork wk;
  wk.Vfull = ws;
  wk.Fg = ws + (size_t)ctas * m * m;
  wk.Q = wk.Fg + (size_t)ctas * P;
  wk.Lg = nullptr;
  wk.kmax = kmax;
  wk.tol = 1e-13;
  wk.l_in_smem = 1;
  wk.ctas = ctas;
  spg::PrimParams pp{};
  pp.op = 0;
  pp.count = count;
  pp.x = x;
  pp.v = v;
  pp.t_minus = t_minus;
  pp.t_plus = t_plus;
  pp.u = nullptr;
  pp.status = status;
  e = spg::launch_prim_fp64(sp, wk, pp, st);
  if (e != cudaSuccess)
    return spg_set_error(SP_ECUDA, "sp_intersect_noalloc: kernel launch failed");
  return SP_OK;
}
