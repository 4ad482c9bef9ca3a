// srhd_cfl_dt_noalloc: the CFL time step of a batch of interior patches
// without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc. Typical cases are a
// host application whose device memory is entirely owned by its own pool
// allocator (every byte must come from that pool, so a library may not
// allocate behind its back), and time-step loops that must never make the
// device synchronise (cudaMalloc and cudaFree can synchronise implicitly).
// srhd_cfl_dt needs a context, and creating a context allocates its scratch;
// this entry point needs neither.
//
// Where its scratch lives: a file-scope static __device__ array, sized for
// at most kMaxPatches patches, that every GPU which loads the library keeps
// until the process exits (1.5 MB per device). In host code the array's
// name is only a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress once per device, the first time the entry point
// is called with that device current, and cached. That first call should
// therefore be made before any stream capture begins.
//
// All calls share the one array and each call leaves its per-patch results
// in it; calls whose kernels overlap on the GPU (for example on two
// streams) race on it and must be serialised by the caller. Every call
// writes all the slots it later reads, so nothing needs clearing.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "srhd.h"
#include "srhd_physics.cuh"

namespace srhd {
void set_last_error(const char* msg);  // srhd_api.cu
}

namespace {

constexpr int kMaxPatches = 1 << 17;   // 131072 patches of 8^3 cells
constexpr int kMaxDevices = 64;
constexpr int kCells = 512;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_patch_dt[kMaxPatches];
static __device__ __align__(256) int32_t g_patch_bad[kMaxPatches];

std::mutex g_mu;
double* g_dt_addr[kMaxDevices] = {};
int32_t* g_bad_addr[kMaxDevices] = {};

// One block per patch: the minimum of C dh / S_max over its 512 cells (or
// C dh in light-speed mode) and a flag for unphysical cells.
template <class P, class E>
__global__ void __launch_bounds__(kThreads) patch_cfl_kernel(const typename P::S* cons, double dh,
                                                             double cfl, int ndim, int mode,
                                                             int maxit, double* patch_dt,
                                                             int32_t* patch_bad, int ori, E eos) {
  using S = typename P::S;
  using R = S;
  __shared__ double s_m[kThreads / 32];
  __shared__ int s_b[kThreads / 32];
  const S* base = cons + (size_t)blockIdx.x * 5 * kCells;
  double m = DBL_MAX;
  int bad = 0;
  for (int c = threadIdx.x; c < kCells; c += kThreads) {
    srhd::PrimX<R> W;
    int st = srhd::con2pri<P>(base[c], base[kCells + c], base[2 * kCells + c],
                              base[3 * kCells + c], base[4 * kCells + c], W, maxit,
                              S(0), ori, eos);
    if (st == 1) { bad = 1; continue; }
    m = (mode == 1) ? fmin(m, cfl * dh)
                    : fmin(m, cfl * dh / double(srhd::smax_of(W, ndim, eos)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { s_m[threadIdx.x >> 5] = m; s_b[threadIdx.x >> 5] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = DBL_MAX;
    int bb = 0;
    for (int w = 0; w < kThreads / 32; ++w) { mm = fmin(mm, s_m[w]); bb |= s_b[w]; }
    patch_dt[blockIdx.x] = mm;
    patch_bad[blockIdx.x] = bb;
  }
}

// One block: minimum over the n per-patch values; NaN if any patch had an
// unphysical cell, +inf for an empty batch.
__global__ void __launch_bounds__(kThreads) patch_cfl_reduce_kernel(const double* patch_dt,
                                                                    const int32_t* patch_bad,
                                                                    int n, double* dt_out) {
  __shared__ double s_m[kThreads / 32];
  __shared__ int s_b[kThreads / 32];
  double m = DBL_MAX;
  int b = 0;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    m = fmin(m, patch_dt[i]);
    b |= patch_bad[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    b |= __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { s_m[threadIdx.x >> 5] = m; s_b[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = DBL_MAX;
    int bb = 0;
    for (int w = 0; w < kThreads / 32; ++w) { mm = fmin(mm, s_m[w]); bb |= s_b[w]; }
    if (bb) mm = __longlong_as_double(0x7ff8000000000000ULL);
    else if (mm == DBL_MAX) mm = __longlong_as_double(0x7ff0000000000000ULL);
    dt_out[0] = mm;
  }
}

template <class P, class E>
void launch_patch_cfl(const void* cons, int32_t npatch, double dh, const srhd_params& p, int maxit,
                      double* patch_dt, int32_t* patch_bad, int ori, E eos, cudaStream_t s) {
  patch_cfl_kernel<P, E><<<npatch, kThreads, 0, s>>>(
      static_cast<const typename P::S*>(cons), dh, p.cfl, p.ndim, p.cfl_mode, maxit, patch_dt,
      patch_bad, ori, eos);
}

template <class P>
void launch_patch_cfl(const void* cons, int32_t npatch, double dh, const srhd_params& p, int maxit,
                      double* patch_dt, int32_t* patch_bad, int ori, cudaStream_t s) {
  if (p.eos == SRHD_EOS_POLYTROPIC)
    launch_patch_cfl<P>(cons, npatch, dh, p, maxit, patch_dt, patch_bad, ori,
                        srhd::EosPoly{p.gamma}, s);
  else
    launch_patch_cfl<P>(cons, npatch, dh, p, maxit, patch_dt, patch_bad, ori, srhd::EosTM{}, s);
}

srhd_status noalloc_fail(srhd_status st, const char* msg) {
  char buf[256];
  snprintf(buf, sizeof(buf), "srhd_cfl_dt_noalloc: %s", msg);
  srhd::set_last_error(buf);  // reported by srhd_last_error()
  return st;
}

// Device addresses of the static scratch on the current device, looked up
// once per device.
srhd_status scratch_for_current_device(double** dt_addr, int32_t** bad_addr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(SRHD_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SRHD_ERR_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dt_addr[dev]) {
    void* a = nullptr;
    void* b = nullptr;
    e = cudaGetSymbolAddress(&a, g_patch_dt);
    if (e != cudaSuccess) return noalloc_fail(SRHD_ERR_CUDA, cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&b, g_patch_bad);
    if (e != cudaSuccess) return noalloc_fail(SRHD_ERR_CUDA, cudaGetErrorString(e));
    g_dt_addr[dev] = static_cast<double*>(a);
    g_bad_addr[dev] = static_cast<int32_t*>(b);
  }
  *dt_addr = g_dt_addr[dev];
  *bad_addr = g_bad_addr[dev];
  return SRHD_OK;
}

}  // namespace

extern "C" srhd_status srhd_cfl_dt_noalloc(srhd_prec prec, const void* cons, int32_t npatch,
                                           double dh, const srhd_params* params, double* dt_out,
                                           void* stream) {
  srhd_params p;
  if (params) p = *params; else srhd_default_params(&p);
  if (prec != SRHD_FP64 && prec != SRHD_MIXED && prec != SRHD_MIXED_CF)
    return noalloc_fail(SRHD_ERR_ARG, "invalid precision");
  if (npatch < 0) return noalloc_fail(SRHD_ERR_ARG, "npatch < 0");
  if (npatch > kMaxPatches)
    return noalloc_fail(SRHD_ERR_ARG,
                        "npatch exceeds the static scratch capacity of 131072 patches");
  if (!dt_out) return noalloc_fail(SRHD_ERR_ARG, "dt_out is NULL");
  if (npatch > 0 && !cons) return noalloc_fail(SRHD_ERR_ARG, "cons is NULL");
  if (!(dh > 0.0) || !std::isfinite(dh)) return noalloc_fail(SRHD_ERR_ARG, "dh must be positive");
  if (!(p.cfl > 0.0) || !(p.cfl <= 1.0)) return noalloc_fail(SRHD_ERR_ARG, "cfl must be in (0, 1]");
  if (p.ndim < 1 || p.ndim > 3) return noalloc_fail(SRHD_ERR_ARG, "ndim must be 1, 2 or 3");
  if (p.cfl_mode != SRHD_CFL_SIGNAL && p.cfl_mode != SRHD_CFL_LIGHT)
    return noalloc_fail(SRHD_ERR_ARG, "invalid cfl_mode");
  if (p.newton_max_iter < 0 || p.newton_max_iter > 1000)
    return noalloc_fail(SRHD_ERR_ARG, "newton_max_iter must be in [0, 1000]");
  if (p.scheme != SRHD_SCHEME_REDUCED && p.scheme != SRHD_SCHEME_TOTAL)
    return noalloc_fail(SRHD_ERR_ARG, "invalid scheme");
  if (p.eos != SRHD_EOS_TM && p.eos != SRHD_EOS_POLYTROPIC)
    return noalloc_fail(SRHD_ERR_ARG, "invalid eos");
  if (p.eos == SRHD_EOS_POLYTROPIC && !(p.gamma > 1.0 && p.gamma <= 5.0 / 3.0 + 1e-12))
    return noalloc_fail(SRHD_ERR_ARG, "gamma of the polytropic EoS must be in (1, 5/3]");
  const int ori = p.scheme == SRHD_SCHEME_TOTAL ? 1 : 0;
  double* patch_dt = nullptr;
  int32_t* patch_bad = nullptr;
  srhd_status st = scratch_for_current_device(&patch_dt, &patch_bad);
  if (st != SRHD_OK) return st;
  const int maxit = p.newton_max_iter > 0 ? p.newton_max_iter : (prec == SRHD_FP64 ? 50 : 30);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (npatch > 0) {
    if (prec == SRHD_FP64)
      launch_patch_cfl<srhd::PrecFP64>(cons, npatch, dh, p, maxit, patch_dt, patch_bad, ori, s);
    else if (prec == SRHD_MIXED)
      launch_patch_cfl<srhd::PrecMixed>(cons, npatch, dh, p, maxit, patch_dt, patch_bad, ori, s);
    else
      launch_patch_cfl<srhd::PrecMixedCF>(cons, npatch, dh, p, maxit, patch_dt, patch_bad, ori, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(SRHD_ERR_CUDA, cudaGetErrorString(e));
  }
  patch_cfl_reduce_kernel<<<1, kThreads, 0, s>>>(patch_dt, patch_bad, npatch, dt_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(SRHD_ERR_CUDA, cudaGetErrorString(e));
  return SRHD_OK;
}
