// C ABI of libsrhd (declared in include/srhd.h): context management,
// argument validation and launches. Device work is in srhd_kernels.cuh.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <cudaTypedefs.h>

#include "srhd.h"
#include "srhd_amr.cuh"
#include "srhd_kernels.cuh"

namespace srhd {
extern template struct Launch<PrecFP64>;
extern template struct Launch<PrecMixed>;
extern template struct Launch<PrecMixedCF>;

__global__ void cfl_finalize_kernel(const double* partial, const int32_t* bad, int n,
                                    double* dt_out) {
  __shared__ double s_m[32];
  __shared__ int s_b[32];
  double m = DBL_MAX;
  int b = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    m = fmin(m, partial[i]);
    b |= bad[i];
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
    for (int w = 0; w < int(blockDim.x >> 5); ++w) { mm = fmin(mm, s_m[w]); bb |= s_b[w]; }
    if (bb) mm = __longlong_as_double(0x7ff8000000000000ULL);
    else if (mm == DBL_MAX) mm = __longlong_as_double(0x7ff0000000000000ULL);  // +inf: no cells
    dt_out[0] = mm;
  }
}

// (dt, dh) of every patch of a uniform step.
__global__ void set_dt_dh_kernel(double* dt_dh, int64_t n, double dt, double dh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dt_dh[2 * i] = dt;
    dt_dh[2 * i + 1] = dh;
  }
}

// Minimum of n per-chunk CFL bounds: NaN if one is NaN (an unphysical cell).
__global__ void min_dt_kernel(const double* v, int n, double* out) {
  double m = __longlong_as_double(0x7ff0000000000000ULL);
  bool bad = false;
  for (int i = 0; i < n; ++i) {
    bad |= isnan(v[i]);
    m = fmin(m, v[i]);
  }
  out[0] = bad ? __longlong_as_double(0x7ff8000000000000ULL) : m;
}
}  // namespace srhd

// Device buffers, streams and events of srhd_advance_uniform_host: made on
// its first call, grown when a larger grid or a wider storage type arrives,
// freed by srhd_destroy.
struct UniformStage {
  static constexpr int kMaxChunks = 64;
  int64_t cap_cells = 0;  // bytes of in and of out
  int64_t cap_patches = 0;
  void* in = nullptr;       // interior state at t^n, [np][5][8^3]
  void* out = nullptr;      // interior state at t^n+1
  double* dt_dh = nullptr;  // [np][2]
  int32_t* status = nullptr;
  double* dn = nullptr;       // per-chunk CFL bounds, then their minimum
  double* host_dn = nullptr;  // pinned copy of the minimum
  double* part_dt = nullptr;  // CFL partial minima of the two compute streams, [2][slots]
  int32_t* part_bad = nullptr;
  // host-to-device, two compute streams (even and odd chunks), device-to-host
  cudaStream_t s[4] = {};
  cudaEvent_t copied[kMaxChunks] = {}, stepped[kMaxChunks] = {}, start = nullptr,
              fin = nullptr;
  bool have_streams = false;

  void free_buffers() {
    cudaFree(in);
    cudaFree(out);
    cudaFree(dt_dh);
    cudaFree(status);
    in = out = nullptr;
    dt_dh = nullptr;
    status = nullptr;
    cap_cells = cap_patches = 0;
  }
  ~UniformStage() {
    free_buffers();
    cudaFree(dn);
    cudaFree(part_dt);
    cudaFree(part_bad);
    if (host_dn) cudaFreeHost(host_dn);
    // handles a failed creation left null are skipped
    for (auto& x : s)
      if (x) cudaStreamDestroy(x);
    for (int k = 0; k < kMaxChunks; ++k) {
      if (copied[k]) cudaEventDestroy(copied[k]);
      if (stepped[k]) cudaEventDestroy(stepped[k]);
    }
    if (start) cudaEventDestroy(start);
    if (fin) cudaEventDestroy(fin);
  }
};

struct srhd_ctx {
  srhd_params params;
  int device;
  int num_sms;
  int patch_grid[3][srhd::kPatchVariants];  // persistent grid per precision and variant
  int poly_grid[3];                         // persistent grid of the polytropic kernels
  int vl_grid[3][2];                        // persistent grid of the VL kernels [prec][poly]
  int scratch_slots;      // capacity of the partial-minimum arrays
  double* partial_dt;     // scratch [scratch_slots]
  int32_t* partial_bad;   // scratch [scratch_slots]
  UniformStage* uniform;  // srhd_advance_uniform_host's state (NULL until its first call)
};

namespace {

thread_local char g_err[512] = "";

srhd_status fail(srhd_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

srhd_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SRHD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool valid_prec(srhd_prec p) { return p == SRHD_FP64 || p == SRHD_MIXED || p == SRHD_MIXED_CF; }

// Calls f with the launcher of the precision tag that prec selects.
template <class F> cudaError_t dispatch(srhd_prec prec, F&& f) {
  switch (prec) {
    case SRHD_FP64: return f(srhd::Launch<srhd::PrecFP64>{});
    case SRHD_MIXED: return f(srhd::Launch<srhd::PrecMixed>{});
    default: return f(srhd::Launch<srhd::PrecMixedCF>{});
  }
}

int newton_maxit(const srhd_ctx* c, srhd_prec prec) {
  if (c->params.newton_max_iter > 0) return c->params.newton_max_iter;
  return prec == SRHD_FP64 ? 50 : 30;
}

int grid_for(const srhd_ctx* c, int64_t n, int per_sm) {
  int64_t g = (n + 255) / 256;
  int64_t cap = (int64_t)c->num_sms * per_sm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : int(g);
}

// Blocks of the ghost fill: one per patch, at most eight per SM (grid-stride).
int ghost_grid(const srhd_ctx* c, int64_t npatch) {
  int64_t g = std::min<int64_t>(npatch, (int64_t)c->num_sms * 8);
  return g < 1 ? 1 : int(g);
}

srhd_status check_params(const srhd_params* p) {
  if (!(p->cfl > 0.0) || !(p->cfl <= 1.0)) return fail(SRHD_ERR_ARG, "cfl must be in (0, 1]");
  if (!(p->theta >= 0.0) || !(p->theta <= 2.0)) return fail(SRHD_ERR_ARG, "theta must be in [0, 2]");
  if (!(p->retry_factor > 0.0) || !(p->retry_factor < 1.0))
    return fail(SRHD_ERR_ARG, "retry_factor must be in (0, 1)");
  if (!(p->theta_floor > 0.0) || !(p->theta_floor < 1.0))
    return fail(SRHD_ERR_ARG, "theta_floor must be in (0, 1)");
  if (p->riemann != SRHD_HLLC && p->riemann != SRHD_HLLE)
    return fail(SRHD_ERR_ARG, "riemann must be SRHD_HLLC or SRHD_HLLE");
  if (p->cfl_mode != SRHD_CFL_SIGNAL && p->cfl_mode != SRHD_CFL_LIGHT)
    return fail(SRHD_ERR_ARG, "cfl_mode must be SRHD_CFL_SIGNAL or SRHD_CFL_LIGHT");
  if (p->ndim < 1 || p->ndim > 3) return fail(SRHD_ERR_ARG, "ndim must be 1, 2 or 3");
  if (p->newton_max_iter < 0 || p->newton_max_iter > 1000)
    return fail(SRHD_ERR_ARG, "newton_max_iter must be in [0, 1000]");
  if (p->scheme != SRHD_SCHEME_REDUCED && p->scheme != SRHD_SCHEME_TOTAL)
    return fail(SRHD_ERR_ARG, "scheme must be SRHD_SCHEME_REDUCED or SRHD_SCHEME_TOTAL");
  if (p->patch_variant < 0 || p->patch_variant >= srhd::kPatchVariants)
    return fail(SRHD_ERR_ARG, "patch_variant must be in [0, %d)", srhd::kPatchVariants);
  if (p->eos != SRHD_EOS_TM && p->eos != SRHD_EOS_POLYTROPIC)
    return fail(SRHD_ERR_ARG, "eos must be SRHD_EOS_TM or SRHD_EOS_POLYTROPIC");
  if (p->eos == SRHD_EOS_POLYTROPIC && !(p->gamma > 1.0 && p->gamma <= 5.0 / 3.0 + 1e-12))
    return fail(SRHD_ERR_ARG, "gamma of the polytropic EoS must be in (1, 5/3]");
  return SRHD_OK;
}

srhd::EosArg eos_arg(const srhd_params& p) {
  return srhd::EosArg{p.eos == SRHD_EOS_POLYTROPIC ? 1 : 0, p.gamma};
}

srhd_status check_ctx(const srhd_ctx* c) {
  if (!c) return fail(SRHD_ERR_ARG, "ctx is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return fail(SRHD_ERR_ARG, "ctx was created on device %d but device %d is current", c->device,
                dev);
  return SRHD_OK;
}

}  // namespace

namespace srhd {
// Sets the message returned by srhd_last_error() on the calling thread (used
// by entry points defined in other translation units).
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace srhd

extern "C" {

srhd_status srhd_default_params(srhd_params* p) {
  if (!p) return fail(SRHD_ERR_ARG, "params is NULL");
  p->cfl = 0.5;
  p->theta = 1.5;
  p->retry_factor = 0.75;
  p->theta_floor = 1e-2;
  p->riemann = SRHD_HLLC;
  p->cfl_mode = SRHD_CFL_SIGNAL;
  p->ndim = 3;
  p->newton_max_iter = 0;
  p->patch_variant = 0;
  p->scheme = SRHD_SCHEME_REDUCED;
  p->eos = SRHD_EOS_TM;
  p->gamma = 5.0 / 3.0;
  return SRHD_OK;
}

const char* srhd_last_error(void) { return g_err; }

srhd_status srhd_create(srhd_ctx** out, const srhd_params* p) {
  if (!out) return fail(SRHD_ERR_ARG, "ctx output pointer is NULL");
  *out = nullptr;
  srhd_params prm;
  if (p) prm = *p; else srhd_default_params(&prm);
  srhd_status st = check_params(&prm);
  if (st != SRHD_OK) return st;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if ((e = srhd::Launch<srhd::PrecFP64>::setup()) != cudaSuccess) return cuda_fail(e, "setup fp64");
  if ((e = srhd::Launch<srhd::PrecMixed>::setup()) != cudaSuccess) return cuda_fail(e, "setup mixed");
  if ((e = srhd::Launch<srhd::PrecMixedCF>::setup()) != cudaSuccess)
    return cuda_fail(e, "setup mixed_cf");
  srhd_ctx* c = new (std::nothrow) srhd_ctx;
  if (!c) return fail(SRHD_ERR_ARG, "out of host memory");
  c->params = prm;
  c->device = dev;
  c->num_sms = nsm;
  for (int v = 0; v < srhd::kPatchVariants; ++v) {
    int b64 = srhd::Launch<srhd::PrecFP64>::patch_blocks_per_sm(v);
    int b32 = srhd::Launch<srhd::PrecMixed>::patch_blocks_per_sm(v);
    int bcf = srhd::Launch<srhd::PrecMixedCF>::patch_blocks_per_sm(v);
    if (b64 < 1 || b32 < 1 || bcf < 1) {
      delete c;
      return fail(SRHD_ERR_CUDA, "patch kernel variant %d does not fit on an SM (%d, %d, %d)", v,
                  b64, b32, bcf);
    }
    c->patch_grid[SRHD_FP64][v] = nsm * b64;
    c->patch_grid[SRHD_MIXED][v] = nsm * b32;
    c->patch_grid[SRHD_MIXED_CF][v] = nsm * bcf;
  }
  {
    int b64 = srhd::Launch<srhd::PrecFP64>::poly_blocks_per_sm();
    int b32 = srhd::Launch<srhd::PrecMixed>::poly_blocks_per_sm();
    int bcf = srhd::Launch<srhd::PrecMixedCF>::poly_blocks_per_sm();
    if (b64 < 1 || b32 < 1 || bcf < 1) {
      delete c;
      return fail(SRHD_ERR_CUDA, "polytropic patch kernel does not fit on an SM");
    }
    c->poly_grid[SRHD_FP64] = nsm * b64;
    c->poly_grid[SRHD_MIXED] = nsm * b32;
    c->poly_grid[SRHD_MIXED_CF] = nsm * bcf;
    for (int poly = 0; poly < 2; ++poly) {
      int v64 = srhd::Launch<srhd::PrecFP64>::vl_blocks_per_sm(poly);
      int v32 = srhd::Launch<srhd::PrecMixed>::vl_blocks_per_sm(poly);
      int vcf = srhd::Launch<srhd::PrecMixedCF>::vl_blocks_per_sm(poly);
      if (v64 < 1 || v32 < 1 || vcf < 1) {
        delete c;
        return fail(SRHD_ERR_CUDA, "VL patch kernel does not fit on an SM");
      }
      c->vl_grid[SRHD_FP64][poly] = nsm * v64;
      c->vl_grid[SRHD_MIXED][poly] = nsm * v32;
      c->vl_grid[SRHD_MIXED_CF][poly] = nsm * vcf;
    }
  }
  c->scratch_slots = nsm * 8;
  c->uniform = nullptr;
  c->partial_dt = nullptr;
  c->partial_bad = nullptr;
  e = cudaMalloc(&c->partial_dt, sizeof(double) * c->scratch_slots);
  if (e == cudaSuccess) e = cudaMalloc(&c->partial_bad, sizeof(int32_t) * c->scratch_slots);
  if (e != cudaSuccess) {
    cudaFree(c->partial_dt);
    delete c;
    return cuda_fail(e, "cudaMalloc scratch");
  }
  *out = c;
  g_err[0] = 0;
  return SRHD_OK;
}

srhd_status srhd_destroy(srhd_ctx* c) {
  if (!c) return SRHD_OK;
  cudaFree(c->partial_dt);
  cudaFree(c->partial_bad);
  delete c->uniform;
  delete c;
  return SRHD_OK;
}

srhd_status srhd_prim2con(srhd_ctx* c, srhd_prec prec, const void* prim, void* cons, int64_t n,
                          int64_t var_stride, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (n < 0 || var_stride < n) return fail(SRHD_ERR_ARG, "need 0 <= n <= var_stride");
  if (n == 0) return SRHD_OK;
  if (!prim || !cons) return fail(SRHD_ERR_ARG, "prim/cons is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int grid = grid_for(c, n, 16);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::prim2con(prim, cons, n, var_stride, c->params.scheme,
                                 eos_arg(c->params), grid, s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "prim2con launch");
}

srhd_status srhd_con2pri(srhd_ctx* c, srhd_prec prec, const void* cons, void* prim, int64_t n,
                         int64_t var_stride, int32_t* cell_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (n < 0 || var_stride < n) return fail(SRHD_ERR_ARG, "need 0 <= n <= var_stride");
  if (n == 0) return SRHD_OK;
  if (!prim || !cons) return fail(SRHD_ERR_ARG, "prim/cons is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int grid = grid_for(c, n, 16);
  int maxit = newton_maxit(c, prec);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::con2pri(cons, prim, n, var_stride, cell_status, maxit, c->params.scheme,
                                eos_arg(c->params), grid, s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "con2pri launch");
}

static srhd_status launch_patches(srhd_ctx* c, srhd_prec prec, srhd::PatchArgs& a,
                                  double* dt_next, cudaStream_t s, bool vl = false,
                                  double* scratch_dt = nullptr, int32_t* scratch_bad = nullptr) {
  if (!scratch_dt) {
    scratch_dt = c->partial_dt;
    scratch_bad = c->partial_bad;
  }
  const int variant = c->params.patch_variant;
  const int poly = c->params.eos == SRHD_EOS_POLYTROPIC ? 1 : 0;
  int grid = vl ? c->vl_grid[prec][poly]
                : (poly ? c->poly_grid[prec] : c->patch_grid[prec][variant]);
  if (grid > a.npatch) grid = a.npatch;
  if (dt_next) {
    a.partial_dt = scratch_dt;
    a.partial_bad = scratch_bad;
  }
  cudaError_t e = cudaSuccess;
  if (a.npatch > 0) {
    e = dispatch(prec, [&](auto L) {
      return vl ? decltype(L)::patches_vl(a, poly, grid, s)
                : decltype(L)::patches(a, variant, poly, grid, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "patch kernel launch");
  } else {
    grid = 0;
  }
  if (dt_next) {
    srhd::cfl_finalize_kernel<<<1, 256, 0, s>>>(scratch_dt, scratch_bad, grid, dt_next);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cfl finalize launch");
  }
  return SRHD_OK;
}

static void fill_common(const srhd_ctx* c, srhd_prec prec, srhd::PatchArgs& a) {
  a.theta0 = c->params.theta;
  a.retry_factor = c->params.retry_factor;
  a.theta_floor = c->params.theta_floor;
  a.cfl = c->params.cfl;
  a.riemann = c->params.riemann;
  a.cfl_mode = c->params.cfl_mode;
  a.ndim = c->params.ndim;
  a.maxit = newton_maxit(c, prec);
  a.eos_gamma = c->params.gamma;
  a.ori = c->params.scheme == SRHD_SCHEME_TOTAL ? 1 : 0;
  a.partial_dt = nullptr;
  a.partial_bad = nullptr;
  a.gather = 0;
  a.gnx = a.gny = a.gnz = 1;
  a.gbcx = a.gbcy = a.gbcz = 0;
  a.gp0 = 0;
  a.amr_map = nullptr;
  a.amr_old = a.amr_new = a.amr_special = nullptr;
  a.amr_ncells = 0;
  a.amr_w = 0.0;
  a.amr_nspecial = 0;
  a.tma = 0;
}

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime
// (the library does not link libcuda); NULL if the driver lacks it.
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor maps of a uniform grid's array [np][nvar][8][8][8] (the interiors,
// nvar 5, or the primitive cache, nvar 6), viewed as a 5-D tensor (x, y, z,
// var, patch), with the boxes of the staged gather (PatchArgs::tmap:
// interior, x, y and z face slabs, variables 0..4). False when they cannot
// be made (no driver entry point, an address not 16-byte aligned, a refused
// encoding); the kernel then gathers every tile with plain loads.
static bool uniform_tmaps(srhd_prec prec, const void* interior, int64_t np, CUtensorMap (&m)[4],
                          int nvar = 5) {
  const auto fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(interior) & 15) != 0 || np < 1 || np > 0xffffffffLL)
    return false;
  const cuuint64_t es = prec == SRHD_FP64 ? 8 : 4;
  const CUtensorMapDataType dt =
      prec == SRHD_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t dims[5] = {8, 8, 8, cuuint64_t(nvar), cuuint64_t(np)};
  const cuuint64_t strides[4] = {8 * es, 64 * es, 512 * es, cuuint64_t(nvar) * 512 * es};
  const cuuint32_t boxes[4][5] = {{8, 8, 8, 5, 1}, {4, 8, 8, 5, 1}, {8, 2, 8, 5, 1},
                                  {8, 8, 2, 5, 1}};
  const cuuint32_t unit[5] = {1, 1, 1, 1, 1};
  for (int k = 0; k < 4; ++k)
    if (fn(&m[k], dt, 5, const_cast<void*>(interior), dims, strides, boxes[k], unit,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  return true;
}

srhd_status srhd_flux_patches(srhd_ctx* c, srhd_prec prec, const void* cons_ghosted,
                              void* face_flux, int32_t npatch, const double* dt_dh,
                              int32_t* patch_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npatch < 0) return fail(SRHD_ERR_ARG, "npatch < 0");
  if (npatch == 0) return SRHD_OK;
  if (!cons_ghosted || !face_flux || !dt_dh)
    return fail(SRHD_ERR_ARG, "cons_ghosted/face_flux/dt_dh is NULL");
  srhd::PatchArgs a;
  fill_common(c, prec, a);
  a.in = cons_ghosted;
  a.out = nullptr;
  a.pflux = nullptr;
  a.face_flux = face_flux;
  a.npatch = npatch;
  a.dt_dh = dt_dh;
  a.worklist = nullptr;
  a.status = patch_status;
  a.flux_only = 1;
  return launch_patches(c, prec, a, nullptr, static_cast<cudaStream_t>(stream));
}

srhd_status srhd_advance_patches(srhd_ctx* c, srhd_prec prec, const void* cons_ghosted,
                                 void* cons_out, void* patch_face_flux, int32_t npatch,
                                 const double* dt_dh, const int32_t* worklist, double* dt_next,
                                 int32_t* patch_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npatch < 0) return fail(SRHD_ERR_ARG, "npatch < 0");
  if (npatch > 0 && (!cons_ghosted || !cons_out || !dt_dh))
    return fail(SRHD_ERR_ARG, "cons_ghosted/cons_out/dt_dh is NULL");
  if (npatch == 0 && !dt_next) return SRHD_OK;
  srhd::PatchArgs a;
  fill_common(c, prec, a);
  a.in = cons_ghosted;
  a.out = cons_out;
  a.pflux = patch_face_flux;
  a.face_flux = nullptr;
  a.npatch = npatch;
  a.dt_dh = dt_dh;
  a.worklist = worklist;
  a.status = patch_status;
  a.flux_only = 0;
  return launch_patches(c, prec, a, dt_next, static_cast<cudaStream_t>(stream));
}

static srhd_status check_bc(const int32_t* bc) {
  if (!bc) return fail(SRHD_ERR_ARG, "bc is NULL");
  for (int d = 0; d < 3; ++d)
    if (bc[d] != SRHD_BC_PERIODIC && bc[d] != SRHD_BC_OUTFLOW)
      return fail(SRHD_ERR_ARG, "bc[%d] must be SRHD_BC_PERIODIC or SRHD_BC_OUTFLOW", d);
  return SRHD_OK;
}

// The fused step of srhd_advance_patches on patches p0 .. p0+n-1 of a uniform
// grid, reading each 12^3 tile from the grid (gather mode of patch_kernel).
// maps (nullable): tensor maps of `interior` from uniform_tmaps, for the
// staged gather.
static void gather_args(const srhd_ctx* c, srhd_prec prec, srhd::PatchArgs& a,
                        const void* interior, int32_t npx, int32_t npy, int32_t npz,
                        const int32_t* bc, int64_t p0, const CUtensorMap* maps = nullptr) {
  fill_common(c, prec, a);
  if (maps) {
    for (int k = 0; k < 4; ++k) a.tmap[k] = maps[k];
    a.tma = 1;
  }
  a.in = interior;
  a.gather = 1;
  a.gnx = npx;
  a.gny = npy;
  a.gnz = npz;
  a.gbcx = bc[0];
  a.gbcy = bc[1];
  a.gbcz = bc[2];
  a.gp0 = p0;
  a.face_flux = nullptr;
  a.worklist = nullptr;
  a.flux_only = 0;
  a.prim_in = nullptr;
  a.prim_out = nullptr;
}

srhd_status srhd_advance_uniform(srhd_ctx* c, srhd_prec prec, const void* interior, int32_t npx,
                                 int32_t npy, int32_t npz, const int32_t* bc, int32_t p0,
                                 int32_t n, void* cons_out, void* patch_face_flux,
                                 const double* dt_dh, double* dt_next, int32_t* patch_status,
                                 void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  const int64_t np = (int64_t)npx * npy * npz;
  if (np > INT32_MAX) return fail(SRHD_ERR_ARG, "more than 2^31-1 patches");
  if (p0 < 0 || n < 0 || p0 + (int64_t)n > np)
    return fail(SRHD_ERR_ARG, "patch range [%d, %d) outside the grid", p0, p0 + n);
  if ((st = check_bc(bc)) != SRHD_OK) return st;
  if (n > 0 && (!interior || !cons_out || !dt_dh))
    return fail(SRHD_ERR_ARG, "interior/cons_out/dt_dh is NULL");
  if (n == 0 && !dt_next) return SRHD_OK;
  srhd::PatchArgs a;
  CUtensorMap maps[4];
  const bool tma = n > 0 && uniform_tmaps(prec, interior, np, maps);
  gather_args(c, prec, a, interior, npx, npy, npz, bc, p0, tma ? maps : nullptr);
  a.out = cons_out;
  a.pflux = patch_face_flux;
  a.npatch = n;
  a.dt_dh = dt_dh;
  a.status = patch_status;
  return launch_patches(c, prec, a, dt_next, static_cast<cudaStream_t>(stream));
}

srhd_status srhd_con2pri_patches(srhd_ctx* c, srhd_prec prec, const void* cons, int64_t npatch,
                                 void* prim_out, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npatch < 0) return fail(SRHD_ERR_ARG, "npatch < 0");
  if (npatch == 0) return SRHD_OK;
  if (npatch > INT64_MAX / (6 * srhd::kNC)) return fail(SRHD_ERR_ARG, "npatch too large");
  if (!cons || !prim_out) return fail(SRHD_ERR_ARG, "cons/prim_out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(c, npatch * srhd::kNC, 16);
  const int maxit = newton_maxit(c, prec);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::prim_cache(cons, prim_out, npatch, maxit, c->params.scheme,
                                   eos_arg(c->params), grid, s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "con2pri_patches launch");
}

srhd_status srhd_advance_uniform_prim(srhd_ctx* c, srhd_prec prec, const void* interior,
                                      const void* prim_in, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, int32_t p0, int32_t n, void* cons_out,
                                      void* prim_out, void* patch_face_flux, const double* dt_dh,
                                      double* dt_next, int32_t* patch_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  const int64_t np = (int64_t)npx * npy * npz;
  if (np > INT32_MAX) return fail(SRHD_ERR_ARG, "more than 2^31-1 patches");
  if (p0 < 0 || n < 0 || p0 + (int64_t)n > np)
    return fail(SRHD_ERR_ARG, "patch range [%d, %d) outside the grid", p0, p0 + n);
  if ((st = check_bc(bc)) != SRHD_OK) return st;
  if (n > 0 && (!interior || !prim_in || !cons_out || !prim_out || !dt_dh))
    return fail(SRHD_ERR_ARG, "interior/prim_in/cons_out/prim_out/dt_dh is NULL");
  if (n > 0 && (prim_out == prim_in || prim_out == interior || cons_out == prim_in ||
                cons_out == interior))
    return fail(SRHD_ERR_ARG, "prim_out/cons_out must not alias the inputs");
  if (n == 0 && !dt_next) return SRHD_OK;
  srhd::PatchArgs a;
  CUtensorMap maps[4];
  const bool tma = n > 0 && uniform_tmaps(prec, prim_in, np, maps, 6);
  gather_args(c, prec, a, interior, npx, npy, npz, bc, p0, tma ? maps : nullptr);
  a.gather = 3;
  a.prim_in = prim_in;
  a.prim_out = prim_out;
  a.out = cons_out;
  a.pflux = patch_face_flux;
  a.npatch = n;
  a.dt_dh = dt_dh;
  a.status = patch_status;
  return launch_patches(c, prec, a, dt_next, static_cast<cudaStream_t>(stream));
}

srhd_status srhd_advance_patches_vl(srhd_ctx* c, srhd_prec prec, const void* cons_ghosted,
                                    void* cons_out, void* patch_face_flux, int32_t npatch,
                                    const double* dt_dh, const int32_t* worklist,
                                    double* dt_next, int32_t* patch_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npatch < 0) return fail(SRHD_ERR_ARG, "npatch < 0");
  if (npatch > 0 && (!cons_ghosted || !cons_out || !dt_dh))
    return fail(SRHD_ERR_ARG, "cons_ghosted/cons_out/dt_dh is NULL");
  if (npatch == 0 && !dt_next) return SRHD_OK;
  srhd::PatchArgs a;
  fill_common(c, prec, a);
  a.in = cons_ghosted;
  a.out = cons_out;
  a.pflux = patch_face_flux;
  a.face_flux = nullptr;
  a.npatch = npatch;
  a.dt_dh = dt_dh;
  a.worklist = worklist;
  a.status = patch_status;
  a.flux_only = 0;
  return launch_patches(c, prec, a, dt_next, static_cast<cudaStream_t>(stream), true);
}

namespace {
__global__ void reciprocal_f64_kernel(const double* x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = srhd::drcp(x[i]);
}
}  // namespace

srhd_status srhd_reciprocal_f64(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0) return fail(SRHD_ERR_ARG, "n < 0");
  if (n == 0) return SRHD_OK;
  if (!x || !y) return fail(SRHD_ERR_ARG, "x/y is NULL");
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  reciprocal_f64_kernel<<<int(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "reciprocal launch");
}

srhd_status srhd_cfl_dt(srhd_ctx* c, srhd_prec prec, const void* cons, int32_t npatch, double dh,
                        double* dt_out, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npatch < 0) return fail(SRHD_ERR_ARG, "npatch < 0");
  if (!dt_out) return fail(SRHD_ERR_ARG, "dt_out is NULL");
  if (npatch > 0 && !cons) return fail(SRHD_ERR_ARG, "cons is NULL");
  if (!(dh > 0.0) || !std::isfinite(dh)) return fail(SRHD_ERR_ARG, "dh must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t ncell = (int64_t)npatch * srhd::kNC;
  int grid = 0;
  cudaError_t e = cudaSuccess;
  if (ncell > 0) {
    grid = int(std::min<int64_t>((ncell + srhd::kCflThreads - 1) / srhd::kCflThreads,
                                 (int64_t)c->scratch_slots));
    int maxit = newton_maxit(c, prec);
    e = dispatch(prec, [&](auto L) {
      return decltype(L)::cfl(cons, ncell, dh, c->params.cfl, c->params.ndim, c->params.cfl_mode,
                              maxit, c->params.scheme, eos_arg(c->params), c->partial_dt,
                              c->partial_bad, grid, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "cfl launch");
  }
  srhd::cfl_finalize_kernel<<<1, 256, 0, s>>>(c->partial_dt, c->partial_bad, grid, dt_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "cfl finalize launch");
}

srhd_status srhd_fill_ghosts_uniform(srhd_ctx* c, srhd_prec prec, const void* interior,
                                     void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                     const int32_t* bc, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  if (!interior || !ghosted || !bc) return fail(SRHD_ERR_ARG, "interior/ghosted/bc is NULL");
  for (int d = 0; d < 3; ++d)
    if (bc[d] != SRHD_BC_PERIODIC && bc[d] != SRHD_BC_OUTFLOW)
      return fail(SRHD_ERR_ARG, "bc[%d] must be SRHD_BC_PERIODIC or SRHD_BC_OUTFLOW", d);
  const int64_t np = (int64_t)npx * npy * npz;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::fill_ghosts(interior, ghosted, npx, npy, npz, bc, 2, 0, np,
                                    ghost_grid(c, np), s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "fill_ghosts launch");
}

srhd_status srhd_fill_ghosts_uniform_range(srhd_ctx* c, srhd_prec prec, const void* interior,
                                           void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                           const int32_t* bc, int32_t p0, int32_t n, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  const int64_t np = (int64_t)npx * npy * npz;
  if (p0 < 0 || n < 0 || p0 + (int64_t)n > np)
    return fail(SRHD_ERR_ARG, "patch range [%d, %d) outside the grid", p0, p0 + n);
  if (n == 0) return SRHD_OK;
  if (!interior || !ghosted || !bc) return fail(SRHD_ERR_ARG, "interior/ghosted/bc is NULL");
  for (int d = 0; d < 3; ++d)
    if (bc[d] != SRHD_BC_PERIODIC && bc[d] != SRHD_BC_OUTFLOW)
      return fail(SRHD_ERR_ARG, "bc[%d] must be SRHD_BC_PERIODIC or SRHD_BC_OUTFLOW", d);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::fill_ghosts(interior, ghosted, npx, npy, npz, bc, 2, p0, n,
                                    ghost_grid(c, n), s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "fill_ghosts launch");
}

srhd_status srhd_fill_ghosts_uniform3(srhd_ctx* c, srhd_prec prec, const void* interior,
                                      void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  if (!interior || !ghosted || !bc) return fail(SRHD_ERR_ARG, "interior/ghosted/bc is NULL");
  for (int d = 0; d < 3; ++d)
    if (bc[d] != SRHD_BC_PERIODIC && bc[d] != SRHD_BC_OUTFLOW)
      return fail(SRHD_ERR_ARG, "bc[%d] must be SRHD_BC_PERIODIC or SRHD_BC_OUTFLOW", d);
  const int64_t np = (int64_t)npx * npy * npz;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::fill_ghosts(interior, ghosted, npx, npy, npz, bc, 3, 0, np,
                                    ghost_grid(c, np), s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "fill_ghosts3 launch");
}

// ---- AMR ---------------------------------------------------------------------
namespace {
bool is_double(srhd_prec prec) { return prec == SRHD_FP64; }
}  // namespace

srhd_status srhd_amr_fill_ghosts(srhd_ctx* c, srhd_prec prec, const void* cur, const void* prev,
                                 void* ghosted, const int32_t* map, int32_t ntotal, int32_t p0,
                                 int32_t n, double w, const void* special, int32_t nspecial,
                                 void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (ntotal < 1 || p0 < 0 || n < 0 || (int64_t)p0 + n > ntotal)
    return fail(SRHD_ERR_ARG, "patch range [%d, %d) outside [0, %d)", p0, p0 + n, ntotal);
  if (!(w >= 0.0 && w <= 1.0)) return fail(SRHD_ERR_ARG, "time weight w must be in [0, 1]");
  if (nspecial < 0 || (nspecial > 0 && !special))
    return fail(SRHD_ERR_ARG, "special states: nspecial < 0 or NULL array");
  if (n == 0) return SRHD_OK;
  if (!cur || !prev || !ghosted || !map) return fail(SRHD_ERR_ARG, "cur/prev/ghosted/map is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ncells = (int64_t)ntotal * srhd::kAmrInt;
  // four cells per thread when the map and ghosted rows are 16-byte aligned
  // (every row is: 1728 elements of 4 or 8 bytes), else one
  const bool wide = (reinterpret_cast<uintptr_t>(map) % 16 == 0) &&
                    (reinterpret_cast<uintptr_t>(ghosted) % 16 == 0);
  const int grid = grid_for(c, (int64_t)n * srhd::kAmrTile / (wide ? 4 : 1), 16);
  if (is_double(prec)) {
    auto k = wide ? srhd::amr_fill4_kernel<double> : srhd::amr_fill_kernel<double>;
    k<<<grid, 256, 0, s>>>(static_cast<const double*>(cur), static_cast<const double*>(prev),
                           static_cast<double*>(ghosted), map, p0, n, ncells, w,
                           static_cast<const double*>(special), nspecial);
  } else {
    auto k = wide ? srhd::amr_fill4_kernel<float> : srhd::amr_fill_kernel<float>;
    k<<<grid, 256, 0, s>>>(static_cast<const float*>(cur), static_cast<const float*>(prev),
                           static_cast<float*>(ghosted), map, p0, n, ncells, float(w),
                           static_cast<const float*>(special), nspecial);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "amr_fill launch");
}

srhd_status srhd_advance_amr(srhd_ctx* c, srhd_prec prec, const void* level_state,
                             const void* coarse_old, const void* coarse_new, const int32_t* map,
                             int32_t ntotal, double w, const void* special, int32_t nspecial,
                             void* cons_out, void* patch_face_flux, int32_t npatch,
                             const double* dt_dh, const int32_t* worklist, double* dt_next,
                             int32_t* patch_status, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (ntotal < 1 || npatch < 0 || npatch > ntotal)
    return fail(SRHD_ERR_ARG, "need ntotal >= 1 and 0 <= npatch <= ntotal");
  if (!(w >= 0.0 && w <= 1.0)) return fail(SRHD_ERR_ARG, "time weight w must be in [0, 1]");
  if (nspecial < 0 || (nspecial > 0 && !special))
    return fail(SRHD_ERR_ARG, "special states: nspecial < 0 or NULL array");
  if (npatch > 0 && (!level_state || !coarse_old || !coarse_new || !map || !cons_out || !dt_dh))
    return fail(SRHD_ERR_ARG, "level_state/coarse_old/coarse_new/map/cons_out/dt_dh is NULL");
  if (npatch == 0 && !dt_next) return SRHD_OK;
  srhd::PatchArgs a;
  fill_common(c, prec, a);
  a.in = level_state;
  a.gather = 2;
  a.amr_map = map;
  a.amr_old = coarse_old;
  a.amr_new = coarse_new;
  a.amr_special = special;
  a.amr_nspecial = nspecial;
  a.amr_ncells = (int64_t)ntotal * srhd::kAmrInt;
  a.amr_w = w;
  a.out = cons_out;
  a.pflux = patch_face_flux;
  a.face_flux = nullptr;
  a.npatch = npatch;
  a.dt_dh = dt_dh;
  a.worklist = worklist;
  a.status = patch_status;
  a.flux_only = 0;
  return launch_patches(c, prec, a, dt_next, static_cast<cudaStream_t>(stream));
}

srhd_status srhd_amr_restrict(srhd_ctx* c, srhd_prec prec, void* cur, const int32_t* children,
                              int32_t nparent, int32_t ntotal, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (nparent < 0 || ntotal < 1) return fail(SRHD_ERR_ARG, "nparent < 0 or ntotal < 1");
  if (nparent == 0) return SRHD_OK;
  if (!cur || !children) return fail(SRHD_ERR_ARG, "cur/children is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(c, (int64_t)nparent * srhd::kAmrInt, 16);
  if (is_double(prec))
    srhd::amr_restrict_kernel<double><<<grid, 256, 0, s>>>(static_cast<double*>(cur), children,
                                                          nparent, ntotal);
  else
    srhd::amr_restrict_kernel<float><<<grid, 256, 0, s>>>(static_cast<float*>(cur), children,
                                                         nparent, ntotal);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "amr_restrict launch");
}

srhd_status srhd_amr_flux_correct(srhd_ctx* c, srhd_prec prec, void* cur, const void* flux_coarse,
                                  const void* flux_fine0, const void* flux_fine1,
                                  const int32_t* faces, int32_t nrows, const double* dt_dh,
                                  int32_t ntotal, int32_t* skipped, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (nrows < 0 || ntotal < 1) return fail(SRHD_ERR_ARG, "nrows < 0 or ntotal < 1");
  if (nrows == 0) return SRHD_OK;
  if (!cur || !flux_coarse || !flux_fine0 || !flux_fine1 || !faces || !dt_dh)
    return fail(SRHD_ERR_ARG, "a pointer argument is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = nrows < c->num_sms * 8 ? nrows : c->num_sms * 8;
  const int ori = c->params.scheme == SRHD_SCHEME_TOTAL ? 1 : 0;
  if (is_double(prec))
    srhd::amr_flux_correct_kernel<double><<<grid, 256, 0, s>>>(
        static_cast<double*>(cur), static_cast<const double*>(flux_coarse),
        static_cast<const double*>(flux_fine0), static_cast<const double*>(flux_fine1), faces,
        nrows, dt_dh, ntotal, ori, skipped);
  else
    srhd::amr_flux_correct_kernel<float><<<grid, 256, 0, s>>>(
        static_cast<float*>(cur), static_cast<const float*>(flux_coarse),
        static_cast<const float*>(flux_fine0), static_cast<const float*>(flux_fine1), faces,
        nrows, dt_dh, ntotal, ori, skipped);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "amr_flux_correct launch");
}

srhd_status srhd_amr_prolong(srhd_ctx* c, srhd_prec prec, const void* cur, const void* prev,
                             const int32_t* table, int32_t nrows, int32_t ntotal, double w,
                             void* out, int32_t* fallbacks, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (nrows < 0 || ntotal < 1) return fail(SRHD_ERR_ARG, "nrows < 0 or ntotal < 1");
  if (!(w >= 0.0 && w <= 1.0)) return fail(SRHD_ERR_ARG, "time weight w must be in [0, 1]");
  if (nrows == 0) return SRHD_OK;
  if (!cur || !prev || !table || !out) return fail(SRHD_ERR_ARG, "cur/prev/table/out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(c, nrows, 8);
  const int maxit = newton_maxit(c, prec);
  cudaError_t e = dispatch(prec, [&](auto L) {
    return decltype(L)::prolong(cur, prev, table, nrows, w, out,
                                (int64_t)ntotal * srhd::kAmrInt, maxit, c->params.scheme,
                                eos_arg(c->params), fallbacks, grid, s);
  });
  return e == cudaSuccess ? SRHD_OK : cuda_fail(e, "amr_prolong launch");
}

}  // extern "C"

// ---- uniform grid resident in host memory ----------------------------------
namespace {

// Makes the stage's streams and events and sizes its buffers for np patches,
// esz bytes per value.
srhd_status uniform_stage(srhd_ctx* c, int64_t np, int64_t esz) {
  if (!c->uniform) {
    c->uniform = new (std::nothrow) UniformStage;
    if (!c->uniform) return fail(SRHD_ERR_ARG, "out of host memory");
  }
  UniformStage& u = *c->uniform;
  cudaError_t e = cudaSuccess;
  if (!u.have_streams) {
    for (auto& x : u.s)
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    for (int k = 0; k < UniformStage::kMaxChunks && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&u.copied[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&u.stepped[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&u.start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&u.fin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&u.dn, sizeof(double) * (UniformStage::kMaxChunks + 1));
    if (e == cudaSuccess) e = cudaMalloc(&u.part_dt, sizeof(double) * 2 * c->scratch_slots);
    if (e == cudaSuccess) e = cudaMalloc(&u.part_bad, sizeof(int32_t) * 2 * c->scratch_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&u.host_dn, sizeof(double));
    if (e != cudaSuccess) {
      // a partly made stage is destroyed whole and made again on the next call
      delete c->uniform;
      c->uniform = nullptr;
      return cuda_fail(e, "uniform stage streams/events");
    }
    u.have_streams = true;
  }
  const int64_t cells = np * 5 * srhd::kNC * esz;
  if (cells > u.cap_cells || np > u.cap_patches) {
    u.free_buffers();
    e = cudaMalloc(&u.in, cells);
    if (e == cudaSuccess) e = cudaMalloc(&u.out, cells);
    if (e == cudaSuccess) e = cudaMalloc(&u.dt_dh, sizeof(double) * 2 * np);
    if (e == cudaSuccess) e = cudaMalloc(&u.status, sizeof(int32_t) * np);
    if (e != cudaSuccess) {
      u.free_buffers();
      return cuda_fail(e, "cudaMalloc uniform stage");
    }
    u.cap_cells = cells;
    u.cap_patches = np;
  }
  return SRHD_OK;
}

}  // namespace

srhd_status srhd_advance_uniform_host(srhd_ctx* c, srhd_prec prec, const void* host_in,
                                      void* host_out, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, double dt, double dh, double* dt_next,
                                      int32_t* patch_status, int32_t chunks, void* stream) {
  srhd_status st = check_ctx(c);
  if (st != SRHD_OK) return st;
  if (!valid_prec(prec)) return fail(SRHD_ERR_ARG, "invalid precision %d", int(prec));
  if (npx < 1 || npy < 1 || npz < 1) return fail(SRHD_ERR_ARG, "patch counts must be >= 1");
  const int64_t np = (int64_t)npx * npy * npz;
  if (np > INT32_MAX) return fail(SRHD_ERR_ARG, "more than 2^31-1 patches");
  if (!host_in || !host_out) return fail(SRHD_ERR_ARG, "host_in/host_out is NULL");
  if ((st = check_bc(bc)) != SRHD_OK) return st;
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(SRHD_ERR_ARG, "dt must be finite and >= 0");
  if (!(dh > 0.0) || !std::isfinite(dh)) return fail(SRHD_ERR_ARG, "dh must be positive");
  if (chunks < 1 || chunks > UniformStage::kMaxChunks)
    return fail(SRHD_ERR_ARG, "chunks must be in [1, %d]", UniformStage::kMaxChunks);
  // chunk k holds the z slabs z0[k] .. z0[k+1]-1 (a slab is npx*npy patches)
  const int K = chunks < npz ? chunks : npz;
  const int64_t slab = (int64_t)npx * npy;
  int z0[UniformStage::kMaxChunks + 1];
  for (int k = 0; k <= K; ++k) z0[k] = int((int64_t)npz * k / K);
  const int64_t esz = prec == SRHD_FP64 ? 8 : 4;
  const int64_t pbytes = 5 * srhd::kNC * esz;
  st = uniform_stage(c, np, esz);
  if (st != SRHD_OK) return st;
  UniformStage& u = *c->uniform;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaStream_t h2d = u.s[0], d2h = u.s[3];
  const char* what = "uniform step";
  srhd::set_dt_dh_kernel<<<grid_for(c, np, 4), 256, 0, user>>>(u.dt_dh, np, dt, dh);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(u.start, user);
  for (cudaStream_t x : u.s)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(x, u.start, 0);
  // Copies in: with periodic z the first chunk also needs the last one, so
  // that is copied second.
  int order[UniformStage::kMaxChunks];
  const bool zper = bc[2] == SRHD_BC_PERIODIC;
  for (int k = 0, n = 0; k < K; ++k) {
    if (zper && K > 1 && k == 1) order[n++] = K - 1;
    if (!(zper && K > 1 && k == K - 1)) order[n++] = k;
  }
  // The copies are enqueued in that order, each only when a chunk about to
  // be enqueued needs it (one chunk ahead), so that the first step is queued
  // without waiting for the host to queue every copy.
  int ncopied = 0;
  bool issued[UniformStage::kMaxChunks] = {};
  auto issue_through = [&](int k) {
    while (!issued[k] && e == cudaSuccess) {
      const int j = order[ncopied++];
      const int64_t a = z0[j] * slab, n = (z0[j + 1] - z0[j]) * slab;
      e = cudaMemcpyAsync(static_cast<char*>(u.in) + a * pbytes,
                          static_cast<const char*>(host_in) + a * pbytes, n * pbytes,
                          cudaMemcpyHostToDevice, h2d);
      if (e == cudaSuccess) e = cudaEventRecord(u.copied[j], h2d);
      issued[j] = true;
    }
  };
  auto chunk_of = [&](int z) {
    int k = 0;
    while (z >= z0[k + 1]) ++k;
    return k;
  };
  // the chunks whose copies the step of chunk k reads (the ghost zones,
  // two cells deep, reach one slab below and one above)
  auto for_needed = [&](int k, auto&& f) {
    for (int z = z0[k] - 1; z <= z0[k + 1]; ++z) {
      int zz = z;
      if (zz < 0 || zz >= npz) {
        if (!zper) continue;
        zz = (zz + npz) % npz;
      }
      f(chunk_of(zz));
    }
  };
  // Chunk k steps on compute stream k % 2 with CFL scratch k % 2 (its tiles
  // gathered from the grid copy), so that a launch's last partly filled wave
  // overlaps the next chunk's launch.
  CUtensorMap maps[4];
  const bool tma = uniform_tmaps(prec, u.in, np, maps);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const int par = k & 1;
    cudaStream_t comp = u.s[1 + par];
    for_needed(k, issue_through);
    if (k + 1 < K) for_needed(k + 1, issue_through);
    for_needed(k, [&](int j) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, u.copied[j], 0);
    });
    if (e != cudaSuccess) break;
    const int64_t a = z0[k] * slab, n = (z0[k + 1] - z0[k]) * slab;
    srhd::PatchArgs pa;
    gather_args(c, prec, pa, u.in, npx, npy, npz, bc, a, tma ? maps : nullptr);
    pa.out = static_cast<char*>(u.out) + a * pbytes;
    pa.pflux = nullptr;
    pa.npatch = int32_t(n);
    pa.dt_dh = u.dt_dh + 2 * a;
    pa.status = u.status + a;
    st = launch_patches(c, prec, pa, dt_next ? u.dn + k : nullptr, comp, false,
                        u.part_dt + par * c->scratch_slots, u.part_bad + par * c->scratch_slots);
    if (st != SRHD_OK) break;
    e = cudaEventRecord(u.stepped[k], comp);
    if (e != cudaSuccess) break;
    e = cudaStreamWaitEvent(d2h, u.stepped[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(host_out) + a * pbytes,
                          static_cast<const char*>(u.out) + a * pbytes, n * pbytes,
                          cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess && patch_status)
      e = cudaMemcpyAsync(patch_status + a, u.status + a, n * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, d2h);
  }
  if (st != SRHD_OK || e != cudaSuccess) {
    // nothing may still be copying into the caller's buffers after the return
    for (cudaStream_t x : u.s) cudaStreamSynchronize(x);
    return st != SRHD_OK ? st : cuda_fail(e, what);
  }
  if (dt_next) {
    // the device-to-host stream has waited for every chunk's step
    srhd::min_dt_kernel<<<1, 1, 0, d2h>>>(u.dn, K, u.dn + UniformStage::kMaxChunks);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(u.host_dn, u.dn + UniformStage::kMaxChunks, sizeof(double),
                          cudaMemcpyDeviceToHost, d2h);
  }
  // Every stream's work precedes fin: the device-to-host stream waited for
  // each chunk's step, and each step for its copies in.
  if (e == cudaSuccess) e = cudaEventRecord(u.fin, d2h);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, u.fin, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(u.fin);
  if (e != cudaSuccess) {
    for (cudaStream_t x : u.s) cudaStreamSynchronize(x);
    return cuda_fail(e, what);
  }
  if (dt_next) *dt_next = *u.host_dn;
  return SRHD_OK;
}
