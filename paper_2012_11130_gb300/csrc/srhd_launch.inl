// Launchers of the kernels in srhd_kernels.cuh for one precision tag P
// (srhd_physics.cuh). Included by exactly one translation unit per tag
// (srhd_fp64.cu, srhd_mixed.cu, srhd_mixed_cf.cu), which instantiates
// srhd::Launch<P>.
#pragma once

#include "srhd_kernels.cuh"

namespace srhd {

template <class S> struct PatchCfg;
// FP64: 207 KB of shared memory per CTA -> one CTA of 512 threads per SM;
// the FP64 pipe is the bound, so conversions run one state per thread.
template <> struct PatchCfg<double> {
  static constexpr int threads = 512, minb = 1;
  static constexpr bool pair = false;
};
// Float storage: 101 KB per CTA -> two CTAs of 256 threads per SM; latency
// bound, so conversions run two states per thread in lockstep.
template <> struct PatchCfg<float> {
  static constexpr int threads = 256, minb = 2;
  static constexpr bool pair = true;
};

template <class P> cudaError_t Launch<P>::setup() {
  using S = typename P::S;
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  constexpr bool PR = PatchCfg<S>::pair;
  return cudaFuncSetAttribute(patch_kernel<P, NT, MB, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(SmemLayout<S>::bytes));
}

template <class P> int Launch<P>::patch_blocks_per_sm() {
  using S = typename P::S;
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  constexpr bool PR = PatchCfg<S>::pair;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_kernel<P, NT, MB, PR>, NT,
                                                    SmemLayout<S>::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class P> cudaError_t Launch<P>::patches(const PatchArgs& a, int grid, cudaStream_t s) {
  using S = typename P::S;
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  constexpr bool PR = PatchCfg<S>::pair;
  patch_kernel<P, NT, MB, PR><<<grid, NT, SmemLayout<S>::bytes, s>>>(a);
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::prim2con(const void* prim, void* cons, int64_t n, int64_t stride, int grid,
                                cudaStream_t s) {
  using S = typename P::S;
  prim2con_kernel<S><<<grid, 256, 0, s>>>(static_cast<const S*>(prim), static_cast<S*>(cons), n,
                                          stride);
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::con2pri(const void* cons, void* prim, int64_t n, int64_t stride,
                               int32_t* status, int maxit, int grid, cudaStream_t s) {
  using S = typename P::S;
  con2pri_kernel<P><<<grid, 256, 0, s>>>(static_cast<const S*>(cons), static_cast<S*>(prim), n,
                                         stride, status, maxit);
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::cfl(const void* cons, int64_t ncell, double dh, double cfl, int ndim,
                           int mode, int maxit, double* partial, int32_t* bad, int grid,
                           cudaStream_t s) {
  using S = typename P::S;
  cfl_kernel<P, kCflThreads><<<grid, kCflThreads, 0, s>>>(static_cast<const S*>(cons), ncell, dh,
                                                          cfl, ndim, mode, maxit, partial, bad);
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::fill_ghosts(const void* interior, void* ghosted, int npx, int npy, int npz,
                                   const int32_t* bc, int grid, cudaStream_t s) {
  using S = typename P::S;
  fill_ghosts_kernel<S><<<grid, 256, 0, s>>>(static_cast<const S*>(interior),
                                             static_cast<S*>(ghosted), npx, npy, npz, bc[0], bc[1],
                                             bc[2]);
  return cudaGetLastError();
}

}  // namespace srhd
