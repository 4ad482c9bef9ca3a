// Launchers of the kernels in srhd_kernels.cuh for one storage type S.
// Included by exactly one translation unit per precision (srhd_fp64.cu,
// srhd_mixed.cu), which instantiates srhd::Launch<S>.
#pragma once

#include "srhd_kernels.cuh"

namespace srhd {

template <class S> struct PatchCfg;
// FP64: 207 KB of shared memory per CTA -> one CTA of 512 threads per SM.
template <> struct PatchCfg<double> { static constexpr int threads = 512, minb = 1; };
// Mixed: 101 KB per CTA -> two CTAs of 256 threads per SM.
template <> struct PatchCfg<float> { static constexpr int threads = 256, minb = 2; };

template <class S> cudaError_t Launch<S>::setup() {
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  return cudaFuncSetAttribute(patch_kernel<S, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(SmemLayout<S>::bytes));
}

template <class S> int Launch<S>::patch_blocks_per_sm() {
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, patch_kernel<S, NT, MB>, NT,
                                                    SmemLayout<S>::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class S> cudaError_t Launch<S>::patches(const PatchArgs& a, int grid, cudaStream_t s) {
  constexpr int NT = PatchCfg<S>::threads, MB = PatchCfg<S>::minb;
  patch_kernel<S, NT, MB><<<grid, NT, SmemLayout<S>::bytes, s>>>(a);
  return cudaGetLastError();
}

template <class S>
cudaError_t Launch<S>::prim2con(const void* prim, void* cons, int64_t n, int64_t stride, int grid,
                                cudaStream_t s) {
  prim2con_kernel<S><<<grid, 256, 0, s>>>(static_cast<const S*>(prim), static_cast<S*>(cons), n,
                                          stride);
  return cudaGetLastError();
}

template <class S>
cudaError_t Launch<S>::con2pri(const void* cons, void* prim, int64_t n, int64_t stride,
                               int32_t* status, int maxit, int grid, cudaStream_t s) {
  con2pri_kernel<S><<<grid, 256, 0, s>>>(static_cast<const S*>(cons), static_cast<S*>(prim), n,
                                         stride, status, maxit);
  return cudaGetLastError();
}

template <class S>
cudaError_t Launch<S>::cfl(const void* cons, int64_t ncell, double dh, double cfl, int ndim,
                           int mode, int maxit, double* partial, int32_t* bad, int grid,
                           cudaStream_t s) {
  cfl_kernel<S, kCflThreads><<<grid, kCflThreads, 0, s>>>(static_cast<const S*>(cons), ncell, dh,
                                                          cfl, ndim, mode, maxit, partial, bad);
  return cudaGetLastError();
}

template <class S>
cudaError_t Launch<S>::fill_ghosts(const void* interior, void* ghosted, int npx, int npy, int npz,
                                   const int32_t* bc, int grid, cudaStream_t s) {
  fill_ghosts_kernel<S><<<grid, 256, 0, s>>>(static_cast<const S*>(interior),
                                             static_cast<S*>(ghosted), npx, npy, npz, bc[0], bc[1],
                                             bc[2]);
  return cudaGetLastError();
}

}  // namespace srhd
