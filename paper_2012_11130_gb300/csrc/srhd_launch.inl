// Launchers of the kernels in srhd_kernels.cuh for one precision tag P
// (srhd_physics.cuh). Included by exactly one translation unit per tag
// (srhd_fp64.cu, srhd_mixed.cu, srhd_mixed_cf.cu), which instantiates
// srhd::Launch<P>.
#pragma once

#include "srhd_kernels.cuh"
#include "srhd_prolong.cuh"
#include "srhd_vl.cuh"

namespace srhd {

// Launch variants of the patch kernel (threads per CTA, CTAs per SM,
// two Newton solves per thread in lockstep or one). Variant 0 is the
// default; the rest are the search space of the autotuner
// (paper_2012_11130_gb300/autotune.py). Shared memory per CTA is 216 KB for
// double storage (one CTA per SM) and 108 KB for float storage (at most
// two).
template <class S, int V> struct PatchVariant;
template <> struct PatchVariant<double, 0> { static constexpr int nt = 512, minb = 1; static constexpr bool pair = false; };
template <> struct PatchVariant<double, 1> { static constexpr int nt = 256, minb = 1; static constexpr bool pair = false; };
template <> struct PatchVariant<double, 2> { static constexpr int nt = 512, minb = 1; static constexpr bool pair = true; };
template <> struct PatchVariant<double, 3> { static constexpr int nt = 384, minb = 1; static constexpr bool pair = false; };
template <> struct PatchVariant<float, 0> { static constexpr int nt = 384, minb = 2; static constexpr bool pair = true; };
template <> struct PatchVariant<float, 1> { static constexpr int nt = 448, minb = 2; static constexpr bool pair = true; };
template <> struct PatchVariant<float, 2> { static constexpr int nt = 320, minb = 2; static constexpr bool pair = true; };
template <> struct PatchVariant<float, 3> { static constexpr int nt = 256, minb = 2; static constexpr bool pair = true; };

// The polytropic-EoS kernel runs one configuration per storage type.
template <class S> struct PolyVariant;
template <> struct PolyVariant<double> { static constexpr int nt = 512, minb = 1; static constexpr bool pair = false; };
template <> struct PolyVariant<float> { static constexpr int nt = 448, minb = 2; static constexpr bool pair = true; };

template <class P, int G = 0> struct PolyKernel {
  using Cfg = PolyVariant<typename P::S>;
  static constexpr auto fn = patch_kernel<P, Cfg::nt, Cfg::minb, Cfg::pair, EosPoly, G>;
};

// The VL kernel: one configuration per storage type (its shared memory,
// 227 KB double / 114 KB float, allows one / two CTAs per SM).
template <class S> struct VlVariant;
template <> struct VlVariant<double> { static constexpr int nt = 512, minb = 1; };
template <> struct VlVariant<float> { static constexpr int nt = 384, minb = 2; };

template <class P, class E> struct VlKernel {
  using Cfg = VlVariant<typename P::S>;
  static constexpr auto fn = vl_patch_kernel<P, Cfg::nt, Cfg::minb, E>;
};

// G: 0 ghosted batch, 1 uniform-grid gather (srhd_advance_uniform), 2 AMR
// gather (srhd_advance_amr), 3 uniform-grid gather with primitive cache
// (srhd_advance_uniform_prim)
template <class P, int V, int G = 0> struct PatchKernel {
  using S = typename P::S;
  using Cfg = PatchVariant<S, V>;
  static constexpr auto fn = patch_kernel<P, Cfg::nt, Cfg::minb, Cfg::pair, EosTM, G>;
};

template <class P, int V> static cudaError_t setup_variant() {
  cudaError_t e = cudaFuncSetAttribute(PatchKernel<P, V>::fn,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PatchKernel<P, V, 1>::fn,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PatchKernel<P, V, 2>::fn,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PatchKernel<P, V, 3>::fn,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  return e;
}

template <class P> cudaError_t Launch<P>::setup() {
  cudaError_t e = setup_variant<P, 0>();
  if (e == cudaSuccess) e = setup_variant<P, 1>();
  if (e == cudaSuccess) e = setup_variant<P, 2>();
  if (e == cudaSuccess) e = setup_variant<P, 3>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PolyKernel<P>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PolyKernel<P, 1>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PolyKernel<P, 2>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(PolyKernel<P, 3>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SmemLayout<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(VlKernel<P, EosTM>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(VlSmem<typename P::S>::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(VlKernel<P, EosPoly>::fn,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(VlSmem<typename P::S>::bytes));
  return e;
}

template <class P> int Launch<P>::vl_blocks_per_sm(int poly) {
  int nb = 0;
  cudaError_t e = poly ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &nb, VlKernel<P, EosPoly>::fn, VlKernel<P, EosPoly>::Cfg::nt,
                             VlSmem<typename P::S>::bytes)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &nb, VlKernel<P, EosTM>::fn, VlKernel<P, EosTM>::Cfg::nt,
                             VlSmem<typename P::S>::bytes);
  return e == cudaSuccess ? nb : 0;
}

template <class P>
cudaError_t Launch<P>::patches_vl(const PatchArgs& a, int poly, int grid, cudaStream_t s) {
  constexpr size_t smem = VlSmem<typename P::S>::bytes;
  if (poly)
    VlKernel<P, EosPoly>::fn<<<grid, VlKernel<P, EosPoly>::Cfg::nt, smem, s>>>(a);
  else
    VlKernel<P, EosTM>::fn<<<grid, VlKernel<P, EosTM>::Cfg::nt, smem, s>>>(a);
  return cudaGetLastError();
}

template <class P> int Launch<P>::poly_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, PolyKernel<P>::fn,
                                                    PolyKernel<P>::Cfg::nt,
                                                    SmemLayout<typename P::S>::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class P, int V> static int blocks_variant() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, PatchKernel<P, V>::fn,
                                                    PatchKernel<P, V>::Cfg::nt,
                                                    SmemLayout<typename P::S>::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class P> int Launch<P>::patch_blocks_per_sm(int variant) {
  switch (variant) {
    case 0: return blocks_variant<P, 0>();
    case 1: return blocks_variant<P, 1>();
    case 2: return blocks_variant<P, 2>();
    default: return blocks_variant<P, 3>();
  }
}

template <class P, int V, int G>
static cudaError_t launch_variant(const PatchArgs& a, int grid, cudaStream_t s) {
  using K = PatchKernel<P, V, G>;
  K::fn<<<grid, K::Cfg::nt, SmemLayout<typename P::S>::bytes, s>>>(a);
  return cudaGetLastError();
}

template <class P, int G>
static cudaError_t launch_patches(const PatchArgs& a, int variant, int poly, int grid,
                                  cudaStream_t s) {
  if (poly) {
    using K = PolyKernel<P, G>;
    K::fn<<<grid, K::Cfg::nt, SmemLayout<typename P::S>::bytes, s>>>(a);
    return cudaGetLastError();
  }
  switch (variant) {
    case 0: return launch_variant<P, 0, G>(a, grid, s);
    case 1: return launch_variant<P, 1, G>(a, grid, s);
    case 2: return launch_variant<P, 2, G>(a, grid, s);
    default: return launch_variant<P, 3, G>(a, grid, s);
  }
}

template <class P>
cudaError_t Launch<P>::patches(const PatchArgs& a, int variant, int poly, int grid,
                               cudaStream_t s) {
  if (a.gather == 3) return launch_patches<P, 3>(a, variant, poly, grid, s);
  if (a.gather == 2) return launch_patches<P, 2>(a, variant, poly, grid, s);
  if (a.gather == 1) return launch_patches<P, 1>(a, variant, poly, grid, s);
  return launch_patches<P, 0>(a, variant, poly, grid, s);
}

template <class P>
cudaError_t Launch<P>::prim2con(const void* prim, void* cons, int64_t n, int64_t stride, int ori,
                                EosArg eos, int grid, cudaStream_t s) {
  using S = typename P::S;
  if (eos.poly)
    prim2con_kernel<S, EosPoly><<<grid, 256, 0, s>>>(
        static_cast<const S*>(prim), static_cast<S*>(cons), n, stride, ori, EosPoly{eos.gam});
  else
    prim2con_kernel<S, EosTM><<<grid, 256, 0, s>>>(static_cast<const S*>(prim),
                                                   static_cast<S*>(cons), n, stride, ori, EosTM{});
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::con2pri(const void* cons, void* prim, int64_t n, int64_t stride,
                               int32_t* status, int maxit, int ori, EosArg eos, int grid,
                               cudaStream_t s) {
  using S = typename P::S;
  if (eos.poly)
    con2pri_kernel<P, EosPoly><<<grid, 256, 0, s>>>(static_cast<const S*>(cons),
                                                    static_cast<S*>(prim), n, stride, status,
                                                    maxit, ori, EosPoly{eos.gam});
  else
    con2pri_kernel<P, EosTM><<<grid, 256, 0, s>>>(static_cast<const S*>(cons),
                                                  static_cast<S*>(prim), n, stride, status, maxit,
                                                  ori, EosTM{});
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::prim_cache(const void* cons, void* prim, int64_t npatch, int maxit, int ori,
                                  EosArg eos, int grid, cudaStream_t s) {
  using S = typename P::S;
  const int64_t n = npatch * kNC;
  if (eos.poly)
    prim_cache_kernel<P, EosPoly><<<grid, 256, 0, s>>>(static_cast<const S*>(cons),
                                                       static_cast<S*>(prim), n, maxit, ori,
                                                       EosPoly{eos.gam});
  else
    prim_cache_kernel<P, EosTM><<<grid, 256, 0, s>>>(static_cast<const S*>(cons),
                                                     static_cast<S*>(prim), n, maxit, ori,
                                                     EosTM{});
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::cfl(const void* cons, int64_t ncell, double dh, double cfl, int ndim,
                           int mode, int maxit, int ori, EosArg eos, double* partial, int32_t* bad,
                           int grid, cudaStream_t s) {
  using S = typename P::S;
  if (eos.poly)
    cfl_kernel<P, kCflThreads, EosPoly><<<grid, kCflThreads, 0, s>>>(
        static_cast<const S*>(cons), ncell, dh, cfl, ndim, mode, maxit, partial, bad, ori,
        EosPoly{eos.gam});
  else
    cfl_kernel<P, kCflThreads, EosTM><<<grid, kCflThreads, 0, s>>>(
        static_cast<const S*>(cons), ncell, dh, cfl, ndim, mode, maxit, partial, bad, ori,
        EosTM{});
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::fill_ghosts(const void* interior, void* ghosted, int npx, int npy, int npz,
                                   const int32_t* bc, int gh, int64_t p0, int64_t n, int grid,
                                   cudaStream_t s) {
  using S = typename P::S;
  const auto addr = reinterpret_cast<uintptr_t>(ghosted);
  if (gh == 3) {
    const int wide = addr % ghost_store_align<S, 3>() == 0;
    fill_ghosts_kernel<S, 3><<<grid, 256, 0, s>>>(static_cast<const S*>(interior),
                                                  static_cast<S*>(ghosted), npx, npy, npz, bc[0],
                                                  bc[1], bc[2], p0, n, wide);
  } else {
    const int wide = addr % ghost_store_align<S, 2>() == 0;
    fill_ghosts_kernel<S, 2><<<grid, 256, 0, s>>>(static_cast<const S*>(interior),
                                                  static_cast<S*>(ghosted), npx, npy, npz, bc[0],
                                                  bc[1], bc[2], p0, n, wide);
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t Launch<P>::prolong(const void* cur, const void* prev, const int32_t* table,
                               int64_t nrows, double w, void* out, int64_t ncells, int maxit,
                               int ori, EosArg eos, int32_t* fallbacks, int grid, cudaStream_t s) {
  using S = typename P::S;
  if (eos.poly)
    amr_prolong_kernel<P, EosPoly><<<grid, 128, 0, s>>>(
        static_cast<const S*>(cur), static_cast<const S*>(prev), table, nrows, S(w),
        static_cast<S*>(out), ncells, maxit, ori, EosPoly{eos.gam}, fallbacks);
  else
    amr_prolong_kernel<P, EosTM><<<grid, 128, 0, s>>>(
        static_cast<const S*>(cur), static_cast<const S*>(prev), table, nrows, S(w),
        static_cast<S*>(out), ncells, maxit, ori, EosTM{}, fallbacks);
  return cudaGetLastError();
}

}  // namespace srhd
