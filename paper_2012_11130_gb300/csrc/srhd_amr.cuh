// AMR kernels of libsrhd (sm_103a): the steps on either side of the
// per-patch update in a hierarchy of 8^3 patches (Section 3.1 of
// arXiv 2012.11130 and its flux-correction and ghost-zone passage):
//   amr_fill_kernel            ghost zones from a precomputed source map:
//                              same-level copies, piecewise-constant
//                              prolongation from the coarser level (linear in
//                              time between its old and new states),
//                              boundary states;
//   amr_restrict_kernel        fine -> coarse averaging (2x2x2 children);
//   amr_flux_correct_kernel    coarse-fine flux correction with the patch-face
//                              fluxes of the coarse step and of the two fine
//                              substeps, skipped on cells it would leave
//                              unphysical.
// All three move data: they are bound by HBM bandwidth. Every index that
// comes from a map is range checked on the device; an invalid entry gives
// NaN (fill) or is skipped (restriction, correction), never an access out of
// bounds.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace srhd {

constexpr int kAmrTile = 12 * 12 * 12;   // ghosted tile cells
constexpr int kAmrInt = 8 * 8 * 8;       // interior cells
constexpr int32_t kAmrCoarseBit = 1 << 30;

// Linear interpolation in time of a coarse cell, x at w = 0 and y at w = 1,
// one rounding (the same in the fill kernels and in the gathering patch
// kernel, so that both give the same bits).
__device__ __forceinline__ float amr_lerp(float x, float y, float w) {
  return __fmaf_rn(w, y - x, x);
}
__device__ __forceinline__ double amr_lerp(double x, double y, double w) {
  return __fma_rn(w, y - x, x);
}

// One decoded entry of the source map: where the five variables of a tile
// cell come from. get() loads unconditionally (the pointers and stride are
// chosen per kind), so that the loads of a cell issue together.
template <class S> struct AmrSrc {
  const S* a;     // same-level cell, coarse old state, or special state
  const S* b;     // coarse new state (= a for the other kinds)
  int stride;     // between variables: kAmrInt, or 1 for a special state
  bool coarse;    // interpolate in time between a and b
  bool invalid;   // out-of-range entry: NaN
  __device__ __forceinline__ S get(int v, S w) const {
    const S x = a[v * stride], y = b[v * stride];
    const S r = coarse ? amr_lerp(x, y, w) : x;
    return invalid ? S(__longlong_as_double(0x7ff8000000000000ULL)) : r;
  }
};

// Decodes map entry m: >= 0 without kAmrCoarseBit -> same[q]; with it ->
// (old[q], new[q]); < 0 -> special[-1 - m]; out of range -> invalid (its
// pointers then address same[0], which exists).
template <class S>
__device__ __forceinline__ AmrSrc<S> amr_decode(int32_t m, const S* same, const S* old_,
                                                const S* new_, int64_t ncells,
                                                const S* special, int nspecial) {
  if (m < 0) {
    const int k = -1 - m;
    const bool ok = k < nspecial;
    const S* s = ok ? special + k * 5 : same;
    return AmrSrc<S>{s, s, 1, false, !ok};
  }
  const bool coarse = (m & kAmrCoarseBit) != 0;
  const int64_t src = m & ~kAmrCoarseBit;
  const bool ok = src < ncells;
  const int64_t sp = src / kAmrInt, sc = src - sp * kAmrInt;
  const int64_t off = ok ? sp * 5 * kAmrInt + sc : 0;
  const S* x = (coarse ? old_ : same) + off;
  const S* y = (coarse ? new_ : same) + off;
  return AmrSrc<S>{x, y, kAmrInt, coarse, !ok};
}

// ghosted[p][v][c] for p in [p0, p0 + n), c in the 12^3 tile, from
// map[p][c]: >= 0 without kAmrCoarseBit -> cur[q] (q = patch * 512 + cell);
// with kAmrCoarseBit -> (1 - w) prev[q] + w cur[q]; < 0 -> special[-1 - m].
template <class S>
__global__ void amr_fill_kernel(const S* __restrict__ cur, const S* __restrict__ prev,
                                S* __restrict__ ghosted, const int32_t* __restrict__ map,
                                int64_t p0, int64_t n, int64_t ncells, S w,
                                const S* __restrict__ special, int nspecial) {
  const int64_t total = n * kAmrTile;
  const S nan = S(__longlong_as_double(0x7ff8000000000000ULL));
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = q / kAmrTile;
    const int c = int(q - pl * kAmrTile);
    const int64_t p = p0 + pl;
    const int32_t m = map[p * kAmrTile + c];
    S* g = ghosted + p * 5 * kAmrTile + c;
    if (m < 0) {
      const int k = -1 - m;
      const bool ok = k < nspecial;
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v * kAmrTile] = ok ? special[k * 5 + v] : nan;
      continue;
    }
    const bool coarse = (m & kAmrCoarseBit) != 0;
    const int64_t src = m & ~kAmrCoarseBit;
    if (src >= ncells) {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v * kAmrTile] = nan;
      continue;
    }
    const int64_t sp = src / kAmrInt, sc = src - sp * kAmrInt;
    const S* a = cur + sp * 5 * kAmrInt + sc;
    if (coarse) {
      const S* b = prev + sp * 5 * kAmrInt + sc;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const S x = b[v * kAmrInt], y = a[v * kAmrInt];
        g[v * kAmrTile] = amr_lerp(x, y, w);
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v * kAmrTile] = a[v * kAmrInt];
    }
  }
}

// The same fill, four consecutive tile cells per thread: one 16-byte map
// load, twenty independent gathers in flight, and one 4-wide store per
// variable (map and ghosted rows 16-byte aligned, which the launcher checks).
template <class S> __device__ __forceinline__ void store4(S* d, const S (&v)[4]);
template <> __device__ __forceinline__ void store4<float>(float* d, const float (&v)[4]) {
  *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void store4<double>(double* d, const double (&v)[4]) {
  reinterpret_cast<double2*>(d)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(d)[1] = make_double2(v[2], v[3]);
}

template <class S>
__global__ void amr_fill4_kernel(const S* __restrict__ cur, const S* __restrict__ prev,
                                 S* __restrict__ ghosted, const int32_t* __restrict__ map,
                                 int64_t p0, int64_t n, int64_t ncells, S w,
                                 const S* __restrict__ special, int nspecial) {
  constexpr int kQ = kAmrTile / 4;  // 432 groups of four cells per tile
  const int64_t total = n * kQ;
  const S nan = S(__longlong_as_double(0x7ff8000000000000ULL));
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = q / kQ;
    const int c0 = int(q - pl * kQ) * 4;
    const int64_t p = p0 + pl;
    const int4 m4 = *reinterpret_cast<const int4*>(map + p * kAmrTile + c0);
    const int32_t ms[4] = {m4.x, m4.y, m4.z, m4.w};
    S val[5][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int32_t m = ms[e];
      if (m < 0) {
        const int k = -1 - m;
        const bool ok = k < nspecial;
#pragma unroll
        for (int v = 0; v < 5; ++v) val[v][e] = ok ? special[k * 5 + v] : nan;
        continue;
      }
      const bool coarse = (m & kAmrCoarseBit) != 0;
      const int64_t src = m & ~kAmrCoarseBit;
      if (src >= ncells) {
#pragma unroll
        for (int v = 0; v < 5; ++v) val[v][e] = nan;
        continue;
      }
      const int64_t sp = src / kAmrInt, sc = src - sp * kAmrInt;
      const S* a = cur + sp * 5 * kAmrInt + sc;
      if (coarse) {
        const S* b = prev + sp * 5 * kAmrInt + sc;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const S x = b[v * kAmrInt], y = a[v * kAmrInt];
          val[v][e] = amr_lerp(x, y, w);
        }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) val[v][e] = a[v * kAmrInt];
      }
    }
    S* g = ghosted + p * 5 * kAmrTile + c0;
#pragma unroll
    for (int v = 0; v < 5; ++v) store4(g + v * kAmrTile, val[v]);
  }
}

// Every cell of the listed parent patches becomes the mean of the 2x2x2
// cells of the child that covers it. children[r] = {parent, child of octant
// 0..7} (octant = cx + 2 cy + 4 cz). The eight values are summed pairwise in
// a fixed order, then scaled by 1/8 (exact).
template <class S>
__global__ void amr_restrict_kernel(S* __restrict__ cur, const int32_t* __restrict__ children,
                                    int64_t nparent, int64_t npatch_total) {
  const int64_t total = nparent * kAmrInt;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / kAmrInt;
    const int c = int(q - r * kAmrInt);
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int32_t par = children[r * 9];
    const int32_t ch = children[r * 9 + 1 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2)];
    if (par < 0 || par >= npatch_total || ch < 0 || ch >= npatch_total) continue;
    const int fi = 2 * (i & 3), fj = 2 * (j & 3), fk = 2 * (k & 3);
    const int f0 = (fk * 8 + fj) * 8 + fi;
    const S* fsrc = cur + (int64_t)ch * 5 * kAmrInt;
    S* dst = cur + (int64_t)par * 5 * kAmrInt + c;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const S* f = fsrc + v * kAmrInt + f0;
      const S s0 = f[0] + f[1], s1 = f[8] + f[9], s2 = f[64] + f[65], s3 = f[72] + f[73];
      dst[v * kAmrInt] = ((s0 + s1) + (s2 + s3)) * S(0.125);
    }
  }
}

// Eq. (Unphysical result) of a corrected state, evaluated in double with
// IEEE operations in a fixed order (no contraction), for both storage types:
// D > 0 and A = eD (eD + 2) - m2 > 2e-16 with eD = Etilde/D and
// m2 = |M|^2/D^2 (the original scheme, ori = 1: (E/D)^2 - m2 - 1).
template <class S> __device__ __forceinline__ bool amr_physical(const S (&u)[5], int ori) {
  const double D = double(u[0]);
  if (!(D > 0.0)) return false;
  const double M2 = __dadd_rn(__dadd_rn(__dmul_rn(double(u[1]), double(u[1])),
                                        __dmul_rn(double(u[2]), double(u[2]))),
                              __dmul_rn(double(u[3]), double(u[3])));
  const double m2 = __ddiv_rn(M2, __dmul_rn(D, D));
  const double eD = __ddiv_rn(double(u[4]), D);
  const double A = ori ? __dsub_rn(__dsub_rn(__dmul_rn(eD, eD), m2), 1.0)
                       : __dsub_rn(__dmul_rn(eD, __dadd_rn(eD, 2.0)), m2);
  return A > 2e-16;
}

// Flux correction of unrefined coarse patches (Section 3.3 (4)).
// faces[r] = {coarse patch, then for each patch face f = 0..5 (-x, +x, -y,
// +y, -z, +z) the four fine patches across it, ordered qa + 2 qb by the
// quadrant of the face (qa along the lower transverse axis), or -1 where the
// face does not border the finer level}. flux_* are patch-face fluxes
// [patch][6][5][64] (face cell t = a + 8 b, a along the lower transverse
// axis). A coarse cell on face f gets U += s (dt/dh) (F_coarse - <F_fine>),
// s = +1 on a high face, -1 on a low one, <F_fine> the mean over the 2x2
// fine faces and the two fine substeps; a cell on several such faces (an
// edge or corner) takes their corrections in face order. If the corrected
// state fails Eq. (Unphysical result), the cell keeps its uncorrected state
// (the paper ignores the correction on failed cells) and, when `skipped` is
// given, adds one to *skipped. One block per listed coarse patch, one thread
// per cell with all five variables.
template <class S>
__global__ void amr_flux_correct_kernel(S* __restrict__ cur, const S* __restrict__ flux_c,
                                        const S* __restrict__ flux_f0,
                                        const S* __restrict__ flux_f1,
                                        const int32_t* __restrict__ faces, int64_t nface_rows,
                                        const double* __restrict__ dt_dh,
                                        int64_t npatch_total, int ori,
                                        int32_t* __restrict__ skipped) {
  constexpr int kF = 6 * 5 * 64;
  for (int64_t r = blockIdx.x; r < nface_rows; r += gridDim.x) {
    const int32_t cp = faces[r * 25];
    if (cp < 0 || cp >= npatch_total) continue;  // uniform per block
    const S coef = S(dt_dh[2 * cp] / dt_dh[2 * cp + 1]);
    const int32_t* row = faces + r * 25 + 1;
    for (int c = threadIdx.x; c < kAmrInt; c += blockDim.x) {
      const int ijk[3] = {c & 7, (c >> 3) & 7, c >> 6};
      S* u = cur + (int64_t)cp * 5 * kAmrInt + c;
      S un[5];
      bool touched = false;
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, high = f & 1;
        if (ijk[d] != (high ? 7 : 0) || row[4 * f] < 0) continue;
        // face cell (a, b): a along the lower transverse axis
        const int a = d == 0 ? ijk[1] : ijk[0];
        const int b = d == 2 ? ijk[1] : ijk[2];
        const int32_t fine = row[4 * f + (a >> 2) + 2 * (b >> 2)];
        if (fine < 0 || fine >= npatch_total) continue;
        if (!touched) {
#pragma unroll
          for (int v = 0; v < 5; ++v) un[v] = u[v * kAmrInt];
          touched = true;
        }
        // fine face cells covering coarse face cell (a, b)
        const int t0 = (2 * (b & 3)) * 8 + 2 * (a & 3);
        const int fside = 2 * d + (1 - high);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const S* F0 = flux_f0 + (int64_t)fine * kF + (fside * 5 + v) * 64;
          const S* F1 = flux_f1 + (int64_t)fine * kF + (fside * 5 + v) * 64;
          const S fsum = ((F0[t0] + F0[t0 + 1]) + (F0[t0 + 8] + F0[t0 + 9])) +
                         ((F1[t0] + F1[t0 + 1]) + (F1[t0 + 8] + F1[t0 + 9]));
          const S fc = flux_c[(int64_t)cp * kF + (f * 5 + v) * 64 + b * 8 + a];
          const S du = coef * (fc - S(0.125) * fsum);
          un[v] = high ? un[v] + du : un[v] - du;
        }
      }
      if (!touched) continue;
      if (amr_physical(un, ori)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v * kAmrInt] = un[v];
      } else if (skipped) {
        atomicAdd(skipped, 1);
      }
    }
  }
}

}  // namespace srhd
