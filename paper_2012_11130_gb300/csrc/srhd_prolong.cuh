// Limited linear prolongation of the ghost zones of a fine AMR level from
// the coarser level, with the primitive-variable fallback of Section 3.3 (3)
// of arXiv 2012.11130 (ghost-zone interpolation).
//
// Each row of the prolongation table is one fine ghost cell whose source is
// the coarser level: the coarse cell C containing it, C's six face
// neighbours along -x, +x, -y, +y, -z, +z (flat coarse cell indices
// patch * 512 + cell, or -1 where the coarse level does not cover the
// neighbour) and three parity bits (bit d set: the fine cell lies in the
// upper half of C along axis d, i.e. its centre is a quarter of a coarse
// cell above C's centre, otherwise a quarter below). The coarse states are
// first taken at the fine substep's time, (1 - w) prev + w cur (amr_lerp,
// as in the piecewise-constant fill; prev itself at w = 0). Per axis the
// slope is the minmod of the two one-sided differences (0 where a
// neighbour is missing or the differences have opposite signs), and the
// fine value is
//   U_f = U_C + sum_d (+-1/4) slope_d      (axes in the order x, y, z).
// The conserved variables are interpolated; where the result fails
// Eq. (Unphysical result) (amr_physical), the primitive variables
// (rho, U^x, U^y, U^z, p) of the same coarse states are interpolated the same
// way and converted back: along each axis the minmod slope moves a value by
// at most a quarter of its smaller one-sided difference, so rho and p stay
// above a quarter of the coarse values, and any positive rho and p with any
// four-velocity pass Eq. (Unphysical result). The offsets +-1/4 of the
// eight fine cells of a coarse cell cancel, so the conserved interpolation
// keeps the coarse cell's mean.
#pragma once

#include <cstdint>

#include "srhd_amr.cuh"
#include "srhd_physics.cuh"

namespace srhd {

constexpr int kProlongRow = 8;  // int32 per table row: C, -x, +x, -y, +y, -z, +z, parity bits

template <class R> __device__ __forceinline__ R minmod2(R a, R b) {
  return (a * b > R(0)) ? (fabs(a) < fabs(b) ? a : b) : R(0);
}

// out[r][v] for the rows r < nrows of `table`; fallbacks (nullable) counts
// the rows interpolated in primitive variables. A row whose centre index is
// out of range gives NaN; an out-of-range neighbour counts as missing.
template <class P, class E>
__global__ void __launch_bounds__(128)
    amr_prolong_kernel(const typename P::S* __restrict__ cur, const typename P::S* __restrict__ prev,
                       const int32_t* __restrict__ table, int64_t nrows, typename P::S w,
                       typename P::S* __restrict__ out, int64_t ncells, int maxit, int ori, E eos,
                       int32_t* __restrict__ fallbacks) {
  using S = typename P::S;
  const S nan = S(__longlong_as_double(0x7ff8000000000000ULL));
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* row = table + r * kProlongRow;
    S* o = out + r * 5;
    const int32_t qc = row[0];
    if (qc < 0 || qc >= ncells) {
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] = nan;
      continue;
    }
    const int par = row[7];
    // the coarse state of flat cell q at the substep's time (at w = 0 the
    // state before the coarse step itself)
    auto coarse = [&](int32_t q, S (&u)[5]) {
      const int64_t p = q / kAmrInt, c = q - p * kAmrInt;
      const S* a = prev + p * 5 * kAmrInt + c;
      const S* b = cur + p * 5 * kAmrInt + c;
      if (w == S(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = a[v * kAmrInt];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = amr_lerp(a[v * kAmrInt], b[v * kAmrInt], w);
      }
    };
    S uc[5], un[6][5];
    coarse(qc, uc);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int32_t q = row[1 + k];
      if (q >= 0 && q < ncells) coarse(q, un[k]);
      else {  // missing neighbour: zero one-sided difference
#pragma unroll
        for (int v = 0; v < 5; ++v) un[k][v] = uc[v];
      }
    }
    // limited linear interpolation of five values per cell (conserved or
    // primitive), centre c, neighbours n
    auto interp = [&](const S (&c)[5], const S (&n)[6][5], S (&f)[5]) {
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] = c[v];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const S q = ((par >> d) & 1) ? S(0.25) : S(-0.25);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const S lo = c[v] - n[2 * d][v], hi = n[2 * d + 1][v] - c[v];
          f[v] = f[v] + q * minmod2(lo, hi);
        }
      }
    };
    S f[5];
    interp(uc, un, f);
    if (!amr_physical(f, ori)) {
      // Section 3.3 (3): interpolate the primitive variables instead
      S wc[5], wn[6][5];
      PrimX<S> W;
      con2pri<P>(uc[0], uc[1], uc[2], uc[3], uc[4], W, maxit, S(0), ori, eos);
      wc[0] = W.rho; wc[1] = W.u[0]; wc[2] = W.u[1]; wc[3] = W.u[2]; wc[4] = W.p;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        con2pri<P>(un[k][0], un[k][1], un[k][2], un[k][3], un[k][4], W, maxit, S(0), ori, eos);
        wn[k][0] = W.rho; wn[k][1] = W.u[0]; wn[k][2] = W.u[1]; wn[k][3] = W.u[2];
        wn[k][4] = W.p;
      }
      S wf[5];
      interp(wc, wn, wf);
      PrimX<S> Wf;
      Wf.rho = wf[0]; Wf.u[0] = wf[1]; Wf.u[1] = wf[2]; Wf.u[2] = wf[3]; Wf.p = wf[4];
      prim2con(Wf, f, ori, eos);
      if (fallbacks) atomicAdd(fallbacks, 1);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) o[v] = f[v];
  }
}

}  // namespace srhd
