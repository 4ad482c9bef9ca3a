// Kernels of libsrhd (sm_103a): the fused per-patch MUSCL-Hancock step
// (Sections 3.1-3.3 of arXiv 2012.11130), batched conversions, the CFL
// reduction (Section 3.2) and a uniform-grid ghost fill.
//
// Fused patch kernel (one CTA per 8^3 patch, persistent over the batch):
//   phase 1  con2pri of the 1376 cells of the 12^3 tile that the step reads
//            -> primitive tile in shared memory [5][12^3]
//   phase 2  for the 896 cells whose face states are used (the 8^3 interior
//            and one layer around it, edges excluded): PLM slopes in x, y, z,
//            six face states, their conserved form and physical fluxes, and
//            the Hancock half step; the 3456 predicted face states that a
//            flux uses go to shared memory [3][2][5][576]
//   phase 3  per face (3 x 576): con2pri of both predicted states, HLLC or
//            HLLE; the flux overwrites the left state in place
//   phase 4  conservative update of the interior, Eq. (Unphysical result)
//            check, optional CFL bound of the new state
//   retry    if any predicted state or updated cell is unphysical, phases 2-4
//            are redone with the limiter coefficient times retry_factor
//            (block-wide vote), down to theta = 0 (piecewise constant)
// While phase 4 runs, the copy engine stages the CTA's next tile in the
// right-state face slots: one bulk copy per variable for a ghosted batch;
// for a uniform grid the patch interior and its six face slabs as seven
// dense boxes (bulk copies where the source is contiguous, tensor-map
// copies where it is strided; see patch_kernel).
// Shared memory: 27648 elements of S (primitive tile, face slots, warm-start
// values of the tile cells: 216 KB double, 108 KB float).
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "srhd_amr.cuh"
#include "srhd_physics.cuh"

namespace srhd {

constexpr int kG = 12;              // ghosted patch edge
constexpr int kN = 8;               // interior edge
constexpr int kGC = kG * kG * kG;   // 1728 ghosted cells
constexpr int kNC = kN * kN * kN;   // 512 interior cells
constexpr int kNF = 9 * 8 * 8;      // 576 faces per direction
constexpr int kRC = 512 + 6 * 64;   // 896 reconstructed cells

// CODE_STAGE_TIMEOUT: a bulk copy of a tile did not complete within the
// bounded wait of bulk::wait; the CTA stopped (see patch_kernel)
enum { CODE_UNPHYSICAL = 1, CODE_BAD_INPUT = 2, CODE_NOCONV = 4, CODE_STAGE_TIMEOUT = 8 };

struct PatchArgs {
  const void* in;         // [np][5][12^3], or the interior array of a gathered grid
  void* out;              // [np][5][8^3] (advance) or nullptr
  void* pflux;            // [np][6][5][64] (nullable)
  void* face_flux;        // [np][3][5][576] (flux mode)
  int npatch;
  const double* dt_dh;    // [np][2]
  const int32_t* worklist;
  int32_t* status;        // [np] (nullable)
  double* partial_dt;     // [grid] CFL partial minima (nullable = no CFL)
  int32_t* partial_bad;   // [grid]
  double theta0, retry_factor, theta_floor, cfl;
  int riemann, cfl_mode, ndim, maxit;
  int flux_only;
  int ori;                // 1: original scheme (total energy E, flux M)
  double eos_gamma;       // Gamma of the polytropic EoS (used by the EosPoly kernels)
  // Uniform-grid gather (gather = 1): `in` is the interior array [.][5][8^3]
  // of a grid of gnx*gny*gnz patches (patch (ix,iy,iz) at (iz*gny + iy)*gnx
  // + ix); item p is grid patch gp0 + p, whose 12^3 tile the kernel reads
  // from that patch and its neighbours (gbc*: 0 periodic, 1 outflow).
  int gather, gnx, gny, gnz, gbcx, gbcy, gbcz;
  int64_t gp0;
  // gather = 1 with tma = 1: tmap holds 5-D tensor maps of `in` viewed as
  // [patch][var][z][y][x], with boxes (x, y, z, var, patch) of a patch
  // interior (8, 8, 8, 5, 1) and of its x (4, 8, 8, 5, 1), y (8, 2, 8, 5, 1)
  // and z (8, 8, 2, 5, 1) face slabs (kTmapCenter .. kTmapZ).
  int tma;
  CUtensorMap tmap[4];
  // Uniform-grid gather with primitive cache (gather = 3): as gather = 1,
  // but the tile's primitives and solver variable come from prim_in
  // [.][6][8^3] (rho, U^x, U^y, U^z, p, tau of every grid patch) instead of
  // a conversion, and the new state's are written to prim_out [n][6][8^3].
  const void* prim_in;
  void* prim_out;
  // AMR gather (gather = 2): tile cell c of item p comes from amr_map[p][c]
  // (as in srhd_amr_fill_ghosts): entries without the coarse bit from `in`
  // (the same level's state before the step), coarse entries
  // (1 - amr_w) amr_old + amr_w amr_new, negative ones amr_special.
  const int32_t* amr_map;
  const void* amr_old;
  const void* amr_new;
  const void* amr_special;
  int64_t amr_ncells;
  double amr_w;
  int amr_nspecial;
};

// ---- bulk asynchronous copies into shared memory -------------------------
// The copy engine (cp.async.bulk) moves a contiguous global range into
// shared memory and reports the bytes on an mbarrier; the threads that then
// see the barrier's phase complete also see the data. Waits are bounded.
namespace bulk {
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Thread's earlier shared-memory accesses (made visible to it by a barrier)
// are ordered before later copies into the same bytes.
__device__ __forceinline__ void fence_before_copy() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(mbar)),
               "r"(bytes)
               : "memory");
}
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(mbar))
      : "memory");
}
// Tensor copy of the box at coordinates (x, y, z, v, p) of the 5-D map into
// shared memory (128-byte aligned), completing on mbar. x * element size
// must be a multiple of 16 bytes.
__device__ __forceinline__ void copy_box(void* dst, const CUtensorMap* map, int x, int y, int z,
                                         int v, int p, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(p),
      "r"(saddr(mbar))
      : "memory");
}
// Wait for the completion of the barrier phase of this parity; false if it
// has not completed after kWaitPolls polls (each non-blocking, then a sleep
// of about kPollNs nanoseconds: about 1 s in all).
constexpr int kWaitPolls = 1 << 23;
constexpr unsigned kPollNs = 128;
__device__ __forceinline__ bool test_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(ok)
      : "r"(saddr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait(uint64_t* mbar, uint32_t parity) {
  for (int i = 0; i < kWaitPolls; ++i) {
    if (test_wait(mbar, parity)) return true;
    __nanosleep(kPollNs);
  }
  return false;
}
}  // namespace bulk

// EoS object of a launch: the TM tag, or the polytropic EoS with the
// launch's Gamma.
template <class E> __device__ __forceinline__ E make_eos(const PatchArgs& a);
template <> __device__ __forceinline__ EosTM make_eos<EosTM>(const PatchArgs&) { return EosTM{}; }
template <> __device__ __forceinline__ EosPoly make_eos<EosPoly>(const PatchArgs& a) {
  return EosPoly{a.eos_gamma};
}

template <class S> struct SmemLayout {  // S: storage type
  static constexpr size_t prim_elems = 5 * kGC;        // primitive tile
  static constexpr size_t face_elems = 3 * 2 * 5 * kNF; // predicted faces / fluxes
  static constexpr size_t ht_elems = kGC;               // warm-start values of the tile cells (kRatio)
  static constexpr size_t bytes = (prim_elems + face_elems + ht_elems) * sizeof(S);
};

// Class of a ghosted coordinate: 0 interior [2,9], 1 first ghost layer,
// 2 second ghost layer.
__device__ __forceinline__ int gclass(int g) {
  return (g >= 2 && g <= 9) ? 0 : ((g == 1 || g == 10) ? 1 : 2);
}

// Cells of the 12^3 tile whose primitives the step reads: at most one
// coordinate in the ghost zone, or two coordinates both in the first layer.
__device__ __forceinline__ bool tile_cell_needed(int gx, int gy, int gz) {
  int a = gclass(gx), b = gclass(gy), c = gclass(gz);
  int nout = (a > 0) + (b > 0) + (c > 0);
  if (nout <= 1) return true;
  return nout == 2 && a <= 1 && b <= 1 && c <= 1;
}

constexpr int kTileNeeded = 512 + 768 + 96;  // 1376 cells read by the step

// r-th cell of the tile that the step reads (tile_cell_needed), as a
// 12^3 index: the 8^3 interior, then the six faces two layers deep, then the
// twelve edges of the first layer.
__device__ __forceinline__ void needed_tile_coords(int r, int (&g)[3]) {
  if (r < 512) {
    g[0] = 2 + (r & 7); g[1] = 2 + ((r >> 3) & 7); g[2] = 2 + (r >> 6);
  } else if (r < 1280) {
    const int q = r - 512, f = q >> 7, rem = q & 127;
    const int axis = f >> 1, depth = 1 + (rem >> 6), t = rem & 63;
    const int along = (f & 1) ? 9 + depth : 2 - depth;
    const int u = 2 + (t & 7), v = 2 + (t >> 3);
    if (axis == 0) { g[0] = along; g[1] = u; g[2] = v; }
    else if (axis == 1) { g[0] = u; g[1] = along; g[2] = v; }
    else { g[0] = u; g[1] = v; g[2] = along; }
  } else {
    const int q = r - 1280, e = q >> 3, w = 2 + (q & 7);
    const int pair = e >> 2;
    const int ca = (e & 1) ? 10 : 1, cb = (e & 2) ? 10 : 1;
    if (pair == 0) { g[0] = ca; g[1] = cb; g[2] = w; }
    else if (pair == 1) { g[0] = ca; g[1] = w; g[2] = cb; }
    else { g[0] = w; g[1] = ca; g[2] = cb; }
  }
}
__device__ __forceinline__ int needed_tile_cell(int r) {
  int g[3];
  needed_tile_coords(r, g);
  return (g[2] * kG + g[1]) * kG + g[0];
}

// r-th reconstructed cell, interior coordinates in [-1, 8].
__device__ __forceinline__ void recon_cell(int r, int& i, int& j, int& k) {
  if (r < kNC) {
    i = r & 7; j = (r >> 3) & 7; k = r >> 6;
    return;
  }
  r -= kNC;
  int layer = r >> 6, q = r & 63, a = q & 7, b = q >> 3;
  int side = (layer & 1) ? 8 : -1;
  switch (layer >> 1) {
    case 0: i = side; j = a; k = b; break;
    case 1: i = a; j = side; k = b; break;
    default: i = a; j = b; k = side; break;
  }
}

// Source of a ghosted coordinate g in [-GH, kN+GH) of the patch at pc along an
// axis of n patches: the patch q holding it and the cell l in that patch.
// Periodic boundaries (bc 0) wrap the patch index, outflow ones (bc 1) take
// the edge cell of the patch itself.
__device__ __forceinline__ void ghost_src(int g, int pc, int n, int bc, int& q, int& l) {
  const int o = g < 0 ? -1 : (g >= kN ? 1 : 0);
  q = pc + o;
  l = g - kN * o;
  if (q < 0 || q >= n) {
    if (bc == 0) {
      q = q < 0 ? q + n : q - n;
    } else {
      q = pc;
      l = o < 0 ? 0 : kN - 1;
    }
  }
}

__device__ __forceinline__ int tile_index(int i, int j, int k) {  // interior coords
  return ((k + 2) * kG + (j + 2)) * kG + (i + 2);
}

// Face index along d at face coordinate fd (0..8), transverse coordinates
// of the two others; faces ordered with extent 9 along d, x fastest.
template <int d> __device__ __forceinline__ int face_index(int i, int j, int k, int fd) {
  if (d == 0) return (k * 8 + j) * 9 + fd;
  if (d == 1) return (k * 9 + fd) * 8 + i;
  return (fd * 8 + j) * 8 + i;
}

// Face slots are side-major: the 15 slots [d][v] of the left states (side
// 0, overwritten by the fluxes in phase 3) first, then the 15 of the right
// states (side 1). Nothing reads the right states after phase 3, so from
// then until phase 2 of the next patch their 3 x 5 x 576 = 5 x 12^3
// elements hold the next patch's ghosted tile.
template <class S> __device__ __forceinline__ S* face_slot(S* face, int d, int side, int v) {
  return face + ((side * 3 + d) * 5 + v) * kNF;
}
constexpr int kStageOffset = 3 * 5 * kNF;  // first right-state slot
static_assert(5 * kGC == 3 * 5 * kNF, "a ghosted tile fills the right-state slots");

// Uniform-grid tiles staged by the copy engine (gather modes 1 and 3): the
// patch interior and its six face slabs, five variables each, as dense boxes in
// the stage (x fastest): centre [5][8][8][8], then -x and +x [5][8][8][4]
// (neighbour x 4..7 and 0..3: rows of 16 bytes), -y and +y [5][8][2][8]
// (neighbour y 6..7 and 0..1), -z and +z [5][2][8][8]. Every box starts on
// a 128-byte boundary. The 96 first-layer edge cells of the tile are not
// staged.
enum { kTmapCenter = 0, kTmapX = 1, kTmapY = 2, kTmapZ = 3 };
constexpr int kBoxC = 8 * 8 * 8 * 5;
constexpr int kBoxX = 4 * 8 * 8 * 5;
constexpr int kBoxY = 8 * 2 * 8 * 5;
constexpr int kBoxZ = 8 * 8 * 2 * 5;
constexpr int kBoxXm = kBoxC, kBoxXp = kBoxXm + kBoxX, kBoxYm = kBoxXp + kBoxX,
              kBoxYp = kBoxYm + kBoxY, kBoxZm = kBoxYp + kBoxY, kBoxZp = kBoxZm + kBoxZ;
constexpr int kBoxTotal = kBoxZp + kBoxZ;  // 7680
static_assert(kBoxTotal <= 5 * kGC, "the staged boxes fit the stage");
static_assert(kBoxC % 32 == 0 && kBoxX % 32 == 0 && kBoxY % 32 == 0 && kBoxZ % 32 == 0,
              "boxes of 4-byte elements start on 128-byte boundaries");

// Stage offset of variable 0 of tile cell (gx, gy, gz) and the distance
// between its variables, for a cell in the interior or in one face slab;
// false for the first-layer edge cells (two coordinates in the ghost zone).
__device__ __forceinline__ bool box_offset(int gx, int gy, int gz, int& off, int& vstride) {
  const int ax = gx < 2 ? 0 : (gx < 10 ? 1 : 2);
  const int ay = gy < 2 ? 0 : (gy < 10 ? 1 : 2);
  const int az = gz < 2 ? 0 : (gz < 10 ? 1 : 2);
  const int x = gx - 2, y = gy - 2, z = gz - 2;  // patch-interior coordinates
  if (ay == 1 && az == 1) {
    if (ax == 1) {
      off = (z * 8 + y) * 8 + x;
      vstride = 512;
    } else {  // -x slab: gx 0, 1 -> neighbour x 6, 7 -> box x 2, 3; +x: gx 10, 11 -> 0, 1
      off = (ax == 0 ? kBoxXm + gx + 2 : kBoxXp + gx - 10) + (z * 8 + y) * 4;
      vstride = 256;
    }
    return true;
  }
  if (ax == 1 && az == 1) {  // -y slab: gy 0, 1 -> neighbour y 6, 7 -> box y 0, 1
    off = (ay == 0 ? kBoxYm + gy * 8 : kBoxYp + (gy - 10) * 8) + z * 16 + x;
    vstride = 128;
    return true;
  }
  if (ax == 1 && ay == 1) {  // -z slab: gz 0, 1 -> box z 0, 1
    off = (az == 0 ? kBoxZm + gz * 64 : kBoxZp + (gz - 10) * 64) + y * 8 + x;
    vstride = 128;
    return true;
  }
  return false;
}

// LAST: the last direction of the cell; its flux difference completes dF,
// so its two face states take the Hancock half step (- half dF) before they
// are stored (the other directions' are updated by halfstep_direction).
// The same for the r-th needed tile cell (needed_tile_coords) directly from
// r, for r < 1280 (the interior and the six face slabs; the first-layer
// edges are not staged): c its 12^3 tile index, off and vs as box_offset,
// nb the patch the cell lies in (0 the patch itself, 1 + f for the face f =
// -x, +x, -y, +y, -z, +z neighbour) and local its 8^3 index there.
__device__ __forceinline__ void staged_cell(int r, int& c, int& off, int& vs, int& nb,
                                            int& local) {
  if (r < kNC) {
    c = tile_index(r & 7, (r >> 3) & 7, r >> 6);
    off = r;
    vs = kNC;
    nb = 0;
    local = r;
    return;
  }
  const int q = r - kNC, f = q >> 7, rem = q & 127;
  const int depth = 1 + (rem >> 6), t = rem & 63;  // ghost layer 1 or 2, face cell
  const int a = t & 7, b = t >> 3;                   // transverse, lower axis first
  const int lo = 8 - depth, hi = depth - 1;          // neighbour cell along the normal
  nb = 1 + f;
  switch (f) {
    case 0: c = tile_index(-depth, a, b); off = kBoxXm + 4 - depth + 4 * t; vs = 256;
            local = t * 8 + lo; break;
    case 1: c = tile_index(7 + depth, a, b); off = kBoxXp + hi + 4 * t; vs = 256;
            local = t * 8 + hi; break;
    case 2: c = tile_index(a, -depth, b); off = kBoxYm + (2 - depth) * 8 + b * 16 + a; vs = 128;
            local = (b * 8 + lo) * 8 + a; break;
    case 3: c = tile_index(a, 7 + depth, b); off = kBoxYp + hi * 8 + b * 16 + a; vs = 128;
            local = (b * 8 + hi) * 8 + a; break;
    case 4: c = tile_index(a, b, -depth); off = kBoxZm + (2 - depth) * 64 + t; vs = 128;
            local = lo * 64 + t; break;
    default: c = tile_index(a, b, 7 + depth); off = kBoxZp + hi * 64 + t; vs = 128;
             local = hi * 64 + t; break;
  }
}

template <int d, bool LAST = false, class R, class S, class E>
__device__ __forceinline__ void recon_direction(const S* prim, int tc, const PrimX<R>& W, R theta,
                                                int i, int j, int k, bool interior, S* face,
                                                R dF[5], int& bad, int ori, const E& eos,
                                                R half = R(0)) {
  constexpr int off = (d == 0) ? 1 : ((d == 1) ? kG : kG * kG);
  R wc[5] = {W.rho, W.u[0], W.u[1], W.u[2], W.p};
  const int cd = (d == 0) ? i : ((d == 1) ? j : k);
  // A face state is stored only where a flux uses it: the transverse
  // coordinates are interior and the face lies in 0..8 along d.
  const bool trans = interior || (cd < 0 || cd > 7);
  if constexpr (sizeof(R) == 4) {
    // float: the minus (lane x) and plus (lane y) face states in packed form
    float2 Wq[5], Uq[5], Fq[5];
    // limited slopes of the variable pairs (rho, U^x), (U^y, U^z) in packed
    // form, p alone
#pragma unroll
    for (int v = 0; v < 4; v += 2) {
      const float2 c = make_float2(wc[v], wc[v + 1]);
      const float2 lo = make_float2(prim[v * kGC + tc - off], prim[(v + 1) * kGC + tc - off]);
      const float2 hi = make_float2(prim[v * kGC + tc + off], prim[(v + 1) * kGC + tc + off]);
      const float2 dW = limited_slope_x2(pk::sub(c, lo), pk::sub(hi, c), theta);
      Wq[v] = pk::fma(pk::s2(dW.x), make_float2(-0.5f, 0.5f), pk::s2(wc[v]));
      Wq[v + 1] = pk::fma(pk::s2(dW.y), make_float2(-0.5f, 0.5f), pk::s2(wc[v + 1]));
    }
    {
      R lo = R(prim[4 * kGC + tc - off]);
      R hi = R(prim[4 * kGC + tc + off]);
      R dW = limited_slope(wc[4] - lo, hi - wc[4], theta);
      Wq[4] = pk::fma(pk::s2(dW), make_float2(-0.5f, 0.5f), pk::s2(wc[4]));
    }
    bool okm, okp;
    prim2con_flux_x2<d>(Wq, Uq, Fq, okm, okp, ori, eos);
    if (!okm || !okp) bad = 1;
#pragma unroll
    for (int v = 0; v < 5; ++v) dF[v] = dF[v] + (Fq[v].y - Fq[v].x);
    if constexpr (LAST) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Uq[v] = pk::fma(pk::s2(-half), pk::s2(dF[v]), Uq[v]);
    }
    if (trans && cd >= 0) {
      int fi = face_index<d>(i, j, k, cd);
#pragma unroll
      for (int v = 0; v < 5; ++v) face_slot(face, d, 1, v)[fi] = S(Uq[v].x);
    }
    if (trans && cd <= 7) {
      int fi = face_index<d>(i, j, k, cd + 1);
#pragma unroll
      for (int v = 0; v < 5; ++v) face_slot(face, d, 0, v)[fi] = S(Uq[v].y);
    }
  } else {
    PrimX<R> Wm, Wp;
    R fm[5], fp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R lo = R(prim[v * kGC + tc - off]);
      R hi = R(prim[v * kGC + tc + off]);
      R dW = limited_slope(wc[v] - lo, hi - wc[v], theta);
      fm[v] = wc[v] - R(0.5) * dW;
      fp[v] = wc[v] + R(0.5) * dW;
    }
    Wm.rho = fm[0]; Wm.u[0] = fm[1]; Wm.u[1] = fm[2]; Wm.u[2] = fm[3]; Wm.p = fm[4];
    Wp.rho = fp[0]; Wp.u[0] = fp[1]; Wp.u[1] = fp[2]; Wp.u[2] = fp[3]; Wp.p = fp[4];
    R Um[5], Up[5], Fm[5], Fp[5];
    if (!prim2con(Wm, Um, ori, eos)) bad = 1;
    if (!prim2con(Wp, Up, ori, eos)) bad = 1;
    phys_flux<d>(Wm, Um, Fm, ori);
    phys_flux<d>(Wp, Up, Fp, ori);
#pragma unroll
    for (int v = 0; v < 5; ++v) dF[v] = dF[v] + (Fp[v] - Fm[v]);
    if constexpr (LAST) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Um[v] = Um[v] - half * dF[v];
        Up[v] = Up[v] - half * dF[v];
      }
    }
    if (trans && cd >= 0) {
      int fi = face_index<d>(i, j, k, cd);
#pragma unroll
      for (int v = 0; v < 5; ++v) face_slot(face, d, 1, v)[fi] = S(Um[v]);
    }
    if (trans && cd <= 7) {
      int fi = face_index<d>(i, j, k, cd + 1);
#pragma unroll
      for (int v = 0; v < 5; ++v) face_slot(face, d, 0, v)[fi] = S(Up[v]);
    }
  }
}

template <int d, class R, class S>
__device__ __forceinline__ void halfstep_direction(int i, int j, int k, bool interior, S* face,
                                                   const R dF[5], R half) {
  const int cd = (d == 0) ? i : ((d == 1) ? j : k);
  const bool trans = interior || (cd < 0 || cd > 7);
  if (trans && cd >= 0) {
    int fi = face_index<d>(i, j, k, cd);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      S* s = face_slot(face, d, 1, v) + fi;
      *s = S(R(*s) - half * dF[v]);
    }
  }
  if (trans && cd <= 7) {
    int fi = face_index<d>(i, j, k, cd + 1);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      S* s = face_slot(face, d, 0, v) + fi;
      *s = S(R(*s) - half * dF[v]);
    }
  }
}

// Tile index of the cell on the left (side 0) or right (side 1) of face fi
// along d: the cell whose half-step face state sits in that slot.
template <int d> __device__ __forceinline__ int face_owner(int fi, int side) {
  int i, j, k;
  if (d == 0) {
    const int q = fi / 9;                 // (k, j); fd = fi - 9 q
    i = fi - 9 * q - 1 + side; j = q & 7; k = q >> 3;
  } else if (d == 1) {
    const int r = fi >> 3, q = r / 9;     // r = k * 9 + fd
    i = fi & 7; j = r - 9 * q - 1 + side; k = q;
  } else {
    i = fi & 7; j = (fi >> 3) & 7; k = (fi >> 6) - 1 + side;
  }
  return tile_index(i, j, k);
}

// Riemann flux of face fi along d from the two predicted states in its
// slots; their Newton solves start warm from the cells they belong to (the
// predicted state differs from the cell state by half a limited slope and
// half a time step): hts holds the cells' converged solver variable, or with
// RATIO its ratio to the cold start (rt), which the solve multiplies by the
// predicted state's own cold start.
template <int d, class P, bool PAIR, class E, bool RATIO>
__device__ __forceinline__ int face_flux(typename P::S* face, const typename P::S* hts, int fi,
                                         int solver, int maxit, int& code, int ori,
                                         const E& eos) {
  using S = typename P::S;
  using R = S;
  const S gL = hts[face_owner<d>(fi, 0)], gR = hts[face_owner<d>(fi, 1)];
  S UL[5], UR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    UL[v] = face_slot(face, d, 0, v)[fi];
    UR[v] = face_slot(face, d, 1, v)[fi];
  }
  PrimX<R> WL, WR;
  int sl, sr;
  if constexpr (PAIR) {
    con2pri_x2<P, E, true, RATIO>(UL, UR, WL, WR, maxit, sl, sr, gL, gR, ori, eos);
  } else {
    sl = con2pri<P, E, true, RATIO>(UL[0], UL[1], UL[2], UL[3], UL[4], WL, maxit, gL, ori, eos);
    sr = con2pri<P, E, true, RATIO>(UR[0], UR[1], UR[2], UR[3], UR[4], WR, maxit, gR, ori, eos);
  }
  if (sl == 2 || sr == 2) code |= CODE_NOCONV;
  int fail = (sl == 1 || sr == 1);
  R FL_[5] = {R(UL[0]), R(UL[1]), R(UL[2]), R(UL[3]), R(UL[4])};
  R FR_[5] = {R(UR[0]), R(UR[1]), R(UR[2]), R(UR[3]), R(UR[4])};
  R F[5];
  riemann<d>(solver, WL, FL_, WR, FR_, F, ori, eos);
#pragma unroll
  for (int v = 0; v < 5; ++v) face_slot(face, d, 0, v)[fi] = S(F[v]);
  return fail;
}

// GATHER: 0 ghosted batch (a.in), 1 uniform-grid gather, 2 AMR gather
// (a.gather must equal it).
template <class P, int NT, int MINB, bool PAIR, class E = EosTM, int GATHER = 0>
__global__ void __launch_bounds__(NT, MINB) patch_kernel(const __grid_constant__ PatchArgs a) {
  static_assert(NT % 32 == 0 && NT >= 64 && NT <= 1024, "block size");
  using S = typename P::S;
  using R = S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* prim = reinterpret_cast<S*>(smem_raw);
  S* face = prim + SmemLayout<S>::prim_elems;
  S* hts = face + SmemLayout<S>::face_elems;
  __shared__ double s_red[NT / 32];
  __shared__ int s_bad[NT / 32];
  // AMR gather: 1 if some interior tile cell of the patch is not mapped to
  // the patch's own cell of the same level
  [[maybe_unused]] __shared__ int s_nonid;
  const int tid = threadIdx.x;
  const int maxit = a.maxit;
  const int ori = a.ori;
  const E eos = make_eos<E>(a);

  // Limiter constants of the launch and the step factors of the current
  // patch in the arithmetic type, converted by one thread: per-thread double
  // arithmetic would queue every warp of the float kernels on the FP64 pipe
  // (1/64 of the FP32 rate) and keep doubles in registers through the phases.
  __shared__ R s_kc[3];     // theta0, retry_factor, theta_floor * theta0
  __shared__ R s_pc[3];     // dt/dh, dt/(2 dh), C dh (of the current patch)
  __shared__ double s_dtl;  // light-speed CFL mode: min of C dh over the CTA's patches
  if (tid == 0) {
    s_kc[0] = R(a.theta0);
    s_kc[1] = R(a.retry_factor);
    s_kc[2] = R(a.theta_floor * a.theta0);
    s_dtl = DBL_MAX;
  }
  constexpr R kRMax = sizeof(R) == 4 ? R(FLT_MAX) : R(DBL_MAX);
  R dtr = kRMax;  // signal-speed CFL mode: min of C dh / S_max (this thread's cells)
  int cfl_bad = 0;

  // Ghosted batch: while a patch is updated (phase 4) the copy engine brings
  // the CTA's next tile into the right-state face slots (`stage`), where
  // phase 1 of that patch reads it. Needs 16-byte aligned tiles. Uniform
  // grid (gather modes 1 and 3 with tensor maps): the same with the seven
  // boxes of the next patch's tile (box_offset; in mode 3 variables 0..4 of
  // the primitive cache; mode 1 fills the centre and z boxes with plain bulk
  // copies, the rest with tensor copies), for patches whose six face neighbours exist
  // (periodic or interior; other patches, and the first patch of each CTA,
  // gather with plain loads). s_stg:
  // bit 0 the parity of the s_mbar phase that the next copy completes, bit 1
  // set while a copy is issued and not yet waited for. It is kept in shared
  // memory (read by all threads, written by one between barriers) so that
  // it holds no register through the phases.
  [[maybe_unused]] S* stage = face + kStageOffset;
  [[maybe_unused]] __shared__ __align__(8) uint64_t s_mbar;
  [[maybe_unused]] __shared__ uint32_t s_stg;
  [[maybe_unused]] __shared__ int s_stage_timeout;
  constexpr bool kStaged = GATHER == 0 || GATHER == 1 || GATHER == 3;
  // hts holds the tile cells' rt (the ratio of the converged solver
  // variable to its cold start): from the cold conversions of phase 1, or
  // from the cached primitives (mode 3, rt_of_prims); the warm starts of
  // phases 3 and 4 multiply it by each state's own cold start
  constexpr bool kRatio = true;
  auto stage_ok = [&]() {
    // tensor copies need 128-byte aligned destinations (the boxes are laid
    // out on 128-byte boundaries from `stage`)
    if constexpr (GATHER == 1 || GATHER == 3)
      return a.tma != 0 && (bulk::saddr(stage) & 127) == 0;
    return GATHER == 0 && !a.flux_only && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0;
  };
  if constexpr (kStaged) {
    if (stage_ok() && tid == 0) {
      bulk::init(&s_mbar);
      s_stg = 0;
      s_stage_timeout = 0;
    }
  }
  // A copy that did not complete in time sets s_stage_timeout. The patch
  // that waited for it is marked CODE_STAGE_TIMEOUT, the CTA's CFL minimum
  // becomes NaN, and before its next patch (or at its end) the CTA waits
  // once more, bounded, for the last copy it issued and stops; its remaining
  // patches keep their previous contents and status.
  // Parity of the s_mbar phase of the last copy issued, from a stage word
  // (a phase that never began reads as complete).
  [[maybe_unused]] auto last_copy_parity = [](uint32_t st) {
    return (st & 2) ? (st & 1) : ((st & 1) ^ 1);
  };
  [[maybe_unused]] auto stage_abort = [&](int p, uint32_t st) {
    if (tid == 0) {
      if (a.status) a.status[p] = CODE_STAGE_TIMEOUT << 8;
      if (a.partial_dt) {
        a.partial_dt[blockIdx.x] = DBL_MAX;
        a.partial_bad[blockIdx.x] = 1;
      }
    }
    bulk::wait(&s_mbar, last_copy_parity(st));
  };

  for (int w = blockIdx.x; w < a.npatch; w += gridDim.x) {
    const int p = a.worklist ? a.worklist[w] : w;
    const S* base = static_cast<const S*>(a.in);
    // ghosted batch: this patch's tile; gathered grid: this patch's interior
    int gpx = 0, gpy = 0, gpz = 0;
    const S* in;
    if constexpr (GATHER == 2) {
      in = base;
    } else if constexpr (GATHER == 1 || GATHER == 3) {
      const int64_t q = a.gp0 + p;
      gpx = int(q % a.gnx);
      gpy = int((q / a.gnx) % a.gny);
      gpz = int(q / ((int64_t)a.gnx * a.gny));
      in = base + q * 5 * kNC;
    } else {
      in = base + (size_t)p * 5 * kGC;
    }
    // the five conserved variables of tile cell c (12^3 index)
    // AMR gather: the patch's map row; phase 4 reads the old state directly
    // unless s_nonid, else through the map
    [[maybe_unused]] const int32_t* amap = nullptr;
    [[maybe_unused]] S aw = S(0);
    if constexpr (GATHER == 2) {
      amap = a.amr_map + (size_t)p * kGC;
      aw = S(a.amr_w);
    }
    [[maybe_unused]] auto amr_cell = [&](int32_t m) {
      return amr_decode<S>(m, base, static_cast<const S*>(a.amr_old),
                           static_cast<const S*>(a.amr_new), a.amr_ncells,
                           static_cast<const S*>(a.amr_special), a.amr_nspecial);
    };
    // stage word as this patch starts; bit 1: its tile was copied during the
    // last update and phase 1 reads it from `stage`
    [[maybe_unused]] uint32_t st1 = 0;
    // r: the cell's rank in the list of needed tile cells (the first kNC
    // are the interior cells in 8^3 order)
    auto load_tile = [&](int c, [[maybe_unused]] int r, S (&U)[5]) {
      if constexpr (GATHER == 2) {
        const int32_t m = amap[c];
        const AmrSrc<S> src = amr_cell(m);
#pragma unroll
        for (int v = 0; v < 5; ++v) U[v] = src.get(v, aw);
        if (r < kNC && m != (int32_t)((int64_t)p * kNC + r)) s_nonid = 1;
      } else if constexpr (GATHER == 1) {
        if ((st1 & 2) && r < kNC + 768) {  // staged interior or face-slab cell
          int cs, off, vs, nb, local;
          staged_cell(r, cs, off, vs, nb, local);
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = stage[off + v * vs];
          return;
        }
        const int gz = c / (kG * kG), gy = (c / kG) % kG, gx = c % kG;
        int qx, lx, qy, ly, qz, lz;
        ghost_src(gx - 2, gpx, a.gnx, a.gbcx, qx, lx);
        ghost_src(gy - 2, gpy, a.gny, a.gbcy, qy, ly);
        ghost_src(gz - 2, gpz, a.gnz, a.gbcz, qz, lz);
        const S* src = base + ((int64_t)(qz * a.gny + qy) * a.gnx + qx) * (5 * kNC) +
                       ((lz * kN + ly) * kN + lx);
#pragma unroll
        for (int v = 0; v < 5; ++v) U[v] = src[v * kNC];
      } else {
        if (st1 & 2) {
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = stage[v * kGC + c];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = in[v * kGC + c];
        }
      }
    };
    // old state of interior cell c (8^3 index; tc its tile index), variable v
    // (AMR gather: through the map, see amr_cell)
    auto old_state = [&](int v, int c, int tc) -> S {
      if constexpr (GATHER == 1 || GATHER == 3) return in[v * kNC + c];
      else return in[v * kGC + tc];
    };
    int code = 0;

    if constexpr (GATHER == 2) {
      if (tid == 0) s_nonid = 0;
    }
    __syncthreads();  // the previous patch is done with shared memory
    if constexpr (kStaged) {
      if (stage_ok()) st1 = s_stg;
      if ((st1 & 2) && !bulk::wait(&s_mbar, st1 & 1)) s_stage_timeout = 1;
    }
    // ---- phase 1: primitive tile ------------------------------------------
    if constexpr (GATHER == 3) {
      // the primitives that the previous step kept for the cells of the
      // tile: a gather, no conversion; the warm-start ratio of the later
      // solves from them in closed form (rt_of_prims). A state left
      // unphysical by that step is stored as NaN.
      const S* pbase = static_cast<const S*>(a.prim_in);
      int r0 = tid;
      if (st1 & 2) {
        // staged tile (all six face neighbours exist, wrapping where
        // periodic): the interior and face-slab cells by the closed-form
        // mapping, entirely from the stage
        for (int r = tid; r < kNC + 768; r += NT) {
          int c, off, vs, nb, local;
          staged_cell(r, c, off, vs, nb, local);
          S w[6];
#pragma unroll
          for (int v = 0; v < 5; ++v) w[v] = stage[off + v * vs];
          w[5] = rt_of_prims(eos, w[0], w[1], w[2], w[3], w[4]);
          if (!(w[0] > S(0) && w[4] > S(0) && isfinite(w[1] + w[2] + w[3])))
            code |= CODE_BAD_INPUT;
#pragma unroll
          for (int v = 0; v < 5; ++v) prim[v * kGC + c] = w[v];
          hts[c] = w[5];
        }
        r0 = kNC + 768 + tid;  // the first-layer edge cells below
      }
      for (int r = r0; r < kTileNeeded; r += NT) {
        int g[3];
        needed_tile_coords(r, g);
        const int c = (g[2] * kG + g[1]) * kG + g[0];
        int qx, lx, qy, ly, qz, lz;
        ghost_src(g[0] - 2, gpx, a.gnx, a.gbcx, qx, lx);
        ghost_src(g[1] - 2, gpy, a.gny, a.gbcy, qy, ly);
        ghost_src(g[2] - 2, gpz, a.gnz, a.gbcz, qz, lz);
        const S* src = pbase + ((int64_t)(qz * a.gny + qy) * a.gnx + qx) * (6 * kNC) +
                       ((lz * kN + ly) * kN + lx);
        S w[6];
        int off, vs;
        if ((st1 & 2) && box_offset(g[0], g[1], g[2], off, vs)) {
          // variables 0..4 staged by the tensor copies
#pragma unroll
          for (int v = 0; v < 5; ++v) w[v] = stage[off + v * vs];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) w[v] = __ldg(src + v * kNC);
        }
        w[5] = rt_of_prims(eos, w[0], w[1], w[2], w[3], w[4]);
        if (!(w[0] > S(0) && w[4] > S(0) && isfinite(w[1] + w[2] + w[3])))
          code |= CODE_BAD_INPUT;
#pragma unroll
        for (int v = 0; v < 5; ++v) prim[v * kGC + c] = w[v];
        hts[c] = w[5];
      }
    } else if constexpr (PAIR) {
      for (int r = tid; r < kTileNeeded / 2; r += NT) {
        const int ca = needed_tile_cell(r), cb = needed_tile_cell(r + kTileNeeded / 2);
        S Ua[5], Ub[5];
        load_tile(ca, r, Ua);
        load_tile(cb, r + kTileNeeded / 2, Ub);
        PrimX<R> Wa, Wb;
        int sa, sb;
        con2pri_x2<P, E, false, true>(Ua, Ub, Wa, Wb, maxit, sa, sb, S(0), S(0), ori, eos);
        if (sa == 1 || sb == 1) code |= CODE_BAD_INPUT;
        if (sa == 2 || sb == 2) code |= CODE_NOCONV;
        prim[ca] = S(Wa.rho);
        prim[kGC + ca] = S(Wa.u[0]);
        prim[2 * kGC + ca] = S(Wa.u[1]);
        prim[3 * kGC + ca] = S(Wa.u[2]);
        prim[4 * kGC + ca] = S(Wa.p);
        hts[ca] = S(Wa.rt);
        hts[cb] = S(Wb.rt);
        prim[cb] = S(Wb.rho);
        prim[kGC + cb] = S(Wb.u[0]);
        prim[2 * kGC + cb] = S(Wb.u[1]);
        prim[3 * kGC + cb] = S(Wb.u[2]);
        prim[4 * kGC + cb] = S(Wb.p);
      }
    } else {
      for (int r = tid; r < kTileNeeded; r += NT) {
        const int c = needed_tile_cell(r);
        S U[5];
        load_tile(c, r, U);
        PrimX<R> W;
        int st = con2pri<P, E, false, true>(U[0], U[1], U[2], U[3], U[4], W, maxit, S(0), ori,
                                            eos);
        if (st == 1) code |= CODE_BAD_INPUT;
        if (st == 2) code |= CODE_NOCONV;
        prim[c] = S(W.rho);
        prim[kGC + c] = S(W.u[0]);
        prim[2 * kGC + c] = S(W.u[1]);
        prim[3 * kGC + c] = S(W.u[2]);
        prim[4 * kGC + c] = S(W.p);
        hts[c] = S(W.rt);
      }
    }
    // the last thread, which has the least phase-1 work, converts the step
    // factors of the patch (read after the barrier; the previous patch's
    // readers are past its final barrier)
    if (tid == NT - 1) {
      const double dt = a.dt_dh[2 * p], dh = a.dt_dh[2 * p + 1];
      const R coef = R(dt) / R(dh);
      s_pc[0] = coef;
      s_pc[1] = R(0.5) * coef;
      s_pc[2] = R(a.cfl * dh);
      if (a.partial_dt && a.cfl_mode == 1) s_dtl = fmin(s_dtl, a.cfl * dh);
    }
    const int bad_input = __syncthreads_or(code & CODE_BAD_INPUT);
    if constexpr (kStaged) {
      if (stage_ok()) {
        if (s_stage_timeout) {
          stage_abort(p, st1);
          return;
        }
        if ((st1 & 2) && tid == 0) s_stg = (st1 & 1) ^ 1;  // waited: next parity, none pending
      }
    }

    int retries = 0;
    int final_code = 0;
    R att_smax = R(0);          // signal mode: largest S_max of the attempt
    int att_bad = 0;
    if (!bad_input) {
      R theta = s_kc[0];
      for (;;) {
        // ---- phase 2: reconstruction + Hancock half step --------------------
        int fail = 0;
        for (int r = tid; r < kRC; r += NT) {
          int i, j, k;
          recon_cell(r, i, j, k);
          const bool interior = r < kNC;
          const int tc = tile_index(i, j, k);
          PrimX<R> W;
          W.rho = R(prim[tc]);
          W.u[0] = R(prim[kGC + tc]);
          W.u[1] = R(prim[2 * kGC + tc]);
          W.u[2] = R(prim[3 * kGC + tc]);
          W.p = R(prim[4 * kGC + tc]);
          R dF[5] = {R(0), R(0), R(0), R(0), R(0)};
          const R half = s_pc[1];
          recon_direction<0>(prim, tc, W, theta, i, j, k, interior, face, dF, fail, ori, eos);
          recon_direction<1>(prim, tc, W, theta, i, j, k, interior, face, dF, fail, ori, eos);
          recon_direction<2, true>(prim, tc, W, theta, i, j, k, interior, face, dF, fail, ori,
                                   eos, half);
          halfstep_direction<0>(i, j, k, interior, face, dF, half);
          halfstep_direction<1>(i, j, k, interior, face, dF, half);
        }
        __syncthreads();
        // ---- phase 3: Riemann fluxes ----------------------------------------
        for (int f = tid; f < 3 * kNF; f += NT) {
          const int d = f / kNF, fi = f - d * kNF;
          if (d == 0)
            fail |= face_flux<0, P, PAIR, E, kRatio>(face, hts, fi, a.riemann, maxit, code, ori,
                                                     eos);
          else if (d == 1)
            fail |= face_flux<1, P, PAIR, E, kRatio>(face, hts, fi, a.riemann, maxit, code, ori,
                                                     eos);
          else
            fail |= face_flux<2, P, PAIR, E, kRatio>(face, hts, fi, a.riemann, maxit, code, ori,
                                                     eos);
        }
        fail = __syncthreads_or(fail);
        if (a.flux_only) {
          if (fail) final_code |= CODE_UNPHYSICAL;
          break;
        }
        const bool last = (theta == R(0));
        // ---- phase 4: conservative update ----------------------------------
        att_smax = R(0);
        att_bad = 0;
        if (!fail || last) {
          if constexpr (GATHER == 0) {
            // the right states are consumed (phase 3 ended at a barrier):
            // copy the CTA's next tile into their slots. The last thread
            // issues the copy: it has no update work when NT > 256.
            const int wn = w + gridDim.x;  // the CTA's next work item
            if (stage_ok() && wn < a.npatch) {
              if (tid == NT - 1) {
                constexpr uint32_t kVarBytes = kGC * sizeof(S);
                const int pn = a.worklist ? a.worklist[wn] : wn;
                const S* src = base + (size_t)pn * 5 * kGC;
                bulk::fence_before_copy();
                bulk::expect(&s_mbar, 5 * kVarBytes);
#pragma unroll
                for (int v = 0; v < 5; ++v)
                  bulk::copy(stage + v * kGC, src + v * kGC, kVarBytes, &s_mbar);
                s_stg |= 2;  // read next after the phase-4 barrier
              }
            }
          } else if constexpr (GATHER == 1 || GATHER == 3) {
            // uniform grid: the seven boxes of the CTA's next patch, when its
            // six face neighbours exist (mode 3: variables 0..4 of the cache)
            const int wn = w + gridDim.x;
            if (stage_ok() && wn < a.npatch && tid == NT - 1) {
              const int64_t qn = a.gp0 + wn;
              const int cx = int(qn % a.gnx), cy = int((qn / a.gnx) % a.gny);
              const int cz = int(qn / ((int64_t)a.gnx * a.gny));
              // neighbour coordinate along an axis of n patches, -1 if none
              auto nb = [](int c, int n, int bc) {
                if (c >= 0 && c < n) return c;
                if (bc != 0) return -1;
                return c < 0 ? c + n : c - n;
              };
              const int xm = nb(cx - 1, a.gnx, a.gbcx), xp = nb(cx + 1, a.gnx, a.gbcx);
              const int ym = nb(cy - 1, a.gny, a.gbcy), yp = nb(cy + 1, a.gny, a.gbcy);
              const int zm = nb(cz - 1, a.gnz, a.gbcz), zp = nb(cz + 1, a.gnz, a.gbcz);
              if ((xm | xp | ym | yp | zm | zp) >= 0) {
                auto pid = [&](int ix, int iy, int iz) { return (iz * a.gny + iy) * a.gnx + ix; };
                // the patch interior (variables 0..4 contiguous) and the two
                // z slabs (two contiguous planes per variable) are plain
                // bulk copies; the x and y slabs, strided, are tensor boxes
                bulk::fence_before_copy();
                bulk::expect(&s_mbar, kBoxTotal * sizeof(S));
                if constexpr (GATHER == 1) {
                  // the interior array's patch interior (variables
                  // contiguous) and z slabs (two contiguous planes per
                  // variable) as plain bulk copies
                  const S* zms = base + (int64_t)pid(cx, cy, zm) * (5 * kNC) + 6 * 64;
                  const S* zps = base + (int64_t)pid(cx, cy, zp) * (5 * kNC);
                  bulk::copy(stage, base + qn * (5 * kNC), kBoxC * sizeof(S), &s_mbar);
#pragma unroll
                  for (int v = 0; v < 5; ++v) {
                    bulk::copy(stage + kBoxZm + v * 128, zms + v * kNC, 128 * sizeof(S), &s_mbar);
                    bulk::copy(stage + kBoxZp + v * 128, zps + v * kNC, 128 * sizeof(S), &s_mbar);
                  }
                } else {
                  bulk::copy_box(stage, &a.tmap[kTmapCenter], 0, 0, 0, 0, int(qn), &s_mbar);
                  bulk::copy_box(stage + kBoxZm, &a.tmap[kTmapZ], 0, 0, 6, 0, pid(cx, cy, zm),
                                 &s_mbar);
                  bulk::copy_box(stage + kBoxZp, &a.tmap[kTmapZ], 0, 0, 0, 0, pid(cx, cy, zp),
                                 &s_mbar);
                }
                bulk::copy_box(stage + kBoxXm, &a.tmap[kTmapX], 4, 0, 0, 0, pid(xm, cy, cz),
                               &s_mbar);
                bulk::copy_box(stage + kBoxXp, &a.tmap[kTmapX], 0, 0, 0, 0, pid(xp, cy, cz),
                               &s_mbar);
                bulk::copy_box(stage + kBoxYm, &a.tmap[kTmapY], 0, 6, 0, 0, pid(cx, ym, cz),
                               &s_mbar);
                bulk::copy_box(stage + kBoxYp, &a.tmap[kTmapY], 0, 0, 0, 0, pid(cx, yp, cz),
                               &s_mbar);
                s_stg |= 2;  // read next after the phase-4 barrier
              }
            }
          }
          S* out = static_cast<S*>(a.out) + (size_t)p * 5 * kNC;
          int fail4 = 0;
          // PAIR: the work item c0 in [0, 256) updates cells c0 and c0 + 256
          // and converts both in lockstep for the CFL bound (for any NT)
          constexpr int NPC = PAIR ? 2 : 1;
          constexpr int kItems = kNC / NPC;
          // the signal-speed CFL bound converts the new state; its status 1
          // is the Eq. (Unphysical result) check, otherwise made directly.
          // The primitive cache converts it in any case, for prim_out.
          const bool signal = (a.partial_dt && a.cfl_mode != 1) || GATHER == 3;
          for (int c0 = tid; c0 < kItems; c0 += NT) {
            const R coef = s_pc[0];
            S Un[NPC][5];
            S g0[NPC];  // tau of the cell before the step: warm start of the CFL solve
            if constexpr (PAIR && sizeof(R) == 4) {
              // both cells' divergences in packed arithmetic
              int tcq[2], cq[2], fq[2][6];
              [[maybe_unused]] AmrSrc<S> osrc[2];
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int c = c0 + q * kItems;
                const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
                cq[q] = c;
                tcq[q] = tile_index(i, j, k);
                if constexpr (GATHER == 2) {
                  if (s_nonid) osrc[q] = amr_cell(amap[tcq[q]]);
                  else osrc[q] = AmrSrc<S>{base + (size_t)p * 5 * kNC + c,
                                           base + (size_t)p * 5 * kNC + c, kNC, false, false};
                }
                g0[q] = hts[tcq[q]];
                fq[q][0] = face_index<0>(i, j, k, i);
                fq[q][1] = face_index<0>(i, j, k, i + 1);
                fq[q][2] = face_index<1>(i, j, k, j);
                fq[q][3] = face_index<1>(i, j, k, j + 1);
                fq[q][4] = face_index<2>(i, j, k, k);
                fq[q][5] = face_index<2>(i, j, k, k + 1);
              }
              const float2 mcoef = pk::s2(-float(coef));
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                auto ld = [&](int dd, int e) {
                  const S* f = face_slot(face, dd, 0, v);
                  return make_float2(f[fq[0][e]], f[fq[1][e]]);
                };
                const float2 div = pk::add(pk::add(pk::sub(ld(0, 1), ld(0, 0)),
                                                   pk::sub(ld(1, 3), ld(1, 2))),
                                           pk::sub(ld(2, 5), ld(2, 4)));
                float2 old;
                if constexpr (GATHER == 2)
                  old = make_float2(osrc[0].get(v, aw), osrc[1].get(v, aw));
                else
                  old = make_float2(old_state(v, cq[0], tcq[0]), old_state(v, cq[1], tcq[1]));
                const float2 un = pk::fma(mcoef, div, old);
                Un[0][v] = un.x;
                Un[1][v] = un.y;
                out[v * kNC + c0] = un.x;
                out[v * kNC + c0 + kItems] = un.y;
              }
            } else {
#pragma unroll
              for (int q = 0; q < NPC; ++q) {
                const int c = c0 + q * kItems;
                const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
                const int tc = tile_index(i, j, k);
                g0[q] = hts[tc];
                [[maybe_unused]] AmrSrc<S> os1;
                if constexpr (GATHER == 2) {
                  if (s_nonid) os1 = amr_cell(amap[tc]);
                  else os1 = AmrSrc<S>{base + (size_t)p * 5 * kNC + c,
                                       base + (size_t)p * 5 * kNC + c, kNC, false, false};
                }
                const int fx0 = face_index<0>(i, j, k, i), fx1 = face_index<0>(i, j, k, i + 1);
                const int fy0 = face_index<1>(i, j, k, j), fy1 = face_index<1>(i, j, k, j + 1);
                const int fz0 = face_index<2>(i, j, k, k), fz1 = face_index<2>(i, j, k, k + 1);
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                  R div = R(0);
                  div = div + (R(face_slot(face, 0, 0, v)[fx1]) - R(face_slot(face, 0, 0, v)[fx0]));
                  div = div + (R(face_slot(face, 1, 0, v)[fy1]) - R(face_slot(face, 1, 0, v)[fy0]));
                  div = div + (R(face_slot(face, 2, 0, v)[fz1]) - R(face_slot(face, 2, 0, v)[fz0]));
                  S old;
                  if constexpr (GATHER == 2) old = os1.get(v, aw);
                  else old = old_state(v, c, tc);
                  Un[q][v] = S(R(old) - coef * div);
                  out[v * kNC + c] = Un[q][v];
                }
              }
            }
            if (signal) {
              PrimX<R> W[NPC];
              int st[NPC];
              if constexpr (PAIR) {
                con2pri_x2<P, E, true, kRatio>(Un[0], Un[1], W[0], W[1], maxit, st[0], st[1],
                                               g0[0], g0[NPC - 1], ori, eos);
              } else {
                st[0] = con2pri<P, E, true, kRatio>(Un[0][0], Un[0][1], Un[0][2], Un[0][3],
                                                    Un[0][4], W[0], maxit, g0[0], ori, eos);
              }
              if constexpr (GATHER == 3) {
                // keep the new state's primitives (NaN where unphysical)
                S* po = static_cast<S*>(a.prim_out) + (size_t)p * 6 * kNC;
#pragma unroll
                for (int q = 0; q < NPC; ++q) {
                  const int c = c0 + q * kItems;
                  po[c] = S(W[q].rho);
                  po[kNC + c] = S(W[q].u[0]);
                  po[2 * kNC + c] = S(W[q].u[1]);
                  po[3 * kNC + c] = S(W[q].u[2]);
                  po[4 * kNC + c] = S(W[q].p);
                  po[5 * kNC + c] = S(W[q].tau);
                }
              }
#pragma unroll
              for (int q = 0; q < NPC; ++q) {
                // the largest signal speed of the patch; dt = C dh / S_max once
                if (st[q] != 1) {
                  if (GATHER != 3 || a.cfl_mode != 1)
                    att_smax = fmax(att_smax, smax_of(W[q], a.ndim, eos));
                } else {
                  att_bad = 1;
                  fail4 = 1;
                }
              }
            } else {
#pragma unroll
              for (int q = 0; q < NPC; ++q) {
                typename P::AT Ac, m2c;
                if (!A_and_m2<P>(Un[q][0], Un[q][1], Un[q][2], Un[q][3], Un[q][4], Ac, m2c, ori))
                  fail4 = 1;
              }
            }
          }
          fail = __syncthreads_or(fail4) | fail;
        }
        if (!fail) break;
        if (last) { final_code |= CODE_UNPHYSICAL; break; }
        if constexpr (kStaged) {
          // the retry's phase 2 rewrites the right-state slots: let the copy
          // land first; the next patch then reads its tile from `in`
          const uint32_t st = stage_ok() ? s_stg : 0u;
          if (st & 2) {
            if (!bulk::wait(&s_mbar, st & 1)) s_stage_timeout = 1;
            __syncthreads();
            if (tid == 0) s_stg = (st & 1) ^ 1;  // read next in the retry's phase 4
          }
        }

        ++retries;
        theta = theta * s_kc[1];
        if (theta < s_kc[2]) theta = R(0);
      }
      if (att_smax > R(0)) dtr = fmin(dtr, s_pc[2] / att_smax);
      cfl_bad |= att_bad;
    } else {
      final_code |= CODE_BAD_INPUT;
      cfl_bad = 1;
      if (!a.flux_only) {
        S* out = static_cast<S*>(a.out) + (size_t)p * 5 * kNC;
        for (int c = tid; c < 5 * kNC; c += NT) out[c] = S(__longlong_as_double(0x7ff8000000000000ULL));
        if constexpr (GATHER == 3) {
          S* po = static_cast<S*>(a.prim_out) + (size_t)p * 6 * kNC;
          for (int c = tid; c < 6 * kNC; c += NT) po[c] = S(__longlong_as_double(0x7ff8000000000000ULL));
        }
      }
    }
    // ---- outputs ----------------------------------------------------------
    if (a.flux_only && !bad_input) {
      S* ff = static_cast<S*>(a.face_flux) + (size_t)p * 3 * 5 * kNF;
      for (int q = tid; q < 3 * 5 * kNF; q += NT) {
        ff[q] = face[q];  // the flux slots (side 0), [d][v][576]
      }
    }
    if (a.pflux && !a.flux_only && !bad_input) {
      S* pf = static_cast<S*>(a.pflux) + (size_t)p * 6 * 5 * 64;
      for (int q = tid; q < 6 * 5 * 64; q += NT) {
        int side = q / 320, rem = q - side * 320, v = rem >> 6, t = rem & 63;
        int d = side >> 1, fd = (side & 1) ? 8 : 0;
        int a0 = t & 7, b0 = t >> 3;  // transverse coordinates, lower axis fastest
        int fi = (d == 0) ? face_index<0>(0, a0, b0, fd)
                          : (d == 1) ? face_index<1>(a0, 0, b0, fd) : face_index<2>(a0, b0, 0, fd);
        pf[q] = face_slot(face, d, 0, v)[fi];
      }
    }
    code = __syncthreads_or(code & CODE_NOCONV);
    if constexpr (kStaged) {
      if (tid == 0 && stage_ok() && s_stage_timeout) {  // a retry's wait ran out
        final_code |= CODE_STAGE_TIMEOUT;
        cfl_bad = 1;
      }
    }
    if (tid == 0 && a.status) {
      final_code |= code ? CODE_NOCONV : 0;
      a.status[p] = (final_code << 8) | (retries < 255 ? retries : 255);
    }
  }
  if constexpr (kStaged) {
    // a copy that ran out on the CTA's last patch: wait once more (bounded)
    if (stage_ok() && s_stage_timeout) bulk::wait(&s_mbar, last_copy_parity(s_stg));
  }

  // ---- CFL partial minimum of this CTA -------------------------------------
  if (a.partial_dt) {
    for (int o = 16; o > 0; o >>= 1) {
      dtr = fmin(dtr, __shfl_xor_sync(0xffffffffu, dtr, o));
      cfl_bad |= __shfl_xor_sync(0xffffffffu, cfl_bad, o);
    }
    if ((tid & 31) == 0) {
      s_red[tid >> 5] = dtr < kRMax ? double(dtr) : DBL_MAX;
      s_bad[tid >> 5] = cfl_bad;
    }
    __syncthreads();
    if (tid == 0) {
      double m = s_dtl;
      int b = 0;
      for (int q = 0; q < NT / 32; ++q) { m = fmin(m, s_red[q]); b |= s_bad[q]; }
      a.partial_dt[blockIdx.x] = m;
      a.partial_bad[blockIdx.x] = b;
    }
  }
}

// Final reduction of the CFL partial minima (one block).
__global__ void cfl_finalize_kernel(const double* partial, const int32_t* bad, int n,
                                    double* dt_out);

// ---- batched conversions ----------------------------------------------------
template <class S, class E = EosTM>
__global__ void prim2con_kernel(const S* prim, S* cons, int64_t n, int64_t stride, int ori,
                                E eos) {
  using R = S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    PrimX<R> W;
    W.rho = prim[i];
    W.u[0] = prim[stride + i];
    W.u[1] = prim[2 * stride + i];
    W.u[2] = prim[3 * stride + i];
    W.p = prim[4 * stride + i];
    R U[5];
    prim2con(W, U, ori, eos);
#pragma unroll
    for (int v = 0; v < 5; ++v) cons[v * stride + i] = U[v];
  }
}

template <class P, class E = EosTM>
__global__ void con2pri_kernel(const typename P::S* cons, typename P::S* prim, int64_t n,
                               int64_t stride, int32_t* status, int maxit, int ori, E eos) {
  using S = typename P::S;
  using R = S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    PrimX<R> W;
    int st = con2pri<P>(cons[i], cons[stride + i], cons[2 * stride + i], cons[3 * stride + i],
                        cons[4 * stride + i], W, maxit, S(0), ori, eos);
    prim[i] = W.rho;
    prim[stride + i] = W.u[0];
    prim[2 * stride + i] = W.u[1];
    prim[3 * stride + i] = W.u[2];
    prim[4 * stride + i] = W.p;
    if (status) status[i] = st;
  }
}

// Primitive cache of interior patches: cons [np][5][8^3] -> prim
// [np][6][8^3] = (rho, U^x, U^y, U^z, p, tau), tau the converged solver
// variable (conic parameter for TM, htilde for the polytropic EoS); NaN for
// unphysical cells.
template <class P, class E = EosTM>
__global__ void prim_cache_kernel(const typename P::S* cons, typename P::S* prim, int64_t ncell,
                                  int maxit, int ori, E eos) {
  using S = typename P::S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pt = i / kNC;
    const int c = int(i - pt * kNC);
    const S* u = cons + pt * 5 * kNC + c;
    S* w = prim + pt * 6 * kNC + c;
    PrimX<S> W;
    con2pri<P>(u[0], u[kNC], u[2 * kNC], u[3 * kNC], u[4 * kNC], W, maxit, S(0), ori, eos);
    w[0] = W.rho;
    w[kNC] = W.u[0];
    w[2 * kNC] = W.u[1];
    w[3 * kNC] = W.u[2];
    w[4 * kNC] = W.p;
    w[5 * kNC] = W.tau;
  }
}

// CFL bound over interior patches [np][5][8^3]; per-block partial minima.
template <class P, int NT, class E = EosTM>
__global__ void __launch_bounds__(NT) cfl_kernel(const typename P::S* cons, int64_t ncell,
                                                 double dh, double cfl, int ndim, int mode,
                                                 int maxit, double* partial, int32_t* bad_out,
                                                 int ori, E eos) {
  using S = typename P::S;
  using R = S;
  __shared__ double s_red[NT / 32];
  __shared__ int s_bad[NT / 32];
  double m = DBL_MAX;
  int bad = 0;
  for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < ncell;
       q += (int64_t)gridDim.x * NT) {
    const int64_t p = q / kNC, c = q - p * kNC;
    const S* b = cons + p * 5 * kNC + c;
    PrimX<R> W;
    int st = con2pri<P>(b[0], b[kNC], b[2 * kNC], b[3 * kNC], b[4 * kNC], W, maxit, S(0), ori,
                        eos);
    if (st == 1) { bad = 1; continue; }
    if (mode == 1) m = fmin(m, cfl * dh);
    else m = fmin(m, cfl * dh / double(smax_of(W, ndim, eos)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { s_red[threadIdx.x >> 5] = m; s_bad[threadIdx.x >> 5] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = DBL_MAX;
    int bb = 0;
    for (int w = 0; w < NT / 32; ++w) { mm = fmin(mm, s_red[w]); bb |= s_bad[w]; }
    partial[blockIdx.x] = mm;
    bad_out[blockIdx.x] = bb;
  }
}

// Ghost fill of a uniform grid of patches (periodic or outflow per axis),
// GH ghost cells per side (2 for the MUSCL-Hancock tiles, 3 for VL), for the
// patches p0 .. p0+nfill-1 (row pl of ghosted holds patch p0+pl). One block
// per patch (grid-stride), one thread per tile row (variable, z, y): the row
// takes its z and y source from the patch or a neighbour, gathers its TE
// cells along x from the rows of the patch and of its two x neighbours, and
// writes them with vector stores when `wide` (ghosted aligned to the store).
// Periodic boundaries wrap the patch index; outflow ones take the edge cell.
template <class S, int TE>
__device__ __forceinline__ void store_row(S* o, const S (&v)[TE], bool wide) {
  if (wide) {
    if constexpr (sizeof(S) == 4 && TE % 4 == 0) {
#pragma unroll
      for (int i = 0; i < TE; i += 4)
        reinterpret_cast<float4*>(o)[i / 4] = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else if constexpr (sizeof(S) == 4) {
#pragma unroll
      for (int i = 0; i < TE; i += 2)
        reinterpret_cast<float2*>(o)[i / 2] = make_float2(v[i], v[i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < TE; i += 2)
        reinterpret_cast<double2*>(o)[i / 2] = make_double2(v[i], v[i + 1]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < TE; ++i) o[i] = v[i];
  }
}

// Byte alignment the vector stores of store_row need.
template <class S, int GH> constexpr int ghost_store_align() {
  return (sizeof(S) == 4 && (kN + 2 * GH) % 4 != 0) ? 8 : 16;
}

template <class S, int GH>
__global__ void __launch_bounds__(256)
    fill_ghosts_kernel(const S* __restrict__ interior, S* __restrict__ ghosted, int npx, int npy,
                       int npz, int bcx, int bcy, int bcz, int64_t p0, int64_t nfill, int wide) {
  constexpr int TE = kN + 2 * GH, TC = TE * TE * TE, ROWS = 5 * TE * TE;
  for (int64_t pl = blockIdx.x; pl < nfill; pl += gridDim.x) {
    const int64_t p = p0 + pl;
    const int px = int(p % npx), py = int((p / npx) % npy);
    const int pz = int(p / ((int64_t)npx * npy));
    int qxl = px - 1, qxr = px + 1;
    bool cl = false, cr = false;
    if (qxl < 0) {
      if (bcx == 0) qxl += npx; else { qxl = px; cl = true; }
    }
    if (qxr >= npx) {
      if (bcx == 0) qxr -= npx; else { qxr = px; cr = true; }
    }
    S* out = ghosted + pl * (5 * TC);
    for (int r = threadIdx.x; r < ROWS; r += blockDim.x) {
      const int v = r / (TE * TE), rem = r - v * (TE * TE);
      const int tz = rem / TE, ty = rem - tz * TE;
      int qz, lz, qy, ly;
      ghost_src(tz - GH, pz, npz, bcz, qz, lz);
      ghost_src(ty - GH, py, npy, bcy, qy, ly);
      const int64_t plane = ((int64_t)qz * npy + qy) * npx;
      const int cell = (lz * kN + ly) * kN;
      const S* rl = interior + ((plane + qxl) * 5 + v) * kNC + cell;
      const S* rc = interior + ((plane + px) * 5 + v) * kNC + cell;
      const S* rr = interior + ((plane + qxr) * 5 + v) * kNC + cell;
      S val[TE];
#pragma unroll
      for (int i = 0; i < GH; ++i) val[i] = rl[cl ? 0 : kN - GH + i];
#pragma unroll
      for (int i = 0; i < kN; ++i) val[GH + i] = rc[i];
#pragma unroll
      for (int i = 0; i < GH; ++i) val[GH + kN + i] = rr[cr ? kN - 1 : i];
      store_row<S, TE>(out + r * TE, val, wide != 0);
    }
  }
}

// Per-precision launchers (explicitly instantiated in srhd_fp64.cu,
// srhd_mixed.cu and srhd_mixed_cf.cu for the tags of srhd_physics.cuh).
constexpr int kPatchVariants = 4;  // launch variants of patch_kernel per precision

// EoS of a launch: poly = 0 selects the Taub-Mathews kernels, 1 the
// polytropic ones with the given Gamma.
struct EosArg {
  int poly;
  double gam;
};

template <class P> struct Launch {
  static cudaError_t setup();
  static int patch_blocks_per_sm(int variant);
  // a.eos_gamma and `poly` select the EoS; the polytropic EoS runs one
  // launch configuration (PolyVariant) whatever the variant
  static cudaError_t patches(const PatchArgs& a, int variant, int poly, int grid, cudaStream_t s);
  static int poly_blocks_per_sm();
  static cudaError_t prim2con(const void* prim, void* cons, int64_t n, int64_t stride, int ori,
                              EosArg eos, int grid, cudaStream_t s);
  static cudaError_t con2pri(const void* cons, void* prim, int64_t n, int64_t stride,
                             int32_t* status, int maxit, int ori, EosArg eos, int grid,
                             cudaStream_t s);
  // primitive cache of npatch interior patches (prim_cache_kernel)
  static cudaError_t prim_cache(const void* cons, void* prim, int64_t npatch, int maxit, int ori,
                                EosArg eos, int grid, cudaStream_t s);
  static cudaError_t cfl(const void* cons, int64_t ncell, double dh, double cfl, int ndim, int mode,
                         int maxit, int ori, EosArg eos, double* partial, int32_t* bad, int grid,
                         cudaStream_t s);
  // the VL integrator (srhd_vl.cuh) on 14^3 tiles
  static cudaError_t patches_vl(const PatchArgs& a, int poly, int grid, cudaStream_t s);
  static int vl_blocks_per_sm(int poly);
  // uniform-grid ghost fill with gh = 2 or 3 ghost cells, patches p0 .. p0+n-1
  static cudaError_t fill_ghosts(const void* interior, void* ghosted, int npx, int npy, int npz,
                                 const int32_t* bc, int gh, int64_t p0, int64_t n, int grid,
                                 cudaStream_t s);
  // limited linear prolongation of AMR ghost cells (srhd_prolong.cuh)
  static cudaError_t prolong(const void* cur, const void* prev, const int32_t* table,
                             int64_t nrows, double w, void* out, int64_t ncells, int maxit,
                             int ori, EosArg eos, int32_t* fallbacks, int grid, cudaStream_t s);
};

constexpr int kCflThreads = 256;

}  // namespace srhd
