// VL patch kernel of libsrhd (sm_103a): the predictor-corrector integrator
// that GAMER-SR offers beside MUSCL-Hancock (Section 3.1 of arXiv
// 2012.11130; van Leer 2006, Falle 1991), on ghosted patches of 14^3 cells
// (an 8^3 interior and three ghost cells per side: the corrector's PLM
// stencil reaches two cells beyond a face and the predictor one more).
//
// One persistent CTA per patch:
//   phase 1  con2pri of the 1952 tile cells the predictor reads (N)
//            -> W^n in shared memory [5][14^3]
//   phase 2  per direction: first-order Riemann fluxes at the 1408 faces of
//            the half-step cells (H) between piecewise-constant cell states,
//            then each of the 1280 H cells accumulates its flux difference
//   phase 3  U* = U^n - dt/(2 dh) sum_d dF_d and con2pri (warm start from
//            the cell's W^n) -> W* [5][1280] and its solver variable
//   phase 4  corrector: per face (3 x 576) PLM slopes of W* on both sides,
//            face states W* -/+ dW/2, their conserved form, Riemann flux
//   phase 5  conservative update, Eq. (Unphysical result) check and CFL
//            bound as in the MUSCL-Hancock kernel; a failed check redoes
//            phases 4-5 with a smaller limiter coefficient (Section 3.3). An
//            unphysical predicted state stops the patch (SRHD_PATCH_UNPHYSICAL,
//            NaN output): the predictor does not depend on the limiter.
// Shared memory: W^n (13720) + phase-2 fluxes (7040) + W* and its solver
// variable (7680) elements of S; the corrector fluxes (8640) reuse W^n.
#pragma once

#include "srhd_kernels.cuh"

namespace srhd {

constexpr int kVT = 14;                  // VL ghosted tile edge
constexpr int kVTC = kVT * kVT * kVT;    // 2744 tile cells
constexpr int kVN = 1952;                // cells whose W^n the predictor reads
constexpr int kVH = 1280;                // cells whose W* the corrector reads
constexpr int kVPF = 1408;               // predictor faces per direction

template <class S> struct VlSmem {
  static constexpr size_t wn = 5 * kVTC;
  static constexpr size_t fs = 5 * kVPF;
  static constexpr size_t wh = 6 * kVH;
  static constexpr size_t bytes = (wn + fs + wh) * sizeof(S);
  static_assert(3 * 5 * kNF <= wn, "corrector fluxes alias W^n");
};

__device__ __forceinline__ int vl_t14(int i, int j, int k) {
  return ((k + 3) * kVT + (j + 3)) * kVT + (i + 3);
}

__device__ __forceinline__ void vl_place(int axis, int along, int u, int v, int& i, int& j,
                                         int& k) {
  if (axis == 0) { i = along; j = u; k = v; }
  else if (axis == 1) { i = u; j = along; k = v; }
  else { i = u; j = v; k = along; }
}

// r-th cell of N: the interior, the six faces three layers deep, and the
// edge cells of depths (1,1), (1,2), (2,1) (interior coordinates -3..10).
__device__ __forceinline__ void vl_n_cell(int r, int& i, int& j, int& k) {
  if (r < 512) { i = r & 7; j = (r >> 3) & 7; k = r >> 6; return; }
  if (r < 1664) {
    const int q = r - 512, f = q / 192, rem = q - f * 192;
    const int depth = 1 + rem / 64, t = rem & 63;
    const int along = (f & 1) ? 7 + depth : -depth;
    vl_place(f >> 1, along, t & 7, t >> 3, i, j, k);
    return;
  }
  const int q = r - 1664, pair = q / 96, rem = q - pair * 96;
  const int e = rem / 24, rem2 = rem - e * 24, dc = rem2 >> 3, w = rem2 & 7;
  const int da = (dc == 2) ? 2 : 1, db = (dc == 1) ? 2 : 1;
  const int ca = (e & 1) ? 7 + da : -da, cb = (e & 2) ? 7 + db : -db;
  if (pair == 0) { i = ca; j = cb; k = w; }
  else if (pair == 1) { i = ca; j = w; k = cb; }
  else { i = w; j = ca; k = cb; }
}

// r-th cell of H: the interior and the six faces two layers deep.
__device__ __forceinline__ void vl_h_cell(int r, int& i, int& j, int& k) {
  if (r < 512) { i = r & 7; j = (r >> 3) & 7; k = r >> 6; return; }
  const int q = r - 512, f6 = q >> 7, rem = q & 127;
  const int depth = 1 + (rem >> 6), t = rem & 63;
  const int along = (f6 & 1) ? 7 + depth : -depth;
  vl_place(f6 >> 1, along, t & 7, t >> 3, i, j, k);
}

// Index in H of cell (i, j, k) (at most one coordinate outside 0..7, by at
// most two cells).
__device__ __forceinline__ int vl_h_index(int i, int j, int k) {
  int d, x, u, v;
  if (i < 0 || i > 7) { d = 0; x = i; u = j; v = k; }
  else if (j < 0 || j > 7) { d = 1; x = j; u = i; v = k; }
  else if (k < 0 || k > 7) { d = 2; x = k; u = i; v = j; }
  else return (k * 8 + j) * 8 + i;
  const int side = x > 7 ? 1 : 0;
  const int depth = side ? x - 7 : -x;
  return 512 + (2 * d + side) * 128 + (depth - 1) * 64 + v * 8 + u;
}

// r-th predictor face of a direction: between cells f - 1 and f along it,
// transverse coordinates (a, b) (a on the lower transverse axis).
__device__ __forceinline__ void vl_pface(int r, int& f, int& a, int& b) {
  if (r < 832) {
    const int ab = r / 13;
    f = r - ab * 13 - 2;
    a = ab & 7;
    b = ab >> 3;
    return;
  }
  const int q = r - 832, g = q / 288, rem = q - g * 288;
  const int t = rem / 9;
  f = rem - t * 9;
  const int io = t & 3, w = t >> 2;
  const int o = io < 2 ? io - 2 : io + 6;
  if (g == 0) { a = o; b = w; } else { a = w; b = o; }
}

__device__ __forceinline__ int vl_pface_index(int f, int a, int b) {
  const bool ain = a >= 0 && a <= 7, bin = b >= 0 && b <= 7;
  if (ain && bin) return (b * 8 + a) * 13 + (f + 2);
  const int g = ain ? 1 : 0;
  const int o = g == 0 ? a : b, w = g == 0 ? b : a;
  const int io = o < 0 ? o + 2 : o - 6;
  return 832 + g * 288 + (w * 4 + io) * 9 + f;
}

template <int d> __device__ __forceinline__ void vl_cell_of(int x, int a, int b, int& i, int& j,
                                                            int& k) {
  if (d == 0) { i = x; j = a; k = b; }
  else if (d == 1) { i = a; j = x; k = b; }
  else { i = a; j = b; k = x; }
}

// T, h, gamma, 1/gamma of a primitive state known as (rho, U, p).
template <class R, class E>
__device__ __forceinline__ void vl_derive(PrimX<R>& W, const E& eos) {
  W.T = qdiv(W.p, W.rho);
  R ht, hmT;
  eos_ht(eos, W.T, ht, hmT);
  W.ht = ht;
  W.h = R(1) + ht;
  const R g2 = R(1) + (W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2]);
  W.rg = rsqrt_r(g2);
  W.gamma = g2 * W.rg;
}

// vl_derive of two float states with the lane-wise arithmetic packed.
template <class E>
__device__ __forceinline__ void vl_derive_x2(PrimX<float>& A, PrimX<float>& B, const E& eos) {
  using namespace pk;
  const float2 T = make_float2(qdiv(A.p, A.rho), qdiv(B.p, B.rho));
  float2 ht;
  if constexpr (std::is_same<E, EosTM>::value) {
    const float2 q = mul(mul(s2(2.25f), T), T);
    const float2 t2 = make_float2(qdiv(q.x, 1.0f + sqrtf(q.x + 1.0f)),
                                  qdiv(q.y, 1.0f + sqrtf(q.y + 1.0f)));
    ht = fma(s2(2.5f), T, t2);
  } else {
    float hA, mA, hB, mB;
    eos_ht(eos, T.x, hA, mA);
    eos_ht(eos, T.y, hB, mB);
    ht = make_float2(hA, hB);
  }
  const float2 u0 = make_float2(A.u[0], B.u[0]), u1 = make_float2(A.u[1], B.u[1]);
  const float2 u2 = make_float2(A.u[2], B.u[2]);
  const float2 g2 = add(s2(1.0f), fma(u2, u2, fma(u1, u1, mul(u0, u0))));
  const float2 rg = rsq(g2);
  const float2 gm = mul(g2, rg);
  const float2 h = add(s2(1.0f), ht);
  A.T = T.x; B.T = T.y;
  A.ht = ht.x; B.ht = ht.y;
  A.h = h.x; B.h = h.y;
  A.rg = rg.x; B.rg = rg.y;
  A.gamma = gm.x; B.gamma = gm.y;
}

// prim2con of two float states (as the scalar prim2con, lane by lane, with
// the arithmetic packed): conserved variables and the derived T, h, gamma,
// 1/gamma of both; a state with rho <= 0 or p <= 0 gets NaN conserved
// variables and its flag false.
template <class E>
__device__ __forceinline__ void vl_prim2con_x2(PrimX<float>& A, PrimX<float>& B, float (&UA)[5],
                                               float (&UB)[5], bool& okA, bool& okB, int ori,
                                               const E& eos) {
  using namespace pk;
  okA = A.rho > 0.0f && A.p > 0.0f;
  okB = B.rho > 0.0f && B.p > 0.0f;
  const float2 rho = make_float2(A.rho, B.rho), p = make_float2(A.p, B.p);
  const float2 T = make_float2(qdiv(A.p, A.rho), qdiv(B.p, B.rho));
  float2 ht, hmT;
  if constexpr (std::is_same<E, EosTM>::value) {
    const float2 q = mul(mul(s2(2.25f), T), T);
    const float2 t2 = make_float2(qdiv(q.x, 1.0f + sqrtf(q.x + 1.0f)),
                                  qdiv(q.y, 1.0f + sqrtf(q.y + 1.0f)));
    ht = fma(s2(2.5f), T, t2);
    hmT = fma(s2(1.5f), T, t2);
  } else {
    float a0, a1, b0, b1;
    eos_ht(eos, T.x, a0, a1);
    eos_ht(eos, T.y, b0, b1);
    ht = make_float2(a0, b0);
    hmT = make_float2(a1, b1);
  }
  const float2 u0 = make_float2(A.u[0], B.u[0]), u1 = make_float2(A.u[1], B.u[1]);
  const float2 u2v = make_float2(A.u[2], B.u[2]);
  const float2 u2 = fma(u2v, u2v, fma(u1, u1, mul(u0, u0)));
  const float2 g2 = add(s2(1.0f), u2);
  const float2 rg = rsq(g2);
  const float2 gm = mul(g2, rg);
  const float2 D = mul(rho, gm);
  const float2 h = add(s2(1.0f), ht);
  const float2 Dh = mul(D, h);
  float2 U4;
  if (ori) {
    U4 = fma(Dh, gm, neg(p));
  } else {
    const float2 k1 = make_float2(qdiv(u2.x, gm.x + 1.0f), qdiv(u2.y, gm.y + 1.0f));
    U4 = mul(D, fma(fma(ht, u2, hmT), rg, k1));
  }
  const float2 U1 = mul(Dh, u0), U2 = mul(Dh, u1), U3 = mul(Dh, u2v);
  UA[0] = D.x; UA[1] = U1.x; UA[2] = U2.x; UA[3] = U3.x; UA[4] = U4.x;
  UB[0] = D.y; UB[1] = U1.y; UB[2] = U2.y; UB[3] = U3.y; UB[4] = U4.y;
  const float nan = __int_as_float(0x7fc00000);
  if (!okA) for (int v = 0; v < 5; ++v) UA[v] = nan;
  if (!okB) for (int v = 0; v < 5; ++v) UB[v] = nan;
  A.T = T.x; B.T = T.y;
  A.h = h.x; B.h = h.y;
  A.gamma = gm.x; B.gamma = gm.y;
  A.rg = rg.x; B.rg = rg.y;
}

// Start of the conversion solver from a nearby state of temperature T: the
// solver variable itself (tau = htilde - T for TM, htilde for polytropic).
template <class R> __device__ __forceinline__ R vl_guess(const EosTM& e, R T) {
  R ht, hmT;
  eos_ht(e, T, ht, hmT);
  return hmT;
}
template <class R> __device__ __forceinline__ R vl_guess(const EosPoly& e, R T) {
  R ht, hmT;
  eos_ht(e, T, ht, hmT);
  return ht;
}

template <class S> __device__ __forceinline__ void vl_load_prim(const S* Wn, int c,
                                                                PrimX<S>& W) {
  W.rho = Wn[c];
  W.u[0] = Wn[kVTC + c];
  W.u[1] = Wn[2 * kVTC + c];
  W.u[2] = Wn[3 * kVTC + c];
  W.p = Wn[4 * kVTC + c];
}

// Phase 2 for direction d: first-order fluxes, then the flux differences of
// the H cells accumulated into dU.
template <int d, class P, class E, int NT>
__device__ __forceinline__ void vl_predict_dir(const typename P::S* in, const typename P::S* Wn,
                                               typename P::S* Fs, typename P::S* dU,
                                               int solver, int ori, const E& eos) {
  using S = typename P::S;
  const int tid = threadIdx.x;
  for (int r = tid; r < kVPF; r += NT) {
    int f, a, b, i, j, k;
    vl_pface(r, f, a, b);
    vl_cell_of<d>(f - 1, a, b, i, j, k);
    const int cl = vl_t14(i, j, k);
    vl_cell_of<d>(f, a, b, i, j, k);
    const int cr = vl_t14(i, j, k);
    PrimX<S> WL, WR;
    vl_load_prim(Wn, cl, WL);
    vl_load_prim(Wn, cr, WR);
    if constexpr (sizeof(S) == 4) {
      vl_derive_x2(WL, WR, eos);
    } else {
      vl_derive(WL, eos);
      vl_derive(WR, eos);
    }
    S UL[5], UR[5], F[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      UL[v] = in[v * kVTC + cl];
      UR[v] = in[v * kVTC + cr];
    }
    riemann<d>(solver, WL, UL, WR, UR, F, ori, eos);
#pragma unroll
    for (int v = 0; v < 5; ++v) Fs[v * kVPF + r] = F[v];
  }
  __syncthreads();
  for (int r = tid; r < kVH; r += NT) {
    int i, j, k;
    vl_h_cell(r, i, j, k);
    const int x = d == 0 ? i : (d == 1 ? j : k);
    const int a = d == 0 ? j : i, b = d == 2 ? j : k;
    const int rl = vl_pface_index(x, a, b), rr = vl_pface_index(x + 1, a, b);
#pragma unroll
    for (int v = 0; v < 5; ++v) dU[v * kVH + r] += Fs[v * kVPF + rr] - Fs[v * kVPF + rl];
  }
  __syncthreads();
}

template <class P, int NT, int MINB, class E = EosTM>
__global__ void __launch_bounds__(NT, MINB) vl_patch_kernel(PatchArgs a) {
  using S = typename P::S;
  using R = S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* Wn = reinterpret_cast<S*>(smem_raw);
  S* Fs = Wn + VlSmem<S>::wn;
  S* Wh = Fs + VlSmem<S>::fs;       // [5][kVH] W* (dU before phase 3), then [kVH] solver variable
  S* Fc = Wn;                       // corrector fluxes [3][5][576], after phase 3
  __shared__ double s_red[NT / 32];
  __shared__ int s_bad[NT / 32];
  const int tid = threadIdx.x;
  const int maxit = a.maxit;
  const int ori = a.ori;
  const E eos = make_eos<E>(a);
  // limiter constants and per-patch step factors in the arithmetic type,
  // converted by one thread (as in patch_kernel)
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

  for (int w = blockIdx.x; w < a.npatch; w += gridDim.x) {
    const int p = a.worklist ? a.worklist[w] : w;
    const S* in = static_cast<const S*>(a.in) + (size_t)p * 5 * kVTC;
    int code = 0;
    __syncthreads();  // the previous patch is done with shared memory
    // ---- phase 1: W^n on N --------------------------------------------------
    for (int r = tid; r < kVN / 2; r += NT) {
      int i, j, k;
      vl_n_cell(r, i, j, k);
      const int ca = vl_t14(i, j, k);
      vl_n_cell(r + kVN / 2, i, j, k);
      const int cb = vl_t14(i, j, k);
      S Ua[5], Ub[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Ua[v] = in[v * kVTC + ca];
        Ub[v] = in[v * kVTC + cb];
      }
      PrimX<R> Wa, Wb;
      int sa, sb;
      con2pri_x2<P>(Ua, Ub, Wa, Wb, maxit, sa, sb, S(0), S(0), ori, eos);
      if (sa == 1 || sb == 1) code |= CODE_BAD_INPUT;
      if (sa == 2 || sb == 2) code |= CODE_NOCONV;
      Wn[ca] = Wa.rho; Wn[kVTC + ca] = Wa.u[0]; Wn[2 * kVTC + ca] = Wa.u[1];
      Wn[3 * kVTC + ca] = Wa.u[2]; Wn[4 * kVTC + ca] = Wa.p;
      Wn[cb] = Wb.rho; Wn[kVTC + cb] = Wb.u[0]; Wn[2 * kVTC + cb] = Wb.u[1];
      Wn[3 * kVTC + cb] = Wb.u[2]; Wn[4 * kVTC + cb] = Wb.p;
    }
    for (int q = tid; q < 5 * kVH; q += NT) Wh[q] = S(0);
    if (tid == NT - 1) {
      const double dt = a.dt_dh[2 * p], dh = a.dt_dh[2 * p + 1];
      const R coef = R(dt) / R(dh);
      s_pc[0] = coef;
      s_pc[1] = R(0.5) * coef;
      s_pc[2] = R(a.cfl * dh);
      if (a.partial_dt && a.cfl_mode == 1) s_dtl = fmin(s_dtl, a.cfl * dh);
    }
    const int bad_input = __syncthreads_or(code & CODE_BAD_INPUT);
    int retries = 0;
    int final_code = 0;
    R att_smax = R(0);
    int att_bad = 0;
    bool nan_out = bad_input != 0;
    if (!bad_input) {
      // ---- phase 2: first-order fluxes and their differences ---------------
      vl_predict_dir<0, P, E, NT>(in, Wn, Fs, Wh, a.riemann, ori, eos);
      vl_predict_dir<1, P, E, NT>(in, Wn, Fs, Wh, a.riemann, ori, eos);
      vl_predict_dir<2, P, E, NT>(in, Wn, Fs, Wh, a.riemann, ori, eos);
      // ---- phase 3: half-step state and its primitives ---------------------
      const R half = s_pc[1];
      int pbad = 0;
      for (int r = tid; r < kVH / 2; r += NT) {
        int i, j, k;
        vl_h_cell(r, i, j, k);
        const int ca = vl_t14(i, j, k);
        vl_h_cell(r + kVH / 2, i, j, k);
        const int cb = vl_t14(i, j, k);
        S Ua[5], Ub[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          Ua[v] = S(R(in[v * kVTC + ca]) - half * R(Wh[v * kVH + r]));
          Ub[v] = S(R(in[v * kVTC + cb]) - half * R(Wh[v * kVH + r + kVH / 2]));
        }
        const S ga = vl_guess(eos, R(qdiv(Wn[4 * kVTC + ca], Wn[ca])));
        const S gb = vl_guess(eos, R(qdiv(Wn[4 * kVTC + cb], Wn[cb])));
        PrimX<R> Wa, Wb;
        int sa, sb;
        con2pri_x2<P, E, true>(Ua, Ub, Wa, Wb, maxit, sa, sb, ga, gb, ori, eos);
        if (sa == 1 || sb == 1) pbad = 1;
        if (sa == 2 || sb == 2) code |= CODE_NOCONV;
        const int rb = r + kVH / 2;
        Wh[r] = Wa.rho; Wh[kVH + r] = Wa.u[0]; Wh[2 * kVH + r] = Wa.u[1];
        Wh[3 * kVH + r] = Wa.u[2]; Wh[4 * kVH + r] = Wa.p; Wh[5 * kVH + r] = Wa.tau;
        Wh[rb] = Wb.rho; Wh[kVH + rb] = Wb.u[0]; Wh[2 * kVH + rb] = Wb.u[1];
        Wh[3 * kVH + rb] = Wb.u[2]; Wh[4 * kVH + rb] = Wb.p; Wh[5 * kVH + rb] = Wb.tau;
      }
      pbad = __syncthreads_or(pbad);
      if (pbad) {
        final_code |= CODE_UNPHYSICAL;
        nan_out = true;
        att_bad = 1;
      } else {
        R theta = s_kc[0];
        for (;;) {
          // ---- phase 4: corrector fluxes ------------------------------------
          int fail = 0;
          for (int f = tid; f < 3 * kNF; f += NT) {
            const int d = f / kNF, fi = f - d * kNF;
            int fd, ta, tb;   // face coordinate along d, transverse coordinates
            if (d == 0) { fd = fi % 9; ta = (fi / 9) & 7; tb = fi / 72; }
            else if (d == 1) { ta = fi & 7; fd = (fi >> 3) % 9; tb = (fi >> 3) / 9; }
            else { ta = fi & 7; tb = (fi >> 3) & 7; fd = fi >> 6; }
            int hq[4];
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
              int i, j, k;
              const int x = fd - 2 + s4;
              if (d == 0) { i = x; j = ta; k = tb; }
              else if (d == 1) { i = ta; j = x; k = tb; }
              else { i = ta; j = tb; k = x; }
              hq[s4] = vl_h_index(i, j, k);
            }
            PrimX<R> WL, WR;
            R wl[5], wr[5];
            R UL[5], UR[5], F[5];
            if constexpr (sizeof(R) == 4) {
              // float: the left (lane x) and right (lane y) face states in
              // packed form
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                const float w0 = Wh[v * kVH + hq[0]], w1 = Wh[v * kVH + hq[1]];
                const float w2 = Wh[v * kVH + hq[2]], w3 = Wh[v * kVH + hq[3]];
                const float2 sl = limited_slope_x2(make_float2(w1 - w0, w2 - w1),
                                                   make_float2(w2 - w1, w3 - w2), theta);
                const float2 lr = pk::fma(sl, make_float2(0.5f, -0.5f), make_float2(w1, w2));
                wl[v] = lr.x;
                wr[v] = lr.y;
              }
              WL.rho = wl[0]; WL.u[0] = wl[1]; WL.u[1] = wl[2]; WL.u[2] = wl[3]; WL.p = wl[4];
              WR.rho = wr[0]; WR.u[0] = wr[1]; WR.u[1] = wr[2]; WR.u[2] = wr[3]; WR.p = wr[4];
              bool okL, okR;
              vl_prim2con_x2(WL, WR, UL, UR, okL, okR, ori, eos);
              if (!okL || !okR) fail = 1;
            } else {
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                const R w0 = R(Wh[v * kVH + hq[0]]), w1 = R(Wh[v * kVH + hq[1]]);
                const R w2 = R(Wh[v * kVH + hq[2]]), w3 = R(Wh[v * kVH + hq[3]]);
                wl[v] = w1 + R(0.5) * limited_slope(w1 - w0, w2 - w1, theta);
                wr[v] = w2 - R(0.5) * limited_slope(w2 - w1, w3 - w2, theta);
              }
              WL.rho = wl[0]; WL.u[0] = wl[1]; WL.u[1] = wl[2]; WL.u[2] = wl[3]; WL.p = wl[4];
              WR.rho = wr[0]; WR.u[0] = wr[1]; WR.u[1] = wr[2]; WR.u[2] = wr[3]; WR.p = wr[4];
              if (!prim2con(WL, UL, ori, eos)) fail = 1;
              if (!prim2con(WR, UR, ori, eos)) fail = 1;
            }
            if (d == 0) riemann<0>(a.riemann, WL, UL, WR, UR, F, ori, eos);
            else if (d == 1) riemann<1>(a.riemann, WL, UL, WR, UR, F, ori, eos);
            else riemann<2>(a.riemann, WL, UL, WR, UR, F, ori, eos);
#pragma unroll
            for (int v = 0; v < 5; ++v) Fc[(d * 5 + v) * kNF + fi] = S(F[v]);
          }
          fail = __syncthreads_or(fail);
          if (a.flux_only) {
            if (fail) final_code |= CODE_UNPHYSICAL;
            break;
          }
          const bool last = (theta == R(0));
          // ---- phase 5: conservative update ---------------------------------
          att_smax = R(0);
          att_bad = 0;
          if (!fail || last) {
            S* out = static_cast<S*>(a.out) + (size_t)p * 5 * kNC;
            const bool signal = a.partial_dt && a.cfl_mode != 1;
            int fail5 = 0;
            if constexpr (sizeof(R) == 4) {
              // float: the work item c0 < 256 updates cells c0 and c0 + 256
              // in packed arithmetic and converts both in lockstep for the
              // CFL bound (warm starts from their half-step states)
              constexpr int kItems = kNC / 2;
              for (int c0 = tid; c0 < kItems; c0 += NT) {
                const float2 mcoef = pk::s2(-float(s_pc[0]));
                int tcq[2], fq[2][6];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                  const int c = c0 + q * kItems;
                  const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
                  tcq[q] = vl_t14(i, j, k);
                  fq[q][0] = face_index<0>(i, j, k, i);
                  fq[q][1] = face_index<0>(i, j, k, i + 1);
                  fq[q][2] = face_index<1>(i, j, k, j);
                  fq[q][3] = face_index<1>(i, j, k, j + 1);
                  fq[q][4] = face_index<2>(i, j, k, k);
                  fq[q][5] = face_index<2>(i, j, k, k + 1);
                }
                S Un[2][5];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                  auto ld = [&](int dd, int e) {
                    const S* f = Fc + (dd * 5 + v) * kNF;
                    return make_float2(f[fq[0][e]], f[fq[1][e]]);
                  };
                  const float2 div = pk::add(pk::add(pk::sub(ld(0, 1), ld(0, 0)),
                                                     pk::sub(ld(1, 3), ld(1, 2))),
                                             pk::sub(ld(2, 5), ld(2, 4)));
                  const float2 old = make_float2(in[v * kVTC + tcq[0]], in[v * kVTC + tcq[1]]);
                  const float2 un = pk::fma(mcoef, div, old);
                  Un[0][v] = un.x;
                  Un[1][v] = un.y;
                  out[v * kNC + c0] = un.x;
                  out[v * kNC + c0 + kItems] = un.y;
                }
                if (signal) {
                  PrimX<R> W0, W1;
                  int s0, s1;
                  con2pri_x2<P, E, true>(Un[0], Un[1], W0, W1, maxit, s0, s1,
                                         Wh[5 * kVH + c0], Wh[5 * kVH + c0 + kItems], ori, eos);
                  if (s0 != 1) att_smax = fmax(att_smax, smax_of(W0, a.ndim, eos));
                  if (s1 != 1) att_smax = fmax(att_smax, smax_of(W1, a.ndim, eos));
                  if (s0 == 1 || s1 == 1) {
                    att_bad = 1;
                    fail5 = 1;
                  }
                } else {
#pragma unroll
                  for (int q = 0; q < 2; ++q) {
                    typename P::AT Ac, m2c;
                    if (!A_and_m2<P>(Un[q][0], Un[q][1], Un[q][2], Un[q][3], Un[q][4], Ac, m2c,
                                     ori))
                      fail5 = 1;
                  }
                }
              }
            } else {
            for (int c = tid; c < kNC; c += NT) {
              const R coef = s_pc[0];
              const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
              const int tc = vl_t14(i, j, k);
              const int fx0 = face_index<0>(i, j, k, i), fx1 = face_index<0>(i, j, k, i + 1);
              const int fy0 = face_index<1>(i, j, k, j), fy1 = face_index<1>(i, j, k, j + 1);
              const int fz0 = face_index<2>(i, j, k, k), fz1 = face_index<2>(i, j, k, k + 1);
              S Un[5];
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                R div = R(0);
                div = div + (R(Fc[(0 * 5 + v) * kNF + fx1]) - R(Fc[(0 * 5 + v) * kNF + fx0]));
                div = div + (R(Fc[(1 * 5 + v) * kNF + fy1]) - R(Fc[(1 * 5 + v) * kNF + fy0]));
                div = div + (R(Fc[(2 * 5 + v) * kNF + fz1]) - R(Fc[(2 * 5 + v) * kNF + fz0]));
                Un[v] = S(R(in[v * kVTC + tc]) - coef * div);
                out[v * kNC + c] = Un[v];
              }
              if (signal) {
                PrimX<R> W;
                const int st = con2pri<P>(Un[0], Un[1], Un[2], Un[3], Un[4], W, maxit,
                                          Wh[5 * kVH + c], ori, eos);
                if (st != 1) {
                  att_smax = fmax(att_smax, smax_of(W, a.ndim, eos));
                } else {
                  att_bad = 1;
                  fail5 = 1;
                }
              } else {
                typename P::AT Ac, m2c;
                if (!A_and_m2<P>(Un[0], Un[1], Un[2], Un[3], Un[4], Ac, m2c, ori)) fail5 = 1;
              }
            }
            }
            fail = __syncthreads_or(fail5) | fail;
          }
          if (!fail) break;
          if (last) { final_code |= CODE_UNPHYSICAL; break; }
          ++retries;
          theta = theta * s_kc[1];
          if (theta < s_kc[2]) theta = R(0);
        }
      }
      if (att_smax > R(0)) dtr = fmin(dtr, s_pc[2] / att_smax);
      cfl_bad |= att_bad;
    } else {
      final_code |= CODE_BAD_INPUT;
      cfl_bad = 1;
    }
    if (nan_out && !a.flux_only) {
      S* out = static_cast<S*>(a.out) + (size_t)p * 5 * kNC;
      for (int c = tid; c < 5 * kNC; c += NT)
        out[c] = S(__longlong_as_double(0x7ff8000000000000ULL));
    }
    // ---- outputs (face fluxes are valid when the corrector ran) -------------
    const bool corrected = !nan_out;
    if (a.flux_only && corrected) {
      S* ff = static_cast<S*>(a.face_flux) + (size_t)p * 3 * 5 * kNF;
      for (int q = tid; q < 3 * 5 * kNF; q += NT) ff[q] = Fc[q];
    }
    if (a.pflux && !a.flux_only && corrected) {
      S* pf = static_cast<S*>(a.pflux) + (size_t)p * 6 * 5 * 64;
      for (int q = tid; q < 6 * 5 * 64; q += NT) {
        const int side = q / 320, rem = q - side * 320, v = rem >> 6, t = rem & 63;
        const int d = side >> 1, fd = (side & 1) ? 8 : 0;
        const int a0 = t & 7, b0 = t >> 3;
        const int fi = (d == 0) ? face_index<0>(0, a0, b0, fd)
                                : (d == 1) ? face_index<1>(a0, 0, b0, fd)
                                           : face_index<2>(a0, b0, 0, fd);
        pf[q] = Fc[(d * 5 + v) * kNF + fi];
      }
    }
    code = __syncthreads_or(code & CODE_NOCONV);
    if (tid == 0 && a.status) {
      final_code |= code ? CODE_NOCONV : 0;
      a.status[p] = (final_code << 8) | (retries < 255 ? retries : 255);
    }
  }

  // ---- CFL partial minimum of this CTA ---------------------------------------
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

}  // namespace srhd
