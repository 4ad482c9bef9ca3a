// Device physics of the SRHD per-patch update (arXiv 2012.11130, Sections
// 2 and 3): Taub-Mathews EoS, conserved <-> primitive conversion, physical
// fluxes, relativistic HLLC / HLLE, PLM limiter and the signal-speed CFL
// bound. Everything here is written for the GPU from the paper's equations;
// it shares no code with the CPU oracle.
//
// Arithmetic type R is float or double; storage type S (float or double)
// is the element type of the arrays. In the mixed path (S = R = float) the
// left-hand side A of Eq. (transcendental equation) is formed in double
// from the stored values (it is the only cancellation-critical operation,
// Eq. ImprovedRelativeError) and the Newton iteration then runs in float.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace srhd {

// eps_machine of Eq. (Unphysical result) (Section 3.3: 2e-16 for double).
// A is formed in double in both precisions, so both use the double value.
constexpr double kEpsUnphysical = 2e-16;

template <class R> struct NewtonCfg;
template <> struct NewtonCfg<double> {
  static constexpr double tol = 8.8817841970012523e-16;  // 2^-50
  static constexpr double floor = 1e-12;
  static constexpr int maxit = 50;
};
template <> struct NewtonCfg<float> {
  static constexpr float tol = 4.76837158e-07f;  // 2^-21
  static constexpr float floor = 1e-4f;
  static constexpr int maxit = 30;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// Primitive state with the derived quantities reused downstream.
template <class R> struct PrimX {
  R rho, u[3], p;   // W = (rho, U^x, U^y, U^z, p)
  R T, h, gamma;    // T = p/rho, h = 1 + htilde, gamma = sqrt(1 + U.U)
};

// Eq. (T_to_HTilde): htilde(T) without subtraction.
template <class R> __device__ __forceinline__ R htilde_of_T(R T) {
  R a = R(2.25) * T * T;
  return R(2.5) * T + a / (R(1) + sqrt(a + R(1)));
}

// Eq. (T of h) and its derivative Eq. (dT_dh), sharing one reciprocal square
// root and one division: with x = 9 ht^2 + 18 ht + 25, s = sqrt(x),
// den = 5 ht + 5 + s: T = (2 ht^2 + 4 ht)/den and
// dT = [(4 ht + 4) - T ((9 ht + 9)/s + 5)] / den.
template <class R> __device__ __forceinline__ void T_dT_of_htilde(R ht, R& T, R& dT) {
  R x = (R(9) * ht + R(18)) * ht + R(25);
  R rs = rsqrt_r(x);
  R den = R(5) * ht + R(5) + x * rs;
  R rden = R(1) / den;
  T = (R(2) * ht + R(4)) * ht * rden;
  dT = ((R(4) * ht + R(4)) - T * ((R(9) * ht + R(9)) * rs + R(5))) * rden;
}

template <class R> __device__ __forceinline__ R T_of_htilde(R ht) {
  R x = (R(9) * ht + R(18)) * ht + R(25);
  return (R(2) * ht + R(4)) * ht / (R(5) * ht + R(5) + sqrt(x));
}

// Eq. (sound_speed): c_s^2 = T (5h - 8T) / (3h (h - T)).
template <class R> __device__ __forceinline__ R cs2_of(R T, R h) {
  return T * (R(5) * h - R(8) * T) / (R(3) * h * (h - T));
}

// Eq. (transcendental equation) f(htilde) and Appendix A df/dhtilde, in a
// form that cannot overflow float for m^2 up to ~1e30:
// f  = ht (ht + 2) - 2 T h + T^2 hh/q,                 q = hh + m2
// f' = 2h - 2T - 2h T' + 2T/q [T' hh (hh/q) + h (h T' + T) (m2/q)].
template <class R>
__device__ __forceinline__ void f_df(R ht, R T, R dT, R m2, R& f, R& df) {
  R h = ht + R(1);
  R hh = h * h;
  R rq = R(1) / (hh + m2);
  R a1 = hh * rq, a2 = m2 * rq;
  f = ht * (ht + R(2)) - R(2) * T * h + T * T * a1;
  df = R(2) * h - R(2) * T - R(2) * h * dT +
       R(2) * T * rq * (dT * hh * a1 + h * (h * dT + T) * a2);
}

// Appendix A initial guess: hot (4/3) sqrt(A) above the Eq. (ColdHot)
// threshold, else the positive root of the quadratic of Eq. (cold limit of
// transcendental eq) in cancellation-free form.
template <class R> __device__ __forceinline__ R newton_guess(R A, R m2) {
  R P = R(1) + m2;
  R tb = R(1800) * P / (R(437) * m2 + R(117));
  if (A > tb * tb) return R(4.0 / 3.0) * sqrt(A);
  R a = (R(43) * m2 + R(63)) / (R(125) * P);
  return R(2) * A / (R(1.2) + sqrt(R(1.44) + R(4) * a * A));
}

// A = (Et/D)^2 + 2 Et/D - (|M|/D)^2 in double (Eq. transcendental equation,
// left-hand side; Eq. Unphysical result) and m^2 = (|M|/D)^2.
template <class S>
__device__ __forceinline__ double A_of_cons(S D, S Mx, S My, S Mz, S Et, double& m2) {
  double rD = 1.0 / double(D);
  double eD = double(Et) * rD;
  double M2 = double(Mx) * double(Mx) + double(My) * double(My) + double(Mz) * double(Mz);
  m2 = M2 * rD * rD;
  return eD * (eD + 2.0) - m2;
}

// Conserved -> primitive (Section 2.3). Returns 0 ok, 1 unphysical, 2 no
// convergence. Newton-Raphson on f(htilde) = A (monotone f), then
// Eq. (four-velocity), Eq. (new expression of Lorentz factor), Eq. (density),
// Eq. (T of h), Eq. (p=rhoT). A step that would make htilde non-positive
// halves htilde instead. Stops when |dh| <= tol htilde, or when the step no
// longer contracts at the rounding floor, or after maxit steps (status 2).
template <class R, class S>
__device__ __forceinline__ int con2pri(S D, S Mx, S My, S Mz, S Et, PrimX<R>& W, int maxit) {
  double m2d;
  double Ad = A_of_cons(D, Mx, My, Mz, Et, m2d);
  if (!(double(D) > 0.0) || !(Ad > kEpsUnphysical)) {
    R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
    W.rho = W.u[0] = W.u[1] = W.u[2] = W.p = W.T = W.h = W.gamma = nan;
    return 1;
  }
  const R A = R(Ad), m2 = R(m2d);
  R ht = newton_guess(A, m2);
  int status = 2;
  R prev = R(3.0e38);
  for (int k = 1; k <= maxit; ++k) {
    R T, dT, f, df;
    T_dT_of_htilde(ht, T, dT);
    f_df(ht, T, dT, m2, f, df);
    R dh = (f - A) / df;
    R hn = ht - dh;
    if (!(hn > R(0))) hn = R(0.5) * ht;
    R adh = fabs(dh);
    ht = hn;
    if (adh <= NewtonCfg<R>::tol * ht) { status = 0; break; }
    if (k >= 3 && adh >= prev && adh <= NewtonCfg<R>::floor * ht) { status = 0; break; }
    prev = adh;
  }
  R h = R(1) + ht;
  R rDh = R(1) / (R(D) * h);
  W.u[0] = R(Mx) * rDh;
  W.u[1] = R(My) * rDh;
  W.u[2] = R(Mz) * rDh;
  R g2 = R(1) + (W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2]);
  R rg = rsqrt_r(g2);
  W.gamma = g2 * rg;
  W.rho = R(D) * rg;
  W.T = T_of_htilde(ht);
  W.h = h;
  W.p = W.rho * W.T;
  return status;
}

// Primitive -> conserved (Eq. density, momentum, T_to_HTilde, E_D).
// Fills T, h, gamma of W. Returns false if rho <= 0 or p <= 0.
template <class R> __device__ __forceinline__ bool prim2con(PrimX<R>& W, R U[5]) {
  if (!(W.rho > R(0)) || !(W.p > R(0))) {
    R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
    for (int v = 0; v < 5; ++v) U[v] = nan;
    return false;
  }
  R T = W.p / W.rho;
  R ht = htilde_of_T(T);
  R u2 = W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2];
  R gamma = sqrt(R(1) + u2);
  R D = W.rho * gamma;
  R h = R(1) + ht;
  R Dh = D * h;
  U[0] = D;
  U[1] = Dh * W.u[0];
  U[2] = Dh * W.u[1];
  U[3] = Dh * W.u[2];
  R hh = h * h;
  R m2 = hh * u2;
  R f = ht * (ht + R(2)) - R(2) * T * h + T * T * (hh / (hh + m2));
  R s = m2 + f;
  U[4] = D * (s / (R(1) + sqrt(R(1) + s)));
  W.T = T;
  W.h = h;
  W.gamma = gamma;
  return true;
}

// Physical flux along d (Eqs. D evolution, M evolution, ETilde evolution).
template <int d, class R>
__device__ __forceinline__ void phys_flux(const PrimX<R>& W, const R U[5], R F[5]) {
  R v = W.u[d] / W.gamma;
  F[0] = U[0] * v;
  F[1] = U[1] * v;
  F[2] = U[2] * v;
  F[3] = U[3] * v;
  F[1 + d] += W.p;
  F[4] = (U[4] + W.p) * v;
}

// Outer characteristic speeds along d with the TM sound speed, in the
// four-velocity form [gamma U_d (1-cs2) -/+ sqrt(cs2 (1 + U_perp^2 (1-cs2)))]
// / [1 + U^2 (1-cs2)].
template <int d, class R>
__device__ __forceinline__ void char_speeds(const PrimX<R>& W, R& lm, R& lp) {
  R cs2 = cs2_of(W.T, W.h);
  R omc = R(1) - cs2;
  R ud = W.u[d];
  // transverse part summed directly (no u2 - ud^2 cancellation)
  R ua = W.u[d == 0 ? 1 : 0], ub = W.u[d == 2 ? 1 : 2];
  R up2 = ua * ua + ub * ub;
  R u2 = up2 + ud * ud;
  R rden = R(1) / (R(1) + u2 * omc);
  R a = W.gamma * ud * omc;
  R b = sqrt(cs2 * (R(1) + up2 * omc));
  lm = (a - b) * rden;
  lp = (a + b) * rden;
}

// Relativistic HLLC of Mignone & Bodo (2005) with E = Etilde + D inside the
// solver (Section 3.1), HLLE when requested or when the contact state is not
// admissible (discriminant < 0, contact speed outside the outer speeds, or
// non-positive contact pressure). Returns 1 on fallback.
template <int d, class R>
__device__ __forceinline__ int riemann(int solver, const PrimX<R>& WL, const R UL[5],
                                       const PrimX<R>& WR, const R UR[5], R F[5]) {
  R FL[5], FR[5];
  phys_flux<d>(WL, UL, FL);
  phys_flux<d>(WR, UR, FR);
  R lmL, lpL, lmR, lpR;
  char_speeds<d>(WL, lmL, lpL);
  char_speeds<d>(WR, lmR, lpR);
  R sL = fmin(lmL, lmR);
  R sR = fmax(lpL, lpR);
  if (sL >= R(0)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = FL[v];
    return 0;
  }
  if (sR <= R(0)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = FR[v];
    return 0;
  }
  R rds = R(1) / (sR - sL);
  R Uh[5], Fh[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Uh[v] = (sR * UR[v] - sL * UL[v] - FR[v] + FL[v]) * rds;
    Fh[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) * rds;
  }
  if (solver == 0) {
    R E = Uh[4] + Uh[0];
    R FE = Fh[4] + Fh[0];
    R m = Uh[1 + d];
    R Fm = Fh[1 + d];
    R B = E + Fm;
    R disc = B * B - R(4) * FE * m;
    if (disc >= R(0) && B > R(0)) {
      R lam = R(2) * m / (B + sqrt(disc));
      R ps = Fm - lam * FE;
      if (lam > sL && lam < sR && ps > R(0)) {
        const bool left = lam >= R(0);
        const PrimX<R>& Wk = left ? WL : WR;
        const R* Uk = left ? UL : UR;
        const R* Fk = left ? FL : FR;
        R sk = left ? sL : sR;
        R v = Wk.u[d] / Wk.gamma;
        R a = sk - v;
        R rb = R(1) / (sk - lam);
        R Us[5];
        Us[0] = Uk[0] * a * rb;
#pragma unroll
        for (int k = 0; k < 3; ++k) Us[1 + k] = Uk[1 + k] * a * rb;
        Us[1 + d] = (Uk[1 + d] * a + ps - Wk.p) * rb;
        Us[4] = (Uk[4] * a + ps * lam - Wk.p * v) * rb;
#pragma unroll
        for (int v5 = 0; v5 < 5; ++v5) F[v5] = Fk[v5] + sk * (Us[v5] - Uk[v5]);
        return 0;
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = Fh[v];
    return 1;
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = Fh[v];
  return 0;
}

// Hybrid van Leer / generalised minmod slope: 0 at extrema, else the smaller
// in magnitude of 2 dl dr/(dl+dr) and minmod(theta dl, theta dr, (dl+dr)/2).
template <class R> __device__ __forceinline__ R limited_slope(R dl, R dr, R theta) {
  if (!(dl * dr > R(0))) return R(0);
  R vl = R(2) * dl * dr / (dl + dr);
  R gm = fmin(fmin(theta * fabs(dl), theta * fabs(dr)), R(0.5) * fabs(dl + dr));
  R mag = fmin(fabs(vl), gm);
  return dl > R(0) ? mag : -mag;
}

// Signal speed bound S_max of one cell (Section 3.2, Eqs. time_step_U_max
// and SMax; |U_x|+|U_y|+|U_z| and ndim gamma U_s).
template <class R> __device__ __forceinline__ R smax_of(const PrimX<R>& W, int ndim) {
  R cs2 = cs2_of(W.T, W.h);
  R omc = R(1) - cs2;
  R us = sqrt(cs2 / omc);           // U_s = c_s / sqrt(1 - c_s^2)
  R gs = rsqrt_r(omc);              // gamma_s = 1 / sqrt(1 - c_s^2)
  R su = fabs(W.u[0]) + fabs(W.u[1]) + fabs(W.u[2]);
  R umax = gs * su + R(ndim) * W.gamma * us;
  return umax * rsqrt_r(R(1) + umax * umax);
}

}  // namespace srhd
