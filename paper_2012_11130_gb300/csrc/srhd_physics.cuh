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
#include <type_traits>
#include <cuda_runtime.h>

namespace srhd {

// eps_machine of Eq. (Unphysical result) (Section 3.3: 2e-16 for double).
// A is formed in double in both precisions, so both use the double value.
constexpr double kEpsUnphysical = 2e-16;

// Newton stopping rule (for the conic-parameter iteration of the
// conversions below). Near the root the iteration converges quadratically,
// e_{k+1} <= C e_k^2 in relative terms, with C <= 0.56 over the whole range
// of states (measured in double: rho 1e-6..1e2, T 1e-10..1e6, gamma 1..1e6;
// largest 0.557). Once a step satisfies |dtau| <= tol tau the error left
// after applying it is at most C tol^2: 3e-17 for tol = 2^-27 in double and
// 8e-9 for tol = 2^-13 in float, below the rounding of either precision, so
// the iteration stops there instead of taking one more step. (htilde and T
// inherit the relative error of tau up to a factor below 2.) An iteration
// that stalls at the rounding floor (steps of a few ulps of tau) meets the
// rule too, since tol lies far above the rounding of either precision.
template <class R> struct NewtonCfg;
template <> struct NewtonCfg<double> {
  static constexpr double tol = 7.450580596923828e-09;  // 2^-27
  static constexpr int maxit = 50;
};
template <> struct NewtonCfg<float> {
  static constexpr float tol = 1.220703125e-04f;  // 2^-13
  static constexpr int maxit = 30;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// Reciprocal in double by Newton-Raphson refinement of the hardware
// approximation (rcp.approx.ftz.f64): each step r <- r + r (1 - x r) squares
// the relative error, and the approximation is good to about 2^-20 or better, so two
// steps leave only the rounding of the last fused multiply-add (the result
// is within about one ulp of 1/x; tests/test_gpu_fast_rcp.py bounds it
// against the IEEE division). The IEEE division is several times longer on
// the FP64 pipe, which bounds the FP64 kernels. Zero, subnormal, huge
// (|x| >= 2^1021, whose reciprocal is subnormal) and non-finite x take the
// IEEE division, so those keep its results exactly.
__device__ __forceinline__ double drcp(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7ff;
  if (ex == 0 || ex >= 0x7fd) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Quotient and reciprocal in the arithmetic type. In float they are the
// hardware approximate division (at most 2 ulp, like the '/' operator under
// -prec-div=false, but without its range scaling: valid for divisors of
// magnitude below 2^126, which every denominator they are used on stays far
// below); in double the product with drcp (within about two ulp).
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a * drcp(b); }
__device__ __forceinline__ float qrcp(float b) { return __fdividef(1.0f, b); }
__device__ __forceinline__ double qrcp(double b) { return drcp(b); }
// The '/' operator in float (the full-range approximate division under
// -prec-div=false), qdiv in double.
__device__ __forceinline__ float fdiv(float a, float b) { return a / b; }
__device__ __forceinline__ double fdiv(double a, double b) { return qdiv(a, b); }

// Primitive state with the derived quantities reused downstream.
template <class R> struct PrimX {
  R rho, u[3], p;   // W = (rho, U^x, U^y, U^z, p)
  R T, h, gamma;    // T = p/rho, h = 1 + htilde, gamma = sqrt(1 + U.U)
  R rg;             // 1 / gamma (three-velocity v = U rg)
  R ht;             // htilde (set by the conversions from conserved variables)
  R tau;            // solver variable: conic parameter h - T - 1 (TM) or htilde
                    // (polytropic), set by the same conversions
  R rt;             // tau over its cold start (x_start), set by a cold
                    // conversion that is asked for it (RATIO)
};

// Equation of state, selected at compile time by a tag:
//   EosTM    the Taub-Mathews EoS (Eq. TM EOS), the paper's;
//   EosPoly  the polytropic EoS h = 1 + Gamma/(Gamma-1) T (Section 2.2; kept
//            by the paper for pure non-relativistic or ultra-relativistic
//            gas), with Gamma (1 < Gamma <= 5/3) given at run time.
struct EosTM {};
struct EosPoly {
  double gam;
};

// htilde(T) and htilde - T. TM: Eq. (T_to_HTilde) without subtraction,
// htilde - T = 1.5 T + 2.25 T^2/(1 + sqrt(1 + 2.25 T^2)). Polytropic:
// Gamma/(Gamma-1) T and T/(Gamma-1).
template <class R>
__device__ __forceinline__ void eos_ht(const EosTM&, R T, R& ht, R& hmT) {
  const R a = R(2.25) * T * T;
  const R t2 = qdiv(a, R(1) + sqrt(a + R(1)));
  ht = R(2.5) * T + t2;
  hmT = R(1.5) * T + t2;
}
template <class R>
__device__ __forceinline__ void eos_ht(const EosPoly& e, R T, R& ht, R& hmT) {
  hmT = T * R(1.0 / (e.gam - 1.0));
  ht = T + hmT;
}

// The conversions' solver variable of a state of temperature T in closed
// form: the conic parameter tau = h - T - 1 = htilde - T (TM) or htilde
// (polytropic). The root a conversion converges to satisfies it to the
// rounding of that root, so it is a warm start for the solve of a nearby
// state.
template <class R> __device__ __forceinline__ R solver_var_of_T(const EosTM& e, R T) {
  R ht, hmT;
  eos_ht(e, T, ht, hmT);
  return hmT;
}
template <class R> __device__ __forceinline__ R solver_var_of_T(const EosPoly& e, R T) {
  R ht, hmT;
  eos_ht(e, T, ht, hmT);
  return ht;
}

// Sound speed squared. TM: Eq. (sound_speed), c_s^2 = T (5h - 8T) / (3h (h - T)).
// Polytropic: Gamma T / h.
template <class R> __device__ __forceinline__ R cs2_of(const EosTM&, R T, R h) {
  return fdiv(T * (R(5) * h - R(8) * T), R(3) * h * (h - T));
}
template <class R> __device__ __forceinline__ R cs2_of(const EosPoly& e, R T, R h) {
  return fdiv(R(e.gam) * T, h);
}

// Packed FP32: the sm_100 family executes an add, a multiply or a fused
// multiply-add on both lanes of a float2 as one instruction (each lane
// rounded as its scalar counterpart). Paired work (two Newton solves, the
// two face states of a cell, the two sides of a face) is evaluated this
// way; reciprocals and square roots stay per lane.
namespace pk {
__device__ __forceinline__ float2 s2(float a) { return make_float2(a, a); }
// negation and subtraction as one packed instruction each (exact: x (-1))
__device__ __forceinline__ float2 neg(float2 a) { return __fmul2_rn(a, s2(-1.f)); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, s2(-1.f), a); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp(float2 a) { return make_float2(qrcp(a.x), qrcp(a.y)); }
__device__ __forceinline__ float2 rsq(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 sqr(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
}  // namespace pk

// The same operations on one float, one double or a packed float2, for code
// written once for all three (scalar forms may be contracted into FMAs).
namespace ar {
template <class V> __device__ __forceinline__ V c(double x) { return V(x); }
template <> __device__ __forceinline__ float2 c<float2>(double x) { return pk::s2(float(x)); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return pk::add(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return pk::mul(a, b); }
__device__ __forceinline__ float fma(float a, float b, float d) { return fmaf(a, b, d); }
__device__ __forceinline__ double fma(double a, double b, double d) { return ::fma(a, b, d); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 d) { return pk::fma(a, b, d); }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ float2 neg(float2 a) { return pk::neg(a); }
__device__ __forceinline__ float rcp(float a) { return qrcp(a); }
__device__ __forceinline__ double rcp(double a) { return qrcp(a); }
__device__ __forceinline__ float2 rcp(float2 a) { return pk::rcp(a); }
__device__ __forceinline__ float sqr(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqr(double a) { return sqrt(a); }
__device__ __forceinline__ float2 sqr(float2 a) { return pk::sqr(a); }
}  // namespace ar

// ---- conserved -> primitive: Newton-Raphson on the conic parameter --------
// The Taub-Mathews relation (h - 4T)(h - T) = 1 (Eq. TM EOS) is a hyperbola
// in (T, h) with the rational parametrisation t = h - T >= 1,
//   T = (t^2 - 1) / (3t),  h = (4t^2 - 1) / (3t).
// With tau = t - 1 and the identity h^2 - 1 - 2Th + T^2 h^2/(h^2 + m^2) =
// (h - T)^2 - 1 - T^2 m^2/(h^2 + m^2), the function f(htilde) of
// Eq. (transcendental equation) becomes
//   f = P N / Dn,  P = tau (2 + tau),  Q = (1 + 2 tau)(3 + 2 tau) = 4t^2 - 1,
//   N = Q^2 + m^2 (8t^2 + 1),  Dn = Q^2 + 9 t^2 m^2,
// where every term is positive (no cancellation, no square root). The
// conversions solve P N / Dn = A for tau by Newton-Raphson and then take
// htilde = tau (5 + 4 tau) / (3t) and T = tau (2 + tau) / (3t); the root is
// the htilde of Eq. (transcendental equation). The start
// tau0 = A / (1 + sqrt(1 + A)) is the exact root for m = 0 (there N = Dn)
// and within 7 % of the root elsewhere. N and Dn are multiplied by
// lam = 1 / (1 + tau0)^2, which leaves their ratio unchanged and keeps both
// of order t^2 + m^2 (float range) instead of t^2 m^2.

// Start of the iteration (V = float, double or float2).
template <class V> __device__ __forceinline__ V tau_start(V A) {
  using namespace ar;
  return mul(A, rcp(add(c<V>(1.0), sqr(add(c<V>(1.0), A)))));
}

// Newton step delta = (P N/Dn - A) / (d/dtau)(P N/Dn) at tau. ml = m^2 lam,
// ml9 = 9 m^2 lam, nA = -A (fixed per solve).
template <class V>
__device__ __forceinline__ V tau_step(V tau, V ml, V ml9, V nA, V lam) {
  using namespace ar;
  const V t = add(tau, c<V>(1.0));
  const V t2 = add(t, t);
  const V s = mul(t, t);
  const V P = mul(tau, add(tau, c<V>(2.0)));
  const V Q = mul(fma(tau, c<V>(2.0), c<V>(1.0)), fma(tau, c<V>(2.0), c<V>(3.0)));
  const V Ql = mul(Q, lam);
  const V QQl = mul(Q, Ql);
  const V N = fma(ml, fma(s, c<V>(8.0), c<V>(1.0)), QQl);  // lam N
  const V Dn = fma(ml9, s, QQl);                              // lam Dn
  const V rD = rcp(Dn);
  const V r = mul(N, rD);                                      // N / Dn
  const V dN = mul(mul(t2, c<V>(8.0)), add(Ql, ml));          // lam dN/dtau = 16 t (Q + m^2) lam
  const V dD = mul(t2, fma(Ql, c<V>(8.0), ml9));              // lam dDn/dtau = 2t (8Q + 9 m^2) lam
  const V dr = mul(fma(neg(r), dD, dN), rD);                  // dr/dtau
  const V dG = fma(t2, r, mul(P, dr));                        // d(P r)/dtau, P' = 2t
  return mul(fma(P, r, nA), rcp(dG));
}
// In double the same step over the common denominator Dn^2, with one
// reciprocal instead of two (the products stay far inside the double range;
// in float they could overflow): delta = (P N - A Dn) Dn /
// (2t N Dn + P (dN Dn - N dD)). The residual P N - A Dn cancels exactly as
// P N/Dn - A does.
template <>
__device__ __forceinline__ double tau_step<double>(double tau, double ml, double ml9, double nA,
                                                   double lam) {
  const double t = tau + 1.0;
  const double t2 = t + t;
  const double s = t * t;
  const double P = tau * (tau + 2.0);
  const double Q = fma(tau, 2.0, 1.0) * fma(tau, 2.0, 3.0);
  const double Ql = Q * lam;
  const double QQl = Q * Ql;
  const double N = fma(ml, fma(s, 8.0, 1.0), QQl);
  const double Dn = fma(ml9, s, QQl);
  const double dN = (t2 * 8.0) * (Ql + ml);
  const double dD = t2 * fma(Ql, 8.0, ml9);
  const double num = fma(P, N, nA * Dn) * Dn;
  const double den = fma(t2 * N, Dn, P * fma(dN, Dn, -(N * dD)));
  return num * qrcp(den);
}

// ---- conserved -> primitive for the polytropic EoS --------------------------
// With T = k htilde (k = (Gamma-1)/Gamma) and (h - T) = 1 + (1-k) htilde, the
// same identity gives f = (1-k) htilde (2 + (1-k) htilde)
// - k^2 htilde^2 m^2/(h^2 + m^2), rational in htilde; Newton-Raphson on
// htilde from the m = 0 root htilde0 = A / ((1-k)(1 + sqrt(1 + A))). Its
// quadratic constant is <= 0.67 for 1 < Gamma <= 5/3 (measured over
// T 1e-10..1e6, gamma 1..1e6), so the stopping rule of NewtonCfg holds.
template <class V> __device__ __forceinline__ V poly_start(V A, V omk) {
  using namespace ar;
  return mul(A, rcp(mul(omk, add(c<V>(1.0), sqr(add(c<V>(1.0), A))))));
}

// Newton step (f - A)/f' at htilde = x; omk = 1 - k, k2 = k^2, nA = -A.
template <class V>
__device__ __forceinline__ V poly_step(V x, V m2, V omk, V k2, V nA) {
  using namespace ar;
  const V h = add(x, c<V>(1.0));
  const V q = fma(h, h, m2);
  const V rq = rcp(q);
  const V ox = mul(omk, x);
  const V km = mul(mul(k2, m2), rq);                      // k^2 m^2 / q
  const V G = fma(neg(mul(km, x)), x, fma(ox, add(ox, c<V>(2.0)), nA));   // f - A
  // f' = 2 (1-k)(1 + (1-k) x) - 2 k^2 x m^2 (q - x h) / q^2
  const V dG = mul(c<V>(2.0), fma(neg(mul(km, x)), mul(fma(neg(x), h, q), rq),
                                  mul(omk, add(ox, c<V>(1.0)))));
  return mul(G, rcp(dG));
}
// In double the same step times q^2 above and below, with one reciprocal:
// delta = (f - A) q^2 / (f' q^2).
template <>
__device__ __forceinline__ double poly_step<double>(double x, double m2, double omk, double k2,
                                                    double nA) {
  const double h = x + 1.0;
  const double q = fma(h, h, m2);
  const double ox = omk * x;
  const double kmx = (k2 * m2) * x;
  const double Gq = fma(fma(ox, ox + 2.0, nA), q, -(kmx * x));       // (f - A) q
  const double den = 2.0 * fma(omk * (ox + 1.0), q * q, -(kmx * fma(-x, h, q)));  // f' q^2
  return Gq * q * qrcp(den);
}

// Precision tags. S is the storage and arithmetic type; AT is the type in
// which A of Eq. (transcendental equation) is formed.
struct PrecFP64 {     // SRHD_FP64: double everywhere
  using S = double;
  using AT = double;
  static constexpr bool comp_a = false;
};
struct PrecMixed {    // SRHD_MIXED: float, the cancelling part of A in double (A_mixed)
  using S = float;
  using AT = float;
  static constexpr bool comp_a = false;
};
struct PrecMixedCF {  // SRHD_MIXED_CF: float, A by a compensated float sum
  using S = float;
  using AT = float;
  static constexpr bool comp_a = true;
};

// A = (Et/D)^2 + 2 Et/D - (|M|/D)^2 in double (Eq. transcendental equation,
// left-hand side; Eq. Unphysical result) and m^2 = (|M|/D)^2.
// ori = 1: the original scheme's total energy E in the fifth slot, and
// A = (E/D)^2 - (|M|/D)^2 - 1 (Section 2.3: the form that cancels for cold gas).
template <class S>
__device__ __forceinline__ double A_of_cons(S D, S Mx, S My, S Mz, S Et, double& m2,
                                            int ori = 0) {
  double rD = drcp(double(D));
  double eD = double(Et) * rD;
  double M2 = double(Mx) * double(Mx) + double(My) * double(My) + double(Mz) * double(Mz);
  m2 = M2 * rD * rD;
  if (ori) return (eD * eD - m2) - 1.0;
  return eD * (eD + 2.0) - m2;
}

// Correctly rounded float operations on one lane (float) or two lanes
// (float2, packed instructions); the _rn forms keep the compiler from
// contracting them into other FMAs.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vrcp(float a) { return qrcp(a); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return pk::add(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return pk::sub(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return pk::mul(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return pk::fma(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return pk::neg(a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return pk::rcp(a); }
template <class V> __device__ __forceinline__ V vsplat(float a);
template <> __device__ __forceinline__ float vsplat<float>(float a) { return a; }
template <> __device__ __forceinline__ float2 vsplat<float2>(float a) { return make_float2(a, a); }

// Error-free transformations (Knuth's TwoSum; the FMA form of Dekker's
// TwoProduct): a*b = p + e and a+b = s + e exactly, lane by lane.
template <class V> __device__ __forceinline__ void two_prod(V a, V b, V& p, V& e) {
  p = vmul(a, b);
  e = vfma(a, b, vneg(p));
}
template <class V> __device__ __forceinline__ void two_sum(V a, V b, V& s, V& e) {
  s = vadd(a, b);
  V bb = vsub(s, a);
  e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
}

// Power-of-two scale 2^(127 - ex) that brings D into [1, 2) (exact); false
// for a non-positive, denormal-flushed, huge or NaN D.
__device__ __forceinline__ bool comp_scale(float D, float& sc) {
  const int ex = (__float_as_int(D) >> 23) & 0xff;
  sc = __int_as_float((254 - (ex > 253 ? 253 : ex)) << 23);
  return D > 0.0f && ex <= 253;
}

// A and m^2 of a float-stored state with the cancellation in double
// (SRHD_MIXED). The state is first scaled by the power of two that brings D
// into [1, 2) (comp_scale; exact in float, and A and m^2 do not change);
// then A d^2 = e (e + 2d) - |m|^2 (original scheme: e^2 - d^2 - |m|^2) of
// the scaled values is formed in double without a division, rounded to
// float and scaled by 1/d^2 in float, and m^2 = (|m|/d)^2 is formed in
// float: neither step cancels, so A keeps a few float ulps of relative
// accuracy, the precision of the float iteration that uses it, with no
// range limit on D.
__device__ __forceinline__ bool A_mixed(float D, float Mx, float My, float Mz, float Et, float& A,
                                        float& m2, int ori) {
  float sc;
  if (!comp_scale(D, sc)) return false;
  const float d = D * sc, ef = Et * sc, mxf = Mx * sc, myf = My * sc, mzf = Mz * sc;
  const double dd = d, e = ef, mx = mxf, my = myf, mz = mzf;
  double ad2 = ori ? fma(e, e, -(dd * dd)) : e * fma(2.0, dd, e);
  ad2 = fma(-mx, mx, ad2);
  ad2 = fma(-my, my, ad2);
  ad2 = fma(-mz, mz, ad2);
  const float rd = qrcp(d);
  A = float(ad2) * (rd * rd);
  const float ux = mxf * rd, uy = myf * rd, uz = mzf * rd;
  m2 = ux * ux + uy * uy + uz * uz;
  return A > float(kEpsUnphysical);
}

// A and m^2 from float conserved values without double arithmetic.
// A D^2 = Et^2 + 2 Et D - (Mx^2 + My^2 + Mz^2): every product is split exactly
// into a float pair and the sum of the ten parts is compensated, so the
// cancellation between Et^2 + 2 Et D and |M|^2 (the source of the
// (1 + Mach^2) error factor of Eq. ImprovedRelativeError) acts on a sum that
// is accurate to about eps_float^2 of its terms instead of eps_float. The
// inputs (d, e, mx, my, mz here) are first scaled by comp_scale, which keeps
// the products and their error parts clear of the float overflow and
// underflow (flush-to-zero) ranges. V = float or float2 (two states).
template <class V>
__device__ __forceinline__ void A_comp_scaled(V d, V e, V mx, V my, V mz, V& A, V& m2, int ori) {
  V p1, e1, p2, e2, p3, e3, p4, e4, p5, e5;
  two_prod(e, e, p1, e1);
  if (ori) {  // original scheme: A D^2 = E^2 - D^2 - |M|^2
    two_prod(d, d, p2, e2);
    p2 = vneg(p2);
    e2 = vneg(e2);
  } else {    // A D^2 = Et^2 + 2 Et D - |M|^2
    two_prod(e, d, p2, e2);
    p2 = vmul(p2, vsplat<V>(2.0f));
    e2 = vmul(e2, vsplat<V>(2.0f));
  }
  two_prod(mx, mx, p3, e3);
  two_prod(my, my, p4, e4);
  two_prod(mz, mz, p5, e5);
  V sa, ta, sb, tb, t2, ss, ts;
  two_sum(p1, p2, sa, ta);
  two_sum(p3, p4, sb, tb);
  two_sum(sb, p5, sb, t2);
  tb = vadd(tb, t2);
  two_sum(sa, vneg(sb), ss, ts);
  const V low = vadd(vsub(vadd(e1, e2), vadd(vadd(e3, e4), e5)), vadd(vsub(ta, tb), ts));
  const V ad2 = vadd(ss, low);
  // A = ad2 / d^2 with d^2 = dh + dl exact (TwoProduct) and 1/dh from the
  // hardware reciprocal refined by one Newton-Raphson step; one residual
  // correction q += (ad2 - q dh - q dl) / dh then leaves A within about one
  // rounding of the exact quotient.
  V dh, dl;
  two_prod(d, d, dh, dl);
  V r = vrcp(dh);
  r = vfma(r, vfma(vneg(dh), r, vsplat<V>(1.0f)), r);
  const V q = vmul(ad2, r);
  const V res = vsub(vfma(vneg(q), dh, ad2), vmul(q, dl));
  A = vfma(res, r, q);
  m2 = vmul(vadd(sb, tb), r);
}

__device__ __forceinline__ bool A_comp_float(float D, float Mx, float My, float Mz, float Et,
                                             float& A, float& m2, int ori = 0) {
  float sc;
  if (!comp_scale(D, sc)) return false;
  A_comp_scaled(vmul(D, sc), vmul(Et, sc), vmul(Mx, sc), vmul(My, sc), vmul(Mz, sc), A, m2, ori);
  return true;
}

// A_comp_float of two states with packed arithmetic.
__device__ __forceinline__ void A_comp_float_x2(const float (&Ua)[5], const float (&Ub)[5],
                                                float& Aa, float& m2a, bool& oka, float& Ab,
                                                float& m2b, bool& okb, int ori) {
  float sa, sb;
  oka = comp_scale(Ua[0], sa);
  okb = comp_scale(Ub[0], sb);
  const float2 sc = make_float2(sa, sb);
  float2 A, m2;
  A_comp_scaled(pk::mul(make_float2(Ua[0], Ub[0]), sc), pk::mul(make_float2(Ua[4], Ub[4]), sc),
                pk::mul(make_float2(Ua[1], Ub[1]), sc), pk::mul(make_float2(Ua[2], Ub[2]), sc),
                pk::mul(make_float2(Ua[3], Ub[3]), sc), A, m2, ori);
  Aa = A.x;
  Ab = A.y;
  m2a = m2.x;
  m2b = m2.y;
  oka = oka && Aa > float(kEpsUnphysical);
  okb = okb && Ab > float(kEpsUnphysical);
}

// A and m^2 of a conserved state in the precision of P; false when the
// state fails Eq. (Unphysical result) (A <= eps_machine) or D <= 0.
template <class P>
__device__ __forceinline__ bool A_and_m2(typename P::S D, typename P::S Mx, typename P::S My,
                                         typename P::S Mz, typename P::S Et,
                                         typename P::AT& A, typename P::AT& m2, int ori = 0) {
  if constexpr (P::comp_a) {
    if (!A_comp_float(D, Mx, My, Mz, Et, A, m2, ori)) return false;
    return A > float(kEpsUnphysical);
  } else if constexpr (sizeof(typename P::S) == 4) {
    return A_mixed(D, Mx, My, Mz, Et, A, m2, ori);
  } else {
    if (!(double(D) > 0.0)) return false;
    double m2d;
    double Ad = A_of_cons(D, Mx, My, Mz, Et, m2d, ori);
    A = Ad;
    m2 = m2d;
    return Ad > kEpsUnphysical;
  }
}

// Primitives from the converged conic parameter tau (Eq. four-velocity,
// Eq. new expression of Lorentz factor, Eq. density, Eq. p=rhoT):
// htilde = tau (5 + 4 tau) / (3t), T = tau (2 + tau) / (3t), t = 1 + tau.
template <class R, class S>
__device__ __forceinline__ void prims_from_tau(S D, S Mx, S My, S Mz, R tau, PrimX<R>& W) {
  const R r3t = qrcp(R(3) * (R(1) + tau));
  const R ht = tau * (R(5) + R(4) * tau) * r3t;
  const R h = R(1) + ht;
  const R rDh = fdiv(R(1), R(D) * h);
  W.u[0] = R(Mx) * rDh;
  W.u[1] = R(My) * rDh;
  W.u[2] = R(Mz) * rDh;
  const R g2 = R(1) + (W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2]);
  const R rg = rsqrt_r(g2);
  W.gamma = g2 * rg;
  W.rg = rg;
  W.rho = R(D) * rg;
  W.T = tau * (R(2) + tau) * r3t;
  W.h = h;
  W.ht = ht;
  W.tau = tau;
  W.p = W.rho * W.T;
}

// prims_from_tau of two float states with packed arithmetic.
__device__ __forceinline__ void prims_from_tau_x2(const float (&Ua)[5], const float (&Ub)[5],
                                                  float2 tau, PrimX<float>& Wa,
                                                  PrimX<float>& Wb) {
  using namespace pk;
  const float2 r3t = rcp(fma(tau, s2(3.f), s2(3.f)));
  const float2 ht = mul(mul(tau, fma(tau, s2(4.f), s2(5.f))), r3t);
  const float2 T = mul(mul(tau, add(tau, s2(2.f))), r3t);
  const float2 D = make_float2(Ua[0], Ub[0]);
  const float2 h = add(ht, s2(1.f));
  const float2 Dh = mul(D, h);
  const float2 rDh = rcp(Dh);
  const float2 ux = mul(make_float2(Ua[1], Ub[1]), rDh);
  const float2 uy = mul(make_float2(Ua[2], Ub[2]), rDh);
  const float2 uz = mul(make_float2(Ua[3], Ub[3]), rDh);
  const float2 g2 = fma(uz, uz, fma(uy, uy, fma(ux, ux, s2(1.f))));
  const float2 rg = rsq(g2);
  const float2 gamma = mul(g2, rg);
  const float2 rho = mul(D, rg);
  const float2 p = mul(rho, T);
  Wa.rho = rho.x; Wa.u[0] = ux.x; Wa.u[1] = uy.x; Wa.u[2] = uz.x; Wa.p = p.x;
  Wa.T = T.x; Wa.h = h.x; Wa.gamma = gamma.x; Wa.rg = rg.x; Wa.ht = ht.x; Wa.tau = tau.x;
  Wb.rho = rho.y; Wb.u[0] = ux.y; Wb.u[1] = uy.y; Wb.u[2] = uz.y; Wb.p = p.y;
  Wb.T = T.y; Wb.h = h.y; Wb.gamma = gamma.y; Wb.rg = rg.y; Wb.ht = ht.y; Wb.tau = tau.y;
}

// Primitives from the converged htilde of the polytropic EoS (T = k htilde).
template <class R, class S>
__device__ __forceinline__ void prims_from_ht_poly(S D, S Mx, S My, S Mz, R ht, R k,
                                                   PrimX<R>& W) {
  const R h = R(1) + ht;
  const R rDh = fdiv(R(1), R(D) * h);
  W.u[0] = R(Mx) * rDh;
  W.u[1] = R(My) * rDh;
  W.u[2] = R(Mz) * rDh;
  const R g2 = R(1) + (W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2]);
  const R rg = rsqrt_r(g2);
  W.gamma = g2 * rg;
  W.rg = rg;
  W.rho = R(D) * rg;
  W.T = k * ht;
  W.h = h;
  W.ht = ht;
  W.tau = ht;
  W.p = W.rho * W.T;
}

// Cold start of the solver variable for A (the root for m = 0): tau_start
// (TM), poly_start (polytropic). A converged x divided by this start
// changes slowly between neighbouring states (the start follows A exactly
// and the ratio only the dependence on m), so a nearby state's ratio times
// this state's start is a warm start closer to the root than the nearby x
// itself.
template <class V> __device__ __forceinline__ V x_start(const EosTM&, V A) { return tau_start(A); }
template <class V> __device__ __forceinline__ V x_start(const EosPoly& e, V A) {
  return poly_start(A, ar::c<V>(1.0 - (e.gam - 1.0) / e.gam));
}

// rt of a state known by its primitives: its solver variable in closed form
// (solver_var_of_T) over the cold start for its A, with A from the
// primitives (Et/D as in prim2con, m = h |U|). Only a warm start: where A
// cancels to <= 0 the result is not positive and the solve starts cold.
template <class R, class E>
__device__ __forceinline__ R rt_of_prims(const E& eos, R rho, R u0, R u1, R u2, R p) {
  const R T = qdiv(p, rho);
  R ht, hmT;
  eos_ht(eos, T, ht, hmT);
  const R uu = u0 * u0 + u1 * u1 + u2 * u2;
  const R g2 = R(1) + uu;
  const R rg = rsqrt_r(g2);
  const R gamma = g2 * rg;
  const R e = qdiv(uu, gamma + R(1)) + (hmT + ht * uu) * rg;  // Et / D
  const R h = R(1) + ht;
  const R A = e * (e + R(2)) - h * h * uu;
  return qdiv(solver_var_of_T(eos, T), x_start(eos, A));
}

// Solver of Eq. (transcendental equation) per EoS, in the variable x that
// the warm starts carry (tau for TM, htilde for the polytropic EoS):
// init(A, m2) fixes the per-state constants, start() gives x0, step(x) the
// Newton step, prims() the primitives from the converged x.
template <class E, class V> struct Solver;
template <class V> struct Solver<EosTM, V> {
  V ml, ml9, nA, lam;
  // constants of a solve that starts at x0 (the scale lam = 1/(1 + x0)^2)
  __device__ __forceinline__ void prepare(const EosTM&, V A, V m2, V x0) {
    using namespace ar;
    const V t1 = add(x0, c<V>(1.0));
    lam = rcp(mul(t1, t1));
    ml = mul(m2, lam);
    ml9 = mul(ml, c<V>(9.0));
    nA = neg(A);
  }
  __device__ __forceinline__ V init(const EosTM& e, V A, V m2) {
    const V t0 = tau_start(A);
    prepare(e, A, m2, t0);
    return t0;
  }
  __device__ __forceinline__ V step(V x) const { return tau_step(x, ml, ml9, nA, lam); }
};
template <class V> struct Solver<EosPoly, V> {
  V m2, omk, k2, nA;
  __device__ __forceinline__ void prepare(const EosPoly& e, V A, V m2_, V) {
    using namespace ar;
    const double k = (e.gam - 1.0) / e.gam;
    m2 = m2_;
    omk = c<V>(1.0 - k);
    k2 = c<V>(k * k);
    nA = neg(A);
  }
  __device__ __forceinline__ V init(const EosPoly& e, V A, V m2_) {
    prepare(e, A, m2_, A);
    return poly_start(A, omk);
  }
  __device__ __forceinline__ V step(V x) const { return poly_step(x, m2, omk, k2, nA); }
};

template <class R, class S>
__device__ __forceinline__ void prims_from_x(const EosTM&, S D, S Mx, S My, S Mz, R x,
                                             PrimX<R>& W) {
  prims_from_tau(D, Mx, My, Mz, x, W);
}
template <class R, class S>
__device__ __forceinline__ void prims_from_x(const EosPoly& e, S D, S Mx, S My, S Mz, R x,
                                             PrimX<R>& W) {
  prims_from_ht_poly(D, Mx, My, Mz, x, R((e.gam - 1.0) / e.gam), W);
}

template <class R> __device__ __forceinline__ void set_nan(PrimX<R>& W) {
  const R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
  W.rho = W.u[0] = W.u[1] = W.u[2] = W.p = W.T = W.h = W.gamma = W.rg = W.ht = W.tau = W.rt = nan;
}

// Stopping rule of the Newton iterations (per state): the step just applied
// was at most tol of tau.
template <class R> __device__ __forceinline__ bool newton_done(R adh, R tau) {
  return adh <= NewtonCfg<R>::tol * tau;
}

// Conserved -> primitive (Section 2.3). Returns 0 ok, 1 unphysical, 2 no
// convergence. A and m^2 as in Eq. (transcendental equation) and
// Eq. (Unphysical result), then Newton-Raphson for the conic parameter tau
// (see above); a step that would make tau non-positive halves tau instead.
// Stops by newton_done or after maxit steps (status 2). guess > 0 is a tau
// to start from (a warm start from a nearby state); otherwise tau_start(A).
// With RATIO, a warm guess is a nearby state's rt and the start is guess
// times this state's x_start(A), and a cold conversion also returns W.rt.
// The root does not depend on the start.
template <class P, class E = EosTM, bool WARM = false, bool RATIO = false>
__device__ __forceinline__ int con2pri(typename P::S D, typename P::S Mx, typename P::S My,
                                       typename P::S Mz, typename P::S Et,
                                       PrimX<typename P::S>& W, int maxit,
                                       typename P::S guess = typename P::S(0), int ori = 0,
                                       const E& eos = E()) {
  using R = typename P::S;
  typename P::AT Aa, m2a;
  if (!A_and_m2<P>(D, Mx, My, Mz, Et, Aa, m2a, ori)) {
    set_nan(W);
    return 1;
  }
  const R A = R(Aa), m2 = R(m2a);
  Solver<E, R> sv;
  R tau;
  [[maybe_unused]] R t0c = R(1);
  if constexpr (WARM) {
    if constexpr (RATIO) {
      const R x0 = x_start(eos, A);
      tau = guess > R(0) ? guess * x0 : x0;
    } else {
      tau = guess > R(0) ? guess : R(1);
    }
    sv.prepare(eos, A, m2, tau);
  } else {
    const R t0 = sv.init(eos, A, m2);
    t0c = t0;
    tau = guess > R(0) ? guess : t0;
  }
  int status = 2;
  for (int k = 1; k <= maxit; ++k) {
    const R dh = sv.step(tau);
    R tn = tau - dh;
    if (!(tn > R(0))) tn = R(0.5) * tau;
    tau = tn;
    if (newton_done(fabs(dh), tau)) { status = 0; break; }
  }
  prims_from_x(eos, D, Mx, My, Mz, tau, W);
  if constexpr (RATIO && !WARM) W.rt = qdiv(tau, t0c);
  return status;
}

// Two conserved -> primitive conversions advanced in lockstep: the same
// iteration and stopping rule as con2pri, applied to two independent states
// so that their dependency chains interleave (in float, both lanes of each
// step are one packed instruction). The loop runs until both have stopped;
// a state that has stopped is not updated.
template <class P, class E = EosTM, bool WARM = false, bool RATIO = false>
__device__ __forceinline__ void con2pri_x2(const typename P::S (&Ua)[5],
                                           const typename P::S (&Ub)[5],
                                           PrimX<typename P::S>& Wa, PrimX<typename P::S>& Wb,
                                           int maxit, int& sta, int& stb,
                                           typename P::S ga = typename P::S(0),
                                           typename P::S gb = typename P::S(0), int ori = 0,
                                           const E& eos = E()) {
  using R = typename P::S;
  typename P::AT Aa_, ma_, Ab_, mb_;
  bool pa, pb;
  if constexpr (P::comp_a) {
    A_comp_float_x2(Ua, Ub, Aa_, ma_, pa, Ab_, mb_, pb, ori);
  } else {
    pa = A_and_m2<P>(Ua[0], Ua[1], Ua[2], Ua[3], Ua[4], Aa_, ma_, ori);
    pb = A_and_m2<P>(Ub[0], Ub[1], Ub[2], Ub[3], Ub[4], Ab_, mb_, ori);
  }
  // an unphysical state iterates on a harmless stand-in and is discarded
  const R Aa = pa ? R(Aa_) : R(1), m2a = pa ? R(ma_) : R(0);
  const R Ab = pb ? R(Ab_) : R(1), m2b = pb ? R(mb_) : R(0);
  bool da = false, db = false;
  if constexpr (sizeof(R) == 4) {
    using namespace pk;
    Solver<E, float2> sv;
    float2 tau;
    [[maybe_unused]] float2 t0c = make_float2(1.0f, 1.0f);
    if constexpr (WARM) {
      if constexpr (RATIO) {
        const float2 x0 = x_start(eos, make_float2(Aa, Ab));
        tau = make_float2(ga > 0.0f ? ga * x0.x : x0.x, gb > 0.0f ? gb * x0.y : x0.y);
      } else {
        tau = make_float2(ga > 0.0f ? ga : 1.0f, gb > 0.0f ? gb : 1.0f);
      }
      sv.prepare(eos, make_float2(Aa, Ab), make_float2(m2a, m2b), tau);
    } else {
      const float2 t0 = sv.init(eos, make_float2(Aa, Ab), make_float2(m2a, m2b));
      t0c = t0;
      tau = make_float2(ga > 0.0f ? ga : t0.x, gb > 0.0f ? gb : t0.y);
    }
    for (int k = 1; k <= maxit && !(da && db); ++k) {
      const float2 dh = sv.step(tau);
      const float2 tn = sub(tau, dh);
      // a state that has stopped keeps its tau
      const float tx = tn.x > 0.0f ? tn.x : 0.5f * tau.x;
      const float ty = tn.y > 0.0f ? tn.y : 0.5f * tau.y;
      const bool cx = newton_done(fabsf(dh.x), tx), cy = newton_done(fabsf(dh.y), ty);
      tau.x = da ? tau.x : tx;
      tau.y = db ? tau.y : ty;
      da = da || cx;
      db = db || cy;
    }
    if constexpr (std::is_same<E, EosTM>::value) {
      prims_from_tau_x2(Ua, Ub, tau, Wa, Wb);
    } else {
      prims_from_x(eos, Ua[0], Ua[1], Ua[2], Ua[3], tau.x, Wa);
      prims_from_x(eos, Ub[0], Ub[1], Ub[2], Ub[3], tau.y, Wb);
    }
    if constexpr (RATIO && !WARM) {
      Wa.rt = qdiv(tau.x, t0c.x);
      Wb.rt = qdiv(tau.y, t0c.y);
    }
  } else {
    Solver<E, R> sva, svb;
    R ta, tb;
    [[maybe_unused]] R t0ca = R(1), t0cb = R(1);
    if constexpr (WARM) {
      if constexpr (RATIO) {
        const R x0a = x_start(eos, Aa), x0b = x_start(eos, Ab);
        ta = ga > R(0) ? ga * x0a : x0a;
        tb = gb > R(0) ? gb * x0b : x0b;
      } else {
        ta = ga > R(0) ? ga : R(1);
        tb = gb > R(0) ? gb : R(1);
      }
      sva.prepare(eos, Aa, m2a, ta);
      svb.prepare(eos, Ab, m2b, tb);
    } else {
      const R t0a = sva.init(eos, Aa, m2a), t0b = svb.init(eos, Ab, m2b);
      t0ca = t0a;
      t0cb = t0b;
      ta = ga > R(0) ? ga : t0a;
      tb = gb > R(0) ? gb : t0b;
    }
    for (int k = 1; k <= maxit && !(da && db); ++k) {
      const R dha = sva.step(ta);
      const R dhb = svb.step(tb);
      R tna = ta - dha, tnb = tb - dhb;
      if (!(tna > R(0))) tna = R(0.5) * ta;
      if (!(tnb > R(0))) tnb = R(0.5) * tb;
      const bool ca = newton_done(fabs(dha), tna), cb = newton_done(fabs(dhb), tnb);
      ta = da ? ta : tna;
      tb = db ? tb : tnb;
      da = da || ca;
      db = db || cb;
    }
    prims_from_x(eos, Ua[0], Ua[1], Ua[2], Ua[3], ta, Wa);
    prims_from_x(eos, Ub[0], Ub[1], Ub[2], Ub[3], tb, Wb);
    if constexpr (RATIO && !WARM) {
      Wa.rt = qdiv(ta, t0ca);
      Wb.rt = qdiv(tb, t0cb);
    }
  }
  sta = da ? 0 : 2;
  stb = db ? 0 : 2;
  if (!pa) {
    set_nan(Wa);
    sta = 1;
  }
  if (!pb) {
    set_nan(Wb);
    stb = 1;
  }
}

// Primitive -> conserved (Eqs. density, momentum, T_to_HTilde and the
// reduced energy). Fills T, h, gamma, rg of W. Returns false if rho <= 0 or
// p <= 0. The reduced energy uses, instead of Eq. (E_D), the equivalent
// subtraction-free form
//   Et / D = h gamma - 1 - T / gamma = U^2 / (gamma + 1) + (htilde - T + htilde U^2) / gamma
// (gamma - 1 = U^2 / (gamma + 1); htilde - T = 1.5 T + 2.25 T^2 / (1 + sqrt(1 + 2.25 T^2))),
// which shares 1/gamma with the flux and needs one division and no square
// root beyond those of htilde and gamma.
template <class R, class E = EosTM>
__device__ __forceinline__ bool prim2con(PrimX<R>& W, R U[5], int ori = 0, const E& eos = E()) {
  if (!(W.rho > R(0)) || !(W.p > R(0))) {
    R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
    for (int v = 0; v < 5; ++v) U[v] = nan;
    return false;
  }
  const R T = qdiv(W.p, W.rho);
  R ht, hmT;                                     // htilde and htilde - T
  eos_ht(eos, T, ht, hmT);
  const R u2 = W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2];
  const R g2 = R(1) + u2;
  const R rg = rsqrt_r(g2);
  const R gamma = g2 * rg;
  const R D = W.rho * gamma;
  const R h = R(1) + ht;
  const R Dh = D * h;
  U[0] = D;
  U[1] = Dh * W.u[0];
  U[2] = Dh * W.u[1];
  U[3] = Dh * W.u[2];
  if (ori) {
    U[4] = Dh * gamma - W.p;  // original scheme: E = D h gamma - p
  } else {
    U[4] = D * (qdiv(u2, gamma + R(1)) + (hmT + ht * u2) * rg);
  }
  W.T = T;
  W.h = h;
  W.gamma = gamma;
  W.rg = rg;
  return true;
}

// prim2con and phys_flux<d> of two float states (lanes x, y of W[v]) with
// packed arithmetic; a lane with rho <= 0 or p <= 0 gets NaN conserved
// values and its ok flag false.
template <int d, class E = EosTM>
__device__ __forceinline__ void prim2con_flux_x2(const float2 (&W)[5], float2 (&U)[5],
                                                 float2 (&F)[5], bool& okx, bool& oky,
                                                 int ori, const E& eos = E()) {
  using namespace pk;
  okx = W[0].x > 0.0f && W[4].x > 0.0f;
  oky = W[0].y > 0.0f && W[4].y > 0.0f;
  const float2 T = mul(W[4], rcp(W[0]));
  float2 ht, hmT;                                          // htilde and htilde - T
  if constexpr (std::is_same<E, EosTM>::value) {
    const float2 a = mul(mul(s2(2.25f), T), T);
    const float2 sq = add(s2(1.f), make_float2(sqrtf(a.x + 1.0f), sqrtf(a.y + 1.0f)));
    const float2 t2 = mul(a, rcp(sq));                     // htilde - 2.5 T
    ht = fma(s2(2.5f), T, t2);
    hmT = fma(s2(1.5f), T, t2);
  } else {
    hmT = mul(T, s2(float(1.0 / (eos.gam - 1.0))));
    ht = add(T, hmT);
  }
  const float2 u2 = fma(W[3], W[3], fma(W[2], W[2], mul(W[1], W[1])));
  const float2 g2 = add(s2(1.f), u2);
  const float2 rg = rsq(g2);
  const float2 gamma = mul(g2, rg);
  const float2 D = mul(W[0], gamma);
  const float2 Dh = mul(D, add(s2(1.f), ht));
  U[0] = D;
  U[1] = mul(Dh, W[1]);
  U[2] = mul(Dh, W[2]);
  U[3] = mul(Dh, W[3]);
  if (ori) {
    U[4] = fma(Dh, gamma, neg(W[4]));  // original scheme: E = D h gamma - p
  } else {  // Et = D [U^2 / (gamma + 1) + (1.5 T + t2 + htilde U^2) / gamma]
    const float2 k1 = mul(u2, rcp(add(gamma, s2(1.f))));
    U[4] = mul(D, fma(fma(ht, u2, hmT), rg, k1));
  }
  const float2 v = mul(W[1 + d], rg);
  F[0] = mul(U[0], v);
  F[1] = mul(U[1], v);
  F[2] = mul(U[2], v);
  F[3] = mul(U[3], v);
  F[1 + d] = add(F[1 + d], W[4]);
  F[4] = ori ? U[1 + d] : mul(add(U[4], W[4]), v);
  // a state from a non-positive density or pressure: D = NaN marks it
  // unphysical for every later conversion (its attempt is redone anyway)
  const float nan = __int_as_float(0x7fc00000);
  if (!okx) U[0].x = nan;
  if (!oky) U[0].y = nan;
}

// Physical flux along d (Eqs. D evolution, M evolution, ETilde evolution).
template <int d, class R>
__device__ __forceinline__ void phys_flux(const PrimX<R>& W, const R U[5], R F[5], int ori = 0) {
  R v = W.u[d] * W.rg;
  F[0] = U[0] * v;
  F[1] = U[1] * v;
  F[2] = U[2] * v;
  F[3] = U[3] * v;
  F[1 + d] += W.p;
  F[4] = ori ? U[1 + d] : (U[4] + W.p) * v;  // original scheme: flux of E is M_d
}

// Outer characteristic speeds along d with the TM sound speed, in the
// four-velocity form [gamma U_d (1-cs2) -/+ sqrt(cs2 (1 + U_perp^2 (1-cs2)))]
// / [1 + U^2 (1-cs2)].
template <int d, class R, class E = EosTM>
__device__ __forceinline__ void char_speeds(const PrimX<R>& W, R& lm, R& lp, const E& eos = E()) {
  R cs2 = cs2_of(eos, W.T, W.h);
  R omc = R(1) - cs2;
  R ud = W.u[d];
  // transverse part summed directly (no u2 - ud^2 cancellation)
  R ua = W.u[d == 0 ? 1 : 0], ub = W.u[d == 2 ? 1 : 2];
  R up2 = ua * ua + ub * ub;
  R u2 = up2 + ud * ud;
  R rden = qrcp(R(1) + u2 * omc);
  R a = W.gamma * ud * omc;
  R b = sqrt(cs2 * (R(1) + up2 * omc));
  lm = (a - b) * rden;
  lp = (a + b) * rden;
}

// phys_flux<d> and char_speeds<d> of the left and right float states with
// packed arithmetic (lane x left, lane y right).
template <int d, class E = EosTM>
__device__ __forceinline__ void outer_parts_x2(const PrimX<float>& WL, const float UL[5],
                                               const PrimX<float>& WR, const float UR[5],
                                               float FL[5], float FR[5], float& lmL, float& lpL,
                                               float& lmR, float& lpR, int ori,
                                               const E& eos = E()) {
  using namespace pk;
  constexpr int a0 = d == 0 ? 1 : 0, b0 = d == 2 ? 1 : 2;  // transverse components
  const float2 ud = make_float2(WL.u[d], WR.u[d]);
  const float2 v = mul(ud, make_float2(WL.rg, WR.rg));
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = mul(make_float2(UL[q], UR[q]), v);
    FL[q] = f.x;
    FR[q] = f.y;
  }
  FL[1 + d] += WL.p;
  FR[1 + d] += WR.p;
  if (ori) {
    FL[4] = UL[1 + d];
    FR[4] = UR[1 + d];
  } else {
    const float2 f = mul(add(make_float2(UL[4], UR[4]), make_float2(WL.p, WR.p)), v);
    FL[4] = f.x;
    FR[4] = f.y;
  }
  // outer characteristic speeds (char_speeds)
  const float2 T = make_float2(WL.T, WR.T), h = make_float2(WL.h, WR.h);
  float2 cs2;
  if constexpr (std::is_same<E, EosTM>::value) {
    const float2 cnum = mul(T, fma(s2(-8.f), T, mul(s2(5.f), h)));
    const float2 cden = mul(mul(s2(3.f), h), sub(h, T));
    cs2 = make_float2(qdiv(cnum.x, cden.x), qdiv(cnum.y, cden.y));  // cden = 3h(h-T) in [3, 3h^2]
  } else {
    cs2 = mul(mul(s2(float(eos.gam)), T), rcp(h));
  }
  const float2 omc = sub(s2(1.f), cs2);
  const float2 ua = make_float2(WL.u[a0], WR.u[a0]), ub = make_float2(WL.u[b0], WR.u[b0]);
  const float2 up2 = fma(ub, ub, mul(ua, ua));
  const float2 u2 = fma(ud, ud, up2);
  const float2 rden = rcp(fma(u2, omc, s2(1.f)));
  const float2 a = mul(mul(make_float2(WL.gamma, WR.gamma), ud), omc);
  const float2 bb = mul(cs2, fma(up2, omc, s2(1.f)));
  const float2 b = make_float2(sqrtf(bb.x), sqrtf(bb.y));
  const float2 lm = mul(sub(a, b), rden), lp = mul(add(a, b), rden);
  lmL = lm.x;
  lmR = lm.y;
  lpL = lp.x;
  lpR = lp.y;
}

// Relativistic HLLC of Mignone & Bodo (2005) with E = Etilde + D inside the
// solver (Section 3.1), HLLE when requested or when the contact state is not
// admissible (discriminant < 0, contact speed outside the outer speeds, or
// non-positive contact pressure). Returns 1 on fallback.
template <int d, class R, class E = EosTM>
__device__ __forceinline__ int riemann(int solver, const PrimX<R>& WL, const R UL[5],
                                       const PrimX<R>& WR, const R UR[5], R F[5], int ori = 0,
                                       const E& eos = E()) {
  R FL[5], FR[5];
  R lmL, lpL, lmR, lpR;
  if constexpr (sizeof(R) == 4) {
    outer_parts_x2<d>(WL, UL, WR, UR, FL, FR, lmL, lpL, lmR, lpR, ori, eos);
  } else {
    phys_flux<d>(WL, UL, FL, ori);
    phys_flux<d>(WR, UR, FR, ori);
    char_speeds<d>(WL, lmL, lpL, eos);
    char_speeds<d>(WR, lmR, lpR, eos);
  }
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
  const R rds = qrcp(sR - sL);
  // HLL state and flux of component v
  auto hll_u = [&](int v) { return (sR * UR[v] - sL * UL[v] - FR[v] + FL[v]) * rds; };
  auto hll_f = [&](int v) { return (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) * rds; };
  if (solver == 0) {
    // the contact speed needs only the energy and normal-momentum components
    R E = ori ? hll_u(4) : hll_u(4) + hll_u(0);
    R FE = ori ? hll_f(4) : hll_f(4) + hll_f(0);
    R m = hll_u(1 + d);
    R Fm = hll_f(1 + d);
    R B = E + Fm;
    R disc = B * B - R(4) * FE * m;
    if (disc >= R(0) && B > R(0)) {
      R lam = qdiv(R(2) * m, B + sqrt(disc));
      R ps = Fm - lam * FE;
      if (lam > sL && lam < sR && ps > R(0)) {
        const bool left = lam >= R(0);
        const PrimX<R>& Wk = left ? WL : WR;
        const R* Uk = left ? UL : UR;
        const R* Fk = left ? FL : FR;
        R sk = left ? sL : sR;
        R v = Wk.u[d] * Wk.rg;
        R a = sk - v;
        R rb = qrcp(sk - lam);
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
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = hll_f(v);
  return solver == 0;
}

// Hybrid van Leer / generalised minmod slope: 0 at extrema, else the smaller
// in magnitude of 2 dl dr/(dl+dr) and minmod(theta dl, theta dr, (dl+dr)/2).
// Where dl and dr share a sign, |2 dl dr/(dl+dr)| (their harmonic mean) is at
// most |dl+dr|/2 (their arithmetic mean), so the third minmod argument never
// decides the minimum and is left out.
template <class R> __device__ __forceinline__ R limited_slope(R dl, R dr, R theta) {
  if (!(dl * dr > R(0))) return R(0);
  R vl = qdiv(R(2) * dl * dr, dl + dr);
  R mag = fmin(fabs(vl), theta * fmin(fabs(dl), fabs(dr)));
  return copysign(mag, dl);
}

// limited_slope of two independent (dl, dr) pairs, the arithmetic in packed
// form (lane by lane the same operations).
__device__ __forceinline__ float2 limited_slope_x2(float2 dl, float2 dr, float theta) {
  using namespace pk;
  const float2 pr = mul(dl, dr);
  const float2 vl = mul(mul(s2(2.0f), pr), rcp(add(dl, dr)));
  const float2 mn = make_float2(fminf(fabsf(dl.x), fabsf(dr.x)), fminf(fabsf(dl.y), fabsf(dr.y)));
  const float2 tm = mul(s2(theta), mn);
  const float mx = fminf(fabsf(vl.x), tm.x), my = fminf(fabsf(vl.y), tm.y);
  return make_float2(pr.x > 0.0f ? copysignf(mx, dl.x) : 0.0f,
                     pr.y > 0.0f ? copysignf(my, dl.y) : 0.0f);
}

// Signal speed bound S_max of one cell (Section 3.2, Eqs. time_step_U_max
// and SMax; |U_x|+|U_y|+|U_z| and ndim gamma U_s).
template <class R, class E = EosTM>
__device__ __forceinline__ R smax_of(const PrimX<R>& W, int ndim, const E& eos = E()) {
  R cs2 = cs2_of(eos, W.T, W.h);
  R omc = R(1) - cs2;
  R us = sqrt(qdiv(cs2, omc));      // U_s = c_s / sqrt(1 - c_s^2)
  R gs = rsqrt_r(omc);              // gamma_s = 1 / sqrt(1 - c_s^2)
  R su = fabs(W.u[0]) + fabs(W.u[1]) + fabs(W.u[2]);
  R umax = gs * su + R(ndim) * W.gamma * us;
  return umax * rsqrt_r(R(1) + umax * umax);
}

}  // namespace srhd
