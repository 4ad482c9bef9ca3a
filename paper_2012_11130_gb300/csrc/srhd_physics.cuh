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

// Newton stopping rule. Near the root the iteration converges
// quadratically, e_{k+1} <= C e_k^2 in relative terms, with C <= 0.56 over
// the whole range of states (measured with the oracle: rho 1e-6..1e2,
// T 1e-8..1e4, gamma 1..1e4). Once a step satisfies |dh| <= tol htilde the
// error left after applying it is at most C tol^2: 3e-17 for tol = 2^-27 in
// double and 8e-9 for tol = 2^-13 in float, below the rounding of either
// precision, so the iteration stops there instead of taking one more step.
// A step that stops contracting at the rounding floor also ends it.
template <class R> struct NewtonCfg;
template <> struct NewtonCfg<double> {
  static constexpr double tol = 7.450580596923828e-09;  // 2^-27
  static constexpr double floor = 1e-12;
  static constexpr int maxit = 50;
};
template <> struct NewtonCfg<float> {
  static constexpr float tol = 1.220703125e-04f;  // 2^-13
  static constexpr float floor = 1e-4f;
  static constexpr int maxit = 30;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// Quotient and reciprocal in the arithmetic type. In float they are the
// hardware approximate division (at most 2 ulp, like the '/' operator under
// -prec-div=false, but without its range scaling: valid for divisors of
// magnitude below 2^126, which every denominator they are used on stays far
// below); in double they are the IEEE operations.
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qrcp(float b) { return __fdividef(1.0f, b); }
__device__ __forceinline__ double qrcp(double b) { return 1.0 / b; }

// Primitive state with the derived quantities reused downstream.
template <class R> struct PrimX {
  R rho, u[3], p;   // W = (rho, U^x, U^y, U^z, p)
  R T, h, gamma;    // T = p/rho, h = 1 + htilde, gamma = sqrt(1 + U.U)
  R rg;             // 1 / gamma (three-velocity v = U rg)
  R ht;             // htilde (set by the conversions from conserved variables)
};

// Eq. (T_to_HTilde): htilde(T) without subtraction.
template <class R> __device__ __forceinline__ R htilde_of_T(R T) {
  R a = R(2.25) * T * T;
  return R(2.5) * T + qdiv(a, R(1) + sqrt(a + R(1)));
}

// Eq. (T of h) and its derivative Eq. (dT_dh), sharing one reciprocal square
// root and one division: with x = 9 ht^2 + 18 ht + 25, s = sqrt(x),
// den = 5 ht + 5 + s: T = (2 ht^2 + 4 ht)/den and
// dT = [(4 ht + 4) - T ((9 ht + 9)/s + 5)] / den.
template <class R> __device__ __forceinline__ void T_dT_of_htilde(R ht, R& T, R& dT) {
  R x = (R(9) * ht + R(18)) * ht + R(25);
  R rs = rsqrt_r(x);
  R den = R(5) * ht + R(5) + x * rs;
  R rden = qrcp(den);
  T = (R(2) * ht + R(4)) * ht * rden;
  dT = ((R(4) * ht + R(4)) - T * ((R(9) * ht + R(9)) * rs + R(5))) * rden;
}

template <class R> __device__ __forceinline__ R T_of_htilde(R ht) {
  R x = (R(9) * ht + R(18)) * ht + R(25);
  return qdiv((R(2) * ht + R(4)) * ht, R(5) * ht + R(5) + sqrt(x));
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
  R rq = qrcp(hh + m2);
  R a1 = hh * rq, a2 = m2 * rq;
  f = ht * (ht + R(2)) - R(2) * T * h + T * T * a1;
  df = R(2) * h - R(2) * T - R(2) * h * dT +
       R(2) * T * rq * (dT * hh * a1 + h * (h * dT + T) * a2);
}

// Packed FP32: the sm_100 family executes an add, a multiply or a fused
// multiply-add on both lanes of a float2 as one instruction (each lane
// rounded as its scalar counterpart). The paired Newton solves evaluate the
// polynomial part of both states' iterations this way; reciprocals and
// square roots stay per lane.
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

// T_dT_of_htilde and f_df on two lanes.
__device__ __forceinline__ void T_dT_of_htilde(float2 ht, float2& T, float2& dT) {
  const float2 x = fma(fma(ht, s2(9.f), s2(18.f)), ht, s2(25.f));
  const float2 rs = rsq(x);
  const float2 rden = rcp(fma(x, rs, fma(ht, s2(5.f), s2(5.f))));
  T = mul(mul(fma(ht, s2(2.f), s2(4.f)), ht), rden);
  // dT = [(4 ht + 4) + T ((-9 ht - 9) rs - 5)] rden
  dT = mul(fma(T, fma(fma(ht, s2(-9.f), s2(-9.f)), rs, s2(-5.f)), fma(ht, s2(4.f), s2(4.f))),
           rden);
}
__device__ __forceinline__ void f_df(float2 ht, float2 T, float2 dT, float2 m2, float2& f,
                                     float2& df) {
  const float2 h = add(ht, s2(1.f));
  const float2 hh = mul(h, h);
  const float2 rq = rcp(add(hh, m2));
  const float2 a1 = mul(hh, rq), a2 = mul(m2, rq);
  f = fma(mul(T, T), a1, fma(mul(s2(-2.f), T), h, mul(ht, add(ht, s2(2.f)))));
  const float2 inner = fma(dT, mul(hh, a1), mul(mul(h, fma(h, dT, T)), a2));
  // df = 2 [h (1 - dT) - T + T rq inner]
  df = mul(s2(2.f), fma(mul(T, rq), inner, sub(mul(h, fma(dT, s2(-1.f), s2(1.f))), T)));
}
}  // namespace pk

// Appendix A initial guess: hot (4/3) sqrt(A) above the Eq. (ColdHot)
// threshold, else the positive root of the quadratic of Eq. (cold limit of
// transcendental eq) in cancellation-free form.
template <class R> __device__ __forceinline__ R newton_guess(R A, R m2) {
  R P = R(1) + m2;
  R tb = qdiv(R(1800) * P, R(437) * m2 + R(117));
  if (A > tb * tb) return R(4.0 / 3.0) * sqrt(A);
  R a = qdiv(R(43) * m2 + R(63), R(125) * P);
  return qdiv(R(2) * A, R(1.2) + sqrt(R(1.44) + R(4) * a * A));
}

// Precision tags. S is the storage and arithmetic type; AT is the type in
// which A of Eq. (transcendental equation) is formed.
struct PrecFP64 {     // SRHD_FP64: double everywhere
  using S = double;
  using AT = double;
  static constexpr bool comp_a = false;
};
struct PrecMixed {    // SRHD_MIXED: float, A in double
  using S = float;
  using AT = double;
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
  double rD = 1.0 / double(D);
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
  } else {
    if (!(double(D) > 0.0)) return false;
    double m2d;
    double Ad = A_of_cons(D, Mx, My, Mz, Et, m2d, ori);
    A = Ad;
    m2 = m2d;
    return Ad > kEpsUnphysical;
  }
}

// Primitives from a converged htilde (Eq. four-velocity, Eq. new expression
// of Lorentz factor, Eq. density, Eq. T of h, Eq. p=rhoT).
template <class R, class S>
__device__ __forceinline__ void prims_from_htilde(S D, S Mx, S My, S Mz, R ht, PrimX<R>& W) {
  R h = R(1) + ht;
  R rDh = R(1) / (R(D) * h);
  W.u[0] = R(Mx) * rDh;
  W.u[1] = R(My) * rDh;
  W.u[2] = R(Mz) * rDh;
  R g2 = R(1) + (W.u[0] * W.u[0] + W.u[1] * W.u[1] + W.u[2] * W.u[2]);
  R rg = rsqrt_r(g2);
  W.gamma = g2 * rg;
  W.rg = rg;
  W.rho = R(D) * rg;
  W.T = T_of_htilde(ht);
  W.h = h;
  W.ht = ht;
  W.p = W.rho * W.T;
}

// prims_from_htilde of two float states with packed arithmetic.
__device__ __forceinline__ void prims_from_htilde_x2(const float (&Ua)[5], const float (&Ub)[5],
                                                     float ha, float hb, PrimX<float>& Wa,
                                                     PrimX<float>& Wb) {
  using namespace pk;
  const float2 ht = make_float2(ha, hb);
  const float2 D = make_float2(Ua[0], Ub[0]);
  const float2 h = add(ht, s2(1.f));
  const float2 Dh = mul(D, h);
  const float2 rDh = make_float2(1.0f / Dh.x, 1.0f / Dh.y);
  const float2 ux = mul(make_float2(Ua[1], Ub[1]), rDh);
  const float2 uy = mul(make_float2(Ua[2], Ub[2]), rDh);
  const float2 uz = mul(make_float2(Ua[3], Ub[3]), rDh);
  const float2 g2 = fma(uz, uz, fma(uy, uy, fma(ux, ux, s2(1.f))));
  const float2 rg = rsq(g2);
  const float2 gamma = mul(g2, rg);
  const float2 rho = mul(D, rg);
  // T of htilde (Eq. T of h)
  const float2 x = fma(fma(ht, s2(9.f), s2(18.f)), ht, s2(25.f));
  const float2 num = mul(fma(ht, s2(2.f), s2(4.f)), ht);
  const float2 den = add(fma(ht, s2(5.f), s2(5.f)), make_float2(sqrtf(x.x), sqrtf(x.y)));
  const float2 T = make_float2(qdiv(num.x, den.x), qdiv(num.y, den.y));
  const float2 p = mul(rho, T);
  Wa.rho = rho.x; Wa.u[0] = ux.x; Wa.u[1] = uy.x; Wa.u[2] = uz.x; Wa.p = p.x;
  Wa.T = T.x; Wa.h = h.x; Wa.gamma = gamma.x; Wa.rg = rg.x; Wa.ht = ha;
  Wb.rho = rho.y; Wb.u[0] = ux.y; Wb.u[1] = uy.y; Wb.u[2] = uz.y; Wb.p = p.y;
  Wb.T = T.y; Wb.h = h.y; Wb.gamma = gamma.y; Wb.rg = rg.y; Wb.ht = hb;
}

// Conserved -> primitive (Section 2.3). Returns 0 ok, 1 unphysical, 2 no
// convergence. Newton-Raphson on f(htilde) = A (monotone f), then
// Eq. (four-velocity), Eq. (new expression of Lorentz factor), Eq. (density),
// Eq. (T of h), Eq. (p=rhoT). A step that would make htilde non-positive
// halves htilde instead. Stops when |dh| <= tol htilde, or when the step no
// longer contracts at the rounding floor, or after maxit steps (status 2).
// guess > 0 starts the iteration there (a warm start from a nearby state);
// otherwise the Appendix A guess is used. The root does not depend on it.
template <class P>
__device__ __forceinline__ int con2pri(typename P::S D, typename P::S Mx, typename P::S My,
                                       typename P::S Mz, typename P::S Et,
                                       PrimX<typename P::S>& W, int maxit,
                                       typename P::S guess = typename P::S(0), int ori = 0) {
  using R = typename P::S;
  typename P::AT Aa, m2a;
  if (!A_and_m2<P>(D, Mx, My, Mz, Et, Aa, m2a, ori)) {
    R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
    W.rho = W.u[0] = W.u[1] = W.u[2] = W.p = W.T = W.h = W.gamma = W.rg = W.ht = nan;
    return 1;
  }
  const R A = R(Aa), m2 = R(m2a);
  R ht = guess > R(0) ? guess : newton_guess(A, m2);
  int status = 2;
  R prev = R(3.0e38);
  for (int k = 1; k <= maxit; ++k) {
    R T, dT, f, df;
    T_dT_of_htilde(ht, T, dT);
    f_df(ht, T, dT, m2, f, df);
    R dh = qdiv(f - A, df);
    R hn = ht - dh;
    if (!(hn > R(0))) hn = R(0.5) * ht;
    R adh = fabs(dh);
    ht = hn;
    if (adh <= NewtonCfg<R>::tol * ht) { status = 0; break; }
    if (k >= 3 && adh >= prev && adh <= NewtonCfg<R>::floor * ht) { status = 0; break; }
    prev = adh;
  }
  prims_from_htilde(D, Mx, My, Mz, ht, W);
  return status;
}

// Two conserved -> primitive conversions advanced in lockstep: the same
// Newton-Raphson iteration and stopping rule as con2pri, applied to two
// independent states so that their dependency chains interleave (the
// single solve is a chain of dependent square roots and divisions). The loop
// runs until both have stopped; a state that has stopped is not updated.
template <class P>
__device__ __forceinline__ void con2pri_x2(const typename P::S (&Ua)[5],
                                           const typename P::S (&Ub)[5],
                                           PrimX<typename P::S>& Wa, PrimX<typename P::S>& Wb,
                                           int maxit, int& sta, int& stb,
                                           typename P::S ga = typename P::S(0),
                                           typename P::S gb = typename P::S(0), int ori = 0) {
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
  R ha = ga > R(0) ? ga : newton_guess(Aa, m2a);
  R hb = gb > R(0) ? gb : newton_guess(Ab, m2b);
  bool da = false, db = false;
  sta = 2;
  stb = 2;
  R preva = R(3.0e38), prevb = R(3.0e38);
  for (int k = 1; k <= maxit && !(da && db); ++k) {
    R dha, dhb;
    if constexpr (sizeof(R) == 4) {
      float2 T, dT, f, df;
      const float2 h2 = make_float2(ha, hb);
      pk::T_dT_of_htilde(h2, T, dT);
      pk::f_df(h2, T, dT, make_float2(m2a, m2b), f, df);
      const float2 dh = pk::mul(pk::sub(f, make_float2(Aa, Ab)), pk::rcp(df));
      dha = dh.x;
      dhb = dh.y;
    } else {
      R Ta, dTa, fa, dfa, Tb, dTb, fb, dfb;
      T_dT_of_htilde(ha, Ta, dTa);
      T_dT_of_htilde(hb, Tb, dTb);
      f_df(ha, Ta, dTa, m2a, fa, dfa);
      f_df(hb, Tb, dTb, m2b, fb, dfb);
      dha = qdiv(fa - Aa, dfa);
      dhb = qdiv(fb - Ab, dfb);
    }
    if (!da) {
      R hn = ha - dha;
      if (!(hn > R(0))) hn = R(0.5) * ha;
      R adh = fabs(dha);
      ha = hn;
      if (adh <= NewtonCfg<R>::tol * ha ||
          (k >= 3 && adh >= preva && adh <= NewtonCfg<R>::floor * ha)) {
        da = true;
        sta = 0;
      }
      preva = adh;
    }
    if (!db) {
      R hn = hb - dhb;
      if (!(hn > R(0))) hn = R(0.5) * hb;
      R adh = fabs(dhb);
      hb = hn;
      if (adh <= NewtonCfg<R>::tol * hb ||
          (k >= 3 && adh >= prevb && adh <= NewtonCfg<R>::floor * hb)) {
        db = true;
        stb = 0;
      }
      prevb = adh;
    }
  }
  if constexpr (sizeof(R) == 4) {
    prims_from_htilde_x2(Ua, Ub, ha, hb, Wa, Wb);
  } else {
    prims_from_htilde(Ua[0], Ua[1], Ua[2], Ua[3], ha, Wa);
    prims_from_htilde(Ub[0], Ub[1], Ub[2], Ub[3], hb, Wb);
  }
  const R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
  if (!pa) {
    Wa.rho = Wa.u[0] = Wa.u[1] = Wa.u[2] = Wa.p = Wa.T = Wa.h = Wa.gamma = Wa.rg = Wa.ht = nan;
    sta = 1;
  }
  if (!pb) {
    Wb.rho = Wb.u[0] = Wb.u[1] = Wb.u[2] = Wb.p = Wb.T = Wb.h = Wb.gamma = Wb.rg = Wb.ht = nan;
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
template <class R> __device__ __forceinline__ bool prim2con(PrimX<R>& W, R U[5], int ori = 0) {
  if (!(W.rho > R(0)) || !(W.p > R(0))) {
    R nan = R(__longlong_as_double(0x7ff8000000000000ULL));
    for (int v = 0; v < 5; ++v) U[v] = nan;
    return false;
  }
  const R T = qdiv(W.p, W.rho);
  const R a = R(2.25) * T * T;
  const R t2 = qdiv(a, R(1) + sqrt(a + R(1)));  // htilde - 2.5 T
  const R ht = R(2.5) * T + t2;
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
    U[4] = D * (qdiv(u2, gamma + R(1)) + (R(1.5) * T + t2 + ht * u2) * rg);
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
template <int d>
__device__ __forceinline__ void prim2con_flux_x2(const float2 (&W)[5], float2 (&U)[5],
                                                 float2 (&F)[5], bool& okx, bool& oky,
                                                 int ori) {
  using namespace pk;
  okx = W[0].x > 0.0f && W[4].x > 0.0f;
  oky = W[0].y > 0.0f && W[4].y > 0.0f;
  const float2 T = mul(W[4], rcp(W[0]));
  const float2 a = mul(mul(s2(2.25f), T), T);
  const float2 sq = add(s2(1.f), make_float2(sqrtf(a.x + 1.0f), sqrtf(a.y + 1.0f)));
  const float2 t2 = mul(a, rcp(sq));                       // htilde - 2.5 T
  const float2 ht = fma(s2(2.5f), T, t2);
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
    U[4] = mul(D, fma(fma(ht, u2, fma(s2(1.5f), T, t2)), rg, k1));
  }
  const float2 v = mul(W[1 + d], rg);
  F[0] = mul(U[0], v);
  F[1] = mul(U[1], v);
  F[2] = mul(U[2], v);
  F[3] = mul(U[3], v);
  F[1 + d] = add(F[1 + d], W[4]);
  F[4] = ori ? U[1 + d] : mul(add(U[4], W[4]), v);
  const float nan = __int_as_float(0x7fc00000);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if (!okx) U[q].x = nan;
    if (!oky) U[q].y = nan;
  }
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
template <int d, class R>
__device__ __forceinline__ void char_speeds(const PrimX<R>& W, R& lm, R& lp) {
  R cs2 = cs2_of(W.T, W.h);
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
template <int d>
__device__ __forceinline__ void outer_parts_x2(const PrimX<float>& WL, const float UL[5],
                                               const PrimX<float>& WR, const float UR[5],
                                               float FL[5], float FR[5], float& lmL, float& lpL,
                                               float& lmR, float& lpR, int ori) {
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
  const float2 cnum = mul(T, fma(s2(-8.f), T, mul(s2(5.f), h)));
  const float2 cden = mul(mul(s2(3.f), h), sub(h, T));
  const float2 cs2 = make_float2(cnum.x / cden.x, cnum.y / cden.y);
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
template <int d, class R>
__device__ __forceinline__ int riemann(int solver, const PrimX<R>& WL, const R UL[5],
                                       const PrimX<R>& WR, const R UR[5], R F[5], int ori = 0) {
  R FL[5], FR[5];
  R lmL, lpL, lmR, lpR;
  if constexpr (sizeof(R) == 4) {
    outer_parts_x2<d>(WL, UL, WR, UR, FL, FR, lmL, lpL, lmR, lpR, ori);
  } else {
    phys_flux<d>(WL, UL, FL, ori);
    phys_flux<d>(WR, UR, FR, ori);
    char_speeds<d>(WL, lmL, lpL);
    char_speeds<d>(WR, lmR, lpR);
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

// Signal speed bound S_max of one cell (Section 3.2, Eqs. time_step_U_max
// and SMax; |U_x|+|U_y|+|U_z| and ndim gamma U_s).
template <class R> __device__ __forceinline__ R smax_of(const PrimX<R>& W, int ndim) {
  R cs2 = cs2_of(W.T, W.h);
  R omc = R(1) - cs2;
  R us = sqrt(qdiv(cs2, omc));      // U_s = c_s / sqrt(1 - c_s^2)
  R gs = rsqrt_r(omc);              // gamma_s = 1 / sqrt(1 - c_s^2)
  R su = fabs(W.u[0]) + fabs(W.u[1]) + fabs(W.u[2]);
  R umax = gs * su + R(ndim) * W.gamma * us;
  return umax * rsqrt_r(R(1) + umax * umax);
}

}  // namespace srhd
