// Oracle for the per-patch SRHD fluid update of Tseng, Schive & Chiueh,
// "GAMER-SR" (arXiv 2012.11130).
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, FP64 CPU restatement
// of the paper's method, written to check the CUDA library against. Only the
// test-suite, the smoke check and the benchmark's CPU-baseline leg may load
// it. The product path never calls it and shares no code with it.
//
// Units: c = m = k_B = 1 (Section 1 and the Appendix preamble). Primitive
// variables W = (rho, U^x, U^y, U^z, p) use the spatial four-velocity
// (Section 2.1, Eq. new expression of Lorentz factor); conserved variables
// U = (D, M^x, M^y, M^z, Etilde) use the reduced energy Etilde = E - D
// (Eq. ETilde). T below always means k_B T / m c^2 and htilde = h - 1.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (no FMA
// contraction, IEEE sqrt and division, round to nearest).
//
// Numerical kernels are templates over the real type R so that the same
// source can be instantiated with an operation-counting type (OpCount) to
// measure the algorithmic flop count of one cell update; the double
// instantiation is the oracle proper.
//
// Parity pins: every function here is checked by tests/test_oracle_*.py
// against closed forms, high-precision definitions, invariants and the
// exact-solution table of Appendix C (see the individual tests).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

// ----------------------------------------------------------------------------
// Operation-counting real type (used only to count algorithmic flops).
// ----------------------------------------------------------------------------
struct OpTally { uint64_t add = 0, mul = 0, div = 0, sqrt = 0; };
thread_local OpTally g_tally;

struct OpCount {
  double v;
  OpCount() : v(0.0) {}
  OpCount(double x) : v(x) {}  // NOLINT: implicit on purpose (constants)
};
inline OpCount operator+(OpCount a, OpCount b) { ++g_tally.add; return OpCount(a.v + b.v); }
inline OpCount operator-(OpCount a, OpCount b) { ++g_tally.add; return OpCount(a.v - b.v); }
inline OpCount operator*(OpCount a, OpCount b) { ++g_tally.mul; return OpCount(a.v * b.v); }
inline OpCount operator/(OpCount a, OpCount b) { ++g_tally.div; return OpCount(a.v / b.v); }
inline OpCount operator-(OpCount a) { return OpCount(-a.v); }
inline bool operator<(OpCount a, OpCount b) { return a.v < b.v; }
inline bool operator>(OpCount a, OpCount b) { return a.v > b.v; }
inline bool operator<=(OpCount a, OpCount b) { return a.v <= b.v; }
inline bool operator>=(OpCount a, OpCount b) { return a.v >= b.v; }
inline bool operator==(OpCount a, OpCount b) { return a.v == b.v; }
inline bool operator!=(OpCount a, OpCount b) { return a.v != b.v; }
inline OpCount sqrt(OpCount a) { ++g_tally.sqrt; return OpCount(std::sqrt(a.v)); }
inline OpCount fabs(OpCount a) { return OpCount(std::fabs(a.v)); }
inline double val(OpCount a) { return a.v; }
inline double val(double a) { return a; }
inline bool is_finite(OpCount a) { return std::isfinite(a.v); }
inline bool is_finite(double a) { return std::isfinite(a); }

using std::sqrt;
using std::fabs;

template <class R> inline R rmin(R a, R b) { return (b < a) ? b : a; }
template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }

// Status codes (shared meaning with the Python wrapper).
enum {
  OK = 0,
  UNPHYSICAL = 1,   // Eq. (Unphysical result) fails: A <= eps_machine
  NOCONV = 2,       // Newton-Raphson hit its iteration cap
  BADARG = 3,
};

constexpr double kEpsUnphysical = 2e-16;  // Section 3.3: eps_machine, double precision
constexpr int kNewtonMaxIter = 50;

// ----------------------------------------------------------------------------
// Equations of state (Section 2.2): Taub-Mathews (the paper's) or, selected by
// or_set_eos, the polytropic (constant-Gamma) EoS the paper keeps for pure
// non-relativistic or ultra-relativistic gas: h = 1 + Gamma/(Gamma-1) T.
// ----------------------------------------------------------------------------
struct EosSel { int gamma_law = 0; double gam = 5.0 / 3.0; };
thread_local EosSel g_eos;

// Eq. (T_to_HTilde): htilde(T) = 2.5 T + 2.25 T^2 / (1 + sqrt(2.25 T^2 + 1)),
// the TM enthalpy (Eq. TM EOS) minus one, written without a subtraction.
// Polytropic: htilde = Gamma/(Gamma-1) T.
template <class R> R htilde_of_T(R T) {
  if (g_eos.gamma_law) return R(g_eos.gam / (g_eos.gam - 1.0)) * T;
  R a = R(2.25) * T * T;
  return R(2.5) * T + a / (R(1.0) + sqrt(a + R(1.0)));
}

// Eq. (T of h): inverse of the TM EoS in terms of htilde (polytropic:
// T = (Gamma-1)/Gamma htilde).
template <class R> R T_of_htilde(R ht) {
  if (g_eos.gamma_law) return R((g_eos.gam - 1.0) / g_eos.gam) * ht;
  R num = R(2.0) * ht * ht + R(4.0) * ht;
  R den = R(5.0) * ht + R(5.0) + sqrt(R(9.0) * ht * ht + R(18.0) * ht + R(25.0));
  return num / den;
}

// Eq. (dT_dh), Appendix A: derivative of Eq. (T of h) (polytropic: constant).
template <class R> R dT_dhtilde(R ht) {
  if (g_eos.gamma_law) return R((g_eos.gam - 1.0) / g_eos.gam);
  R s = sqrt(R(9.0) * ht * ht + R(18.0) * ht + R(25.0));
  R den = R(5.0) * ht + R(5.0) + s;
  R num = R(2.0) * ht * ht + R(4.0) * ht;
  R t1 = (R(4.0) * ht + R(4.0)) / den;
  R t2 = num * ((R(9.0) * ht + R(9.0)) / s + R(5.0)) / (den * den);
  return t1 - t2;
}

// Eq. (sound_speed): squared TM sound speed c_s^2 as a function of T.
// Polytropic: c_s^2 = Gamma p / (rho h) = Gamma T / h.
template <class R> R cs2_of_T(R T) {
  R h = R(1.0) + htilde_of_T(T);
  if (g_eos.gamma_law) return R(g_eos.gam) * T / h;
  return (T / (R(3.0) * h)) * ((R(5.0) * h - R(8.0) * T) / (h - T));
}

// Eq. (transcendental equation), right-hand side:
// f(htilde) = htilde^2 + 2 htilde - 2 T (htilde+1) + T^2 (htilde+1)^2 / ((htilde+1)^2 + m^2)
// with T = T(htilde) supplied by the caller and m^2 = (|M|/D)^2.
template <class R> R f_of_htilde(R ht, R T, R m2) {
  R h = ht + R(1.0);
  R hh = h * h;
  return ht * ht + R(2.0) * ht - R(2.0) * T * h + T * T * hh / (hh + m2);
}

// Appendix A: df/dhtilde (first equation of the appendix).
template <class R> R df_dhtilde(R ht, R T, R dT, R m2) {
  R h = ht + R(1.0);
  R hh = h * h;
  R q = hh + m2;
  R num = R(2.0) * T * hh * hh * dT + R(2.0) * T * h * m2 * (h * dT + T);
  return R(2.0) * ht + R(2.0) - R(2.0) * T - R(2.0) * h * dT + num / (q * q);
}

// ----------------------------------------------------------------------------
// Primitive -> conserved (Section 2.3, Eqs. density, momentum, T_to_HTilde,
// E_D). W = (rho, Ux, Uy, Uz, p) -> U = (D, Mx, My, Mz, Etilde).
// ----------------------------------------------------------------------------
// ori = 1 selects the "original scheme" the paper compares against (its
// Sections 2.3 and 4): the fifth conserved variable is the total energy
// E = D h gamma - p (Eq. definition of reduced energy, first form) instead of
// Etilde, evolved with the flux M (Eq. E evoltion), and inverted from
// (E/D)^2 - (|M|/D)^2 - 1, which cancels catastrophically for cold gas.
template <class R> int prim2con(const R W[5], R U[5], int ori = 0) {
  R rho = W[0], ux = W[1], uy = W[2], uz = W[3], p = W[4];
  if (!(val(rho) > 0.0) || !(val(p) > 0.0)) return UNPHYSICAL;
  R T = p / rho;
  R ht = htilde_of_T(T);
  R u2 = ux * ux + uy * uy + uz * uz;
  R gamma = sqrt(R(1.0) + u2);       // Eq. (new expression of Lorentz factor)
  R D = rho * gamma;                  // Eq. (density)
  R h = R(1.0) + ht;
  R Dh = D * h;
  U[0] = D;
  U[1] = Dh * ux;                     // Eq. (momentum)
  U[2] = Dh * uy;
  U[3] = Dh * uz;
  if (ori) {
    U[4] = Dh * gamma - p;            // E = D h gamma - p
    return OK;
  }
  R m2 = h * h * u2;                  // (|M|/D)^2
  R f = f_of_htilde(ht, T, m2);
  R s = m2 + f;
  U[4] = D * (s / (R(1.0) + sqrt(R(1.0) + s)));  // Eq. (E_D)
  return OK;
}

// Left-hand side of Eq. (transcendental equation) and of Eq. (Unphysical
// result): A = (Et/D)^2 + 2 (Et/D) - (|M|/D)^2, evaluated as
// eD*(eD+2) - m2 with eD = Et/D and m2 = (Mx^2+My^2+Mz^2)/D^2.
template <class R> R A_of_cons(const R U[5], R* m2_out, int ori = 0) {
  R D = U[0];
  R M2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  R m2 = M2 / (D * D);
  R eD = U[4] / D;
  *m2_out = m2;
  if (ori) return (eD * eD - m2) - R(1.0);   // (E/D)^2 - (|M|/D)^2 - 1
  return eD * (eD + R(2.0)) - m2;
}

// Appendix A: initial guess of htilde for the Newton-Raphson iteration.
// Hot gas (A above the threshold of Eq. ColdHot): Eq. (guess for hot fluid).
// Cold gas: the positive root of the quadratic of Eq. (cold limit of
// transcendental eq), 6/5 h + (43/125 + 4/(25 (1+m^2))) h^2 = A, written in
// the cancellation-free form h = 2A / (6/5 + sqrt(36/25 + 4 a A)) with
// a = (43 m^2 + 63) / (125 (1 + m^2)). (The closed form printed as
// Eq. (guess for cold fluid) does not solve its own quadratic; the root of
// the quadratic is used instead. Its crossing with the hot guess is exactly
// the threshold of Eq. ColdHot, which confirms this reading.)
template <class R> R newton_guess(R A, R m2) {
  if (g_eos.gamma_law) {
    // Polytropic EoS: the root for m = 0, where f = ((1-k) htilde + 1)^2 - 1
    // with k = (Gamma-1)/Gamma, i.e. htilde = A / ((1-k)(1 + sqrt(1 + A))).
    R omk = R(1.0 / g_eos.gam);
    return A / (omk * (R(1.0) + sqrt(R(1.0) + A)));
  }
  R P = R(1.0) + m2;
  R thr_base = R(1800.0) * P / (R(437.0) * m2 + R(117.0));
  R thr = thr_base * thr_base;
  if (A > thr) return R(4.0) / R(3.0) * sqrt(A);
  R a = (R(43.0) * m2 + R(63.0)) / (R(125.0) * P);
  return R(2.0) * A / (R(1.2) + sqrt(R(1.44) + R(4.0) * a * A));
}

struct Con2PriInfo { int iters; double htilde; double A; };

// Conserved -> primitive (Section 2.3): solve f(htilde) = A by Newton-Raphson
// (f is monotonically increasing), then Eq. (four-velocity), Eq. (new
// expression of Lorentz factor), Eq. (density), Eq. (T of h), Eq. (p=rhoT).
// Stopping rule (the paper is silent): stop when |dh| <= 2^-50 htilde, or when
// the step stops contracting at the rounding floor (|dh| >= |dh_prev| with
// |dh| <= 1e-12 htilde); otherwise NOCONV after kNewtonMaxIter steps. A step
// that would make htilde non-positive is replaced by halving htilde.
template <class R> int con2pri(const R U[5], R W[5], R* ht_out, Con2PriInfo* info, int ori = 0) {
  R D = U[0];
  if (!(val(D) > 0.0) || !is_finite(U[4])) {
    for (int v = 0; v < 5; ++v) W[v] = R(NAN);
    if (info) { info->iters = 0; info->htilde = NAN; info->A = NAN; }
    return UNPHYSICAL;
  }
  R m2;
  R A = A_of_cons(U, &m2, ori);
  if (info) { info->A = val(A); info->iters = 0; }
  if (!(val(A) > kEpsUnphysical)) {      // Eq. (Unphysical result)
    for (int v = 0; v < 5; ++v) W[v] = R(NAN);
    if (info) info->htilde = NAN;
    return UNPHYSICAL;
  }
  R ht = newton_guess(A, m2);
  int status = NOCONV;
  double prev = INFINITY;
  int k = 0;
  for (k = 1; k <= kNewtonMaxIter; ++k) {
    R T = T_of_htilde(ht);
    R dT = dT_dhtilde(ht);
    R fval = f_of_htilde(ht, T, m2) - A;
    R df = df_dhtilde(ht, T, dT, m2);
    R dh = fval / df;
    R ht_new = ht - dh;
    if (!(val(ht_new) > 0.0)) ht_new = ht * R(0.5);
    double adh = std::fabs(val(dh));
    ht = ht_new;
    if (adh <= std::ldexp(1.0, -50) * val(ht)) { status = OK; break; }
    if (k >= 3 && adh >= prev && adh <= 1e-12 * val(ht)) { status = OK; break; }
    prev = adh;
  }
  if (info) { info->iters = (k > kNewtonMaxIter) ? kNewtonMaxIter : k; info->htilde = val(ht); }
  R h = R(1.0) + ht;
  R Dh = D * h;
  R ux = U[1] / Dh, uy = U[2] / Dh, uz = U[3] / Dh;   // Eq. (four-velocity)
  R gamma = sqrt(R(1.0) + (ux * ux + uy * uy + uz * uz));
  R rho = D / gamma;
  R T = T_of_htilde(ht);
  W[0] = rho; W[1] = ux; W[2] = uy; W[3] = uz;
  W[4] = rho * T;                                      // Eq. (p=rhoT)
  if (ht_out) *ht_out = ht;
  return status;
}

// Reference root by bisection on f(htilde) = A (brute force check of the
// Newton solve): bracket [0, hi] with f(hi) >= A, bisect to one ulp.
double htilde_bisect(double A, double m2) {
  double lo = 0.0, hi = 1.0;
  while (f_of_htilde(hi, T_of_htilde(hi), m2) < A) hi *= 2.0;
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (f_of_htilde(mid, T_of_htilde(mid), m2) < A) lo = mid; else hi = mid;
  }
  double flo = std::fabs(f_of_htilde(lo, T_of_htilde(lo), m2) - A);
  double fhi = std::fabs(f_of_htilde(hi, T_of_htilde(hi), m2) - A);
  return flo <= fhi ? lo : hi;
}

// ----------------------------------------------------------------------------
// Numerical scheme (Section 3.1: PLM, MUSCL-Hancock, HLLC/HLLE)
// ----------------------------------------------------------------------------

struct Params {
  double theta;          // minmod coefficient of the limiter (Section 3.3)
  double retry_factor;   // 0.75 (Section 3.3, SRHD solver)
  double theta_floor;    // relative floor below which theta is set to 0
  int riemann;           // 0 = HLLC, 1 = HLLE
  int ndim;              // active dimensions for the CFL bound
  double cfl;            // C_CFL (Eq. time_step_sound_speed)
  int cfl_mode;          // 0 = signal speed (Eq. SMax), 1 = speed of light
  int ori;               // 1 = original scheme (total energy E, flux M)
};

// Hybrid van Leer / generalised minmod slope limiter (Section 4.2 names it;
// the formula is the standard pair): zero at extrema; otherwise the smaller
// in magnitude of the van Leer slope 2 dl dr / (dl + dr) and the generalised
// minmod slope minmod(theta dl, theta dr, (dl + dr)/2).
template <class R> R limited_slope(R dl, R dr, R theta) {
  if (!(val(dl * dr) > 0.0)) return R(0.0);
  R vl = R(2.0) * dl * dr / (dl + dr);
  R adl = fabs(dl), adr = fabs(dr);
  R gm = rmin(rmin(theta * adl, theta * adr), R(0.5) * fabs(dl + dr));
  R mag = rmin(fabs(vl), gm);
  return (val(dl) > 0.0) ? mag : -mag;
}

// Physical flux in direction d (Eqs. D evolution, M evolution, ETilde
// evolution): F = (D v, M v + p e_d, (Etilde + p) v), v = U^d / gamma.
template <class R> void phys_flux(int d, const R W[5], const R U[5], R F[5], int ori = 0) {
  R u2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  R gamma = sqrt(R(1.0) + u2);
  R v = W[1 + d] / gamma;
  F[0] = U[0] * v;
  F[1] = U[1] * v;
  F[2] = U[2] * v;
  F[3] = U[3] * v;
  F[1 + d] = F[1 + d] + W[4];
  F[4] = ori ? U[1 + d] : (U[4] + W[4]) * v;   // flux of E is M_d (Eq. E evoltion)
}

// Relativistic characteristic speeds lambda_-/+ along direction d with the TM
// sound speed (Eq. sound_speed), written with four-velocities to avoid the
// 1 - v^2 cancellation: lambda = [gamma U_d (1-cs2) -/+ cs sqrt(1 + U_perp^2
// (1-cs2))] / [1 + U^2 (1-cs2)].
template <class R> void char_speeds(int d, const R W[5], R* lm, R* lp) {
  R ud = W[1 + d];
  R up2 = R(0.0);
  for (int k = 0; k < 3; ++k) if (k != d) up2 = up2 + W[1 + k] * W[1 + k];
  R u2 = up2 + ud * ud;
  R gamma = sqrt(R(1.0) + u2);
  R T = W[4] / W[0];
  R cs2 = cs2_of_T(T);
  R omc = R(1.0) - cs2;
  R den = R(1.0) + u2 * omc;
  R a = gamma * ud * omc;
  R b = sqrt(cs2) * sqrt(R(1.0) + up2 * omc);
  *lm = (a - b) / den;
  *lp = (a + b) / den;
}

// Riemann flux across a face normal to d (Section 3.1: relativistic HLLC of
// Mignone & Bodo 2005, HLLE as an option and as the fallback when the
// contact state is not admissible). Inside the solver the total energy is
// E = Etilde + D; the reduced-energy flux is the total-energy flux minus the
// mass flux, which for every state used here equals (Etilde + p) v.
// Returns 1 if HLLC fell back to HLLE, else 0.
template <class R> int riemann_flux(int d, int solver, const R WL[5], const R UL[5],
                                    const R WR[5], const R UR[5], R F[5], int ori = 0) {
  R FL[5], FR[5];
  phys_flux(d, WL, UL, FL, ori);
  phys_flux(d, WR, UR, FR, ori);
  R lmL, lpL, lmR, lpR;
  char_speeds(d, WL, &lmL, &lpL);
  char_speeds(d, WR, &lmR, &lpR);
  R sL = rmin(lmL, lmR);
  R sR = rmax(lpL, lpR);
  if (val(sL) >= 0.0) { for (int v = 0; v < 5; ++v) F[v] = FL[v]; return 0; }
  if (val(sR) <= 0.0) { for (int v = 0; v < 5; ++v) F[v] = FR[v]; return 0; }
  R ds = sR - sL;
  R Uhll[5], Fhll[5];
  for (int v = 0; v < 5; ++v) {
    Uhll[v] = (sR * UR[v] - sL * UL[v] - FR[v] + FL[v]) / ds;
    Fhll[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) / ds;
  }
  int fallback = 0;
  if (solver == 0) {
    // Contact speed: smaller root of FE lam^2 - (E + Fm) lam + m = 0 on the
    // HLL state (total energy), in the cancellation-free form.
    R E = ori ? Uhll[4] : Uhll[4] + Uhll[0];
    R FE = ori ? Fhll[4] : Fhll[4] + Fhll[0];
    R m = Uhll[1 + d];
    R Fm = Fhll[1 + d];
    R B = E + Fm;
    R disc = B * B - R(4.0) * FE * m;
    bool ok = val(disc) >= 0.0 && val(B) > 0.0;
    R lam = R(0.0), ps = R(0.0);
    if (ok) {
      lam = R(2.0) * m / (B + sqrt(disc));
      ps = Fm - lam * FE;
      ok = val(lam) > val(sL) && val(lam) < val(sR) && val(ps) > 0.0 && is_finite(lam);
    }
    if (ok) {
      const R* Wk = (val(lam) >= 0.0) ? WL : WR;
      const R* Uk = (val(lam) >= 0.0) ? UL : UR;
      const R* Fk = (val(lam) >= 0.0) ? FL : FR;
      R sk = (val(lam) >= 0.0) ? sL : sR;
      R u2 = Wk[1] * Wk[1] + Wk[2] * Wk[2] + Wk[3] * Wk[3];
      R gamma = sqrt(R(1.0) + u2);
      R v = Wk[1 + d] / gamma;
      R p = Wk[4];
      R a = sk - v;
      R b = sk - lam;
      R Us[5];
      Us[0] = Uk[0] * a / b;
      for (int k = 0; k < 3; ++k) Us[1 + k] = Uk[1 + k] * a / b;
      Us[1 + d] = (Uk[1 + d] * a + ps - p) / b;
      Us[4] = (Uk[4] * a + ps * lam - p * v) / b;
      for (int v5 = 0; v5 < 5; ++v5) F[v5] = Fk[v5] + sk * (Us[v5] - Uk[v5]);
      return 0;
    }
    fallback = 1;
  }
  for (int v = 0; v < 5; ++v) F[v] = Fhll[v];
  return fallback;
}

// Signal-speed CFL bound of one cell (Section 3.2, Eqs. time_step_U_max and
// SMax, with |U_x|+|U_y|+|U_z| for the misprinted sum and ndim gamma U_s for
// runs with fewer active dimensions). Returns S_max.
template <class R> R smax_of_prim(const R W[5], int ndim) {
  R T = W[4] / W[0];
  R cs2 = cs2_of_T(T);
  R us = sqrt(cs2 / (R(1.0) - cs2));       // U_s = c_s / sqrt(1 - c_s^2)
  R gs = sqrt(R(1.0) + us * us);           // gamma_s
  R u2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  R gamma = sqrt(R(1.0) + u2);
  R su = fabs(W[1]) + fabs(W[2]) + fabs(W[3]);
  R umax = gs * su + R(double(ndim)) * gamma * us;
  return umax / sqrt(R(1.0) + umax * umax);
}

// ----------------------------------------------------------------------------
// One MUSCL-Hancock step of a block with given ghost zones (Sections 3.1-3.3).
// Layout: cons_in [5][Nz][Ny][Nx], N_d = n_d + 2 g_d with g_d = 2 on active
// dimensions and 0 otherwise; cons_out [5][nz][ny][nx].
// The block is the retry unit of Section 3.3 (1): if any predicted face
// state or any updated cell is unphysical, the whole block is recomputed with
// the limiter coefficient reduced by retry_factor, until it passes; once the
// coefficient drops below theta_floor * theta the last attempt uses theta = 0
// (piecewise-constant reconstruction).
// ----------------------------------------------------------------------------
template <class R> struct Block {
  int n[3], g[3], N[3], act[3];
  int ori;                     // original scheme (total energy)
  std::vector<R> W;            // prims [5][Ncells]
  std::vector<int8_t> Wstat;   // -1 not computed, else con2pri status
  std::vector<R> face;         // predicted face cons [Ncells][3][2][5]
  std::vector<int8_t> fstat;   // -1 not computed, 0 ok, 1 unphysical
  const R* in;
  int ncell() const { return N[0] * N[1] * N[2]; }
  int idx(int i, int j, int k) const {
    return ((k + g[2]) * N[1] + (j + g[1])) * N[0] + (i + g[0]);
  }
};

template <class R> int block_prim(Block<R>& B, int i, int j, int k, R out[5]) {
  int c = B.idx(i, j, k);
  int nc = B.ncell();
  if (B.Wstat[c] < 0) {
    R U[5], W[5];
    for (int v = 0; v < 5; ++v) U[v] = B.in[v * nc + c];
    int st = con2pri(U, W, (R*)nullptr, (Con2PriInfo*)nullptr, B.ori);
    for (int v = 0; v < 5; ++v) B.W[v * nc + c] = W[v];
    B.Wstat[c] = (int8_t)st;
  }
  for (int v = 0; v < 5; ++v) out[v] = B.W[v * nc + c];
  return B.Wstat[c];
}

// Predicted (half-step) face states of one cell, all six faces at once:
// PLM slopes in every active direction from the cell's primitive neighbours,
// face values W -/+ dW/2, their conserved form and physical fluxes, then the
// Hancock half step U_face - dt/(2 dh) sum_d [F_d(W_d+) - F_d(W_d-)].
template <class R> int block_faces(Block<R>& B, int i, int j, int k, R theta, R dt, R dh) {
  int c = B.idx(i, j, k);
  if (B.fstat[c] >= 0) return B.fstat[c];
  R W[5];
  int st = block_prim(B, i, j, k, W);
  if (st == UNPHYSICAL) { B.fstat[c] = 2; return 2; }
  R Wf[3][2][5], Uf[3][2][5], Ff[3][2][5];
  int bad = 0;
  for (int d = 0; d < 3; ++d) {
    if (!B.act[d]) continue;
    int e[3] = {0, 0, 0};
    e[d] = 1;
    R Wm[5], Wp[5];
    int s1 = block_prim(B, i - e[0], j - e[1], k - e[2], Wm);
    int s2 = block_prim(B, i + e[0], j + e[1], k + e[2], Wp);
    if (s1 == UNPHYSICAL || s2 == UNPHYSICAL) { B.fstat[c] = 2; return 2; }
    for (int v = 0; v < 5; ++v) {
      R dW = limited_slope(W[v] - Wm[v], Wp[v] - W[v], theta);
      Wf[d][0][v] = W[v] - R(0.5) * dW;
      Wf[d][1][v] = W[v] + R(0.5) * dW;
    }
    for (int s = 0; s < 2; ++s) {
      if (prim2con(Wf[d][s], Uf[d][s], B.ori) != OK) bad = 1;
      phys_flux(d, Wf[d][s], Uf[d][s], Ff[d][s], B.ori);
    }
  }
  R dF[5];
  for (int v = 0; v < 5; ++v) {
    dF[v] = R(0.0);
    for (int d = 0; d < 3; ++d)
      if (B.act[d]) dF[v] = dF[v] + (Ff[d][1][v] - Ff[d][0][v]);
  }
  R half = R(0.5) * dt / dh;
  for (int d = 0; d < 3; ++d) {
    if (!B.act[d]) continue;
    for (int s = 0; s < 2; ++s)
      for (int v = 0; v < 5; ++v)
        B.face[((size_t)c * 6 + d * 2 + s) * 5 + v] = Uf[d][s][v] - half * dF[v];
  }
  B.fstat[c] = (int8_t)(bad ? 1 : 0);
  return B.fstat[c];
}

// Status codes of a block advance.
enum { BLK_OK = 0, BLK_UNPHYSICAL = 1, BLK_BAD_INPUT = 2, BLK_NOCONV = 4 };

template <class R>
int advance_block(const R* in, R* out, R* flux_out, const int n[3], const int act[3],
                  R dt, R dh, const Params& P, int* retries_out) {
  Block<R> B;
  for (int d = 0; d < 3; ++d) {
    B.n[d] = n[d];
    B.act[d] = act[d];
    B.g[d] = act[d] ? 2 : 0;
    B.N[d] = n[d] + 2 * B.g[d];
  }
  B.in = in;
  B.ori = P.ori;
  int nc = B.ncell();
  B.W.assign((size_t)5 * nc, R(0.0));
  B.Wstat.assign(nc, -1);
  B.face.assign((size_t)nc * 30, R(0.0));
  const int nint = n[0] * n[1] * n[2];
  // Face flux storage: for direction d, faces (n_d+1) along d times the
  // interior extent of the other two directions, [3][5][nface_d].
  int nf[3];
  for (int d = 0; d < 3; ++d) nf[d] = act[d] ? (n[0] * n[1] * n[2] / n[d]) * (n[d] + 1) : 0;
  std::vector<R> Fd[3];
  for (int d = 0; d < 3; ++d) Fd[d].assign((size_t)5 * nf[d], R(0.0));

  double theta0 = P.theta;
  double theta = theta0;
  int attempt = 0;
  int result = BLK_OK;
  int noconv = 0;
  for (;;) {
    B.fstat.assign(nc, -1);
    int fail = 0;
    int badin = 0;
    // Fluxes at every face adjacent to an interior cell.
    for (int d = 0; d < 3 && !fail; ++d) {
      if (!act[d]) continue;
      int ext[3] = {n[0], n[1], n[2]};
      ext[d] = n[d] + 1;
      for (int kk = 0; kk < ext[2] && !fail; ++kk)
        for (int jj = 0; jj < ext[1] && !fail; ++jj)
          for (int ii = 0; ii < ext[0] && !fail; ++ii) {
            // face between cell (ii,jj,kk) - e_d (left) and (ii,jj,kk) (right)
            int e[3] = {0, 0, 0};
            e[d] = 1;
            int sl = block_faces(B, ii - e[0], jj - e[1], kk - e[2], R(theta), dt, dh);
            int sr = block_faces(B, ii, jj, kk, R(theta), dt, dh);
            if (sl == 2 || sr == 2) { badin = 1; fail = 1; break; }
            if (sl != 0 || sr != 0) { fail = 1; break; }
            int cl = B.idx(ii - e[0], jj - e[1], kk - e[2]);
            int cr = B.idx(ii, jj, kk);
            R UL[5], UR[5], WL[5], WR[5];
            for (int v = 0; v < 5; ++v) {
              UL[v] = B.face[((size_t)cl * 6 + d * 2 + 1) * 5 + v];
              UR[v] = B.face[((size_t)cr * 6 + d * 2 + 0) * 5 + v];
            }
            int a = con2pri(UL, WL, (R*)nullptr, (Con2PriInfo*)nullptr, P.ori);
            int b = con2pri(UR, WR, (R*)nullptr, (Con2PriInfo*)nullptr, P.ori);
            if (a == UNPHYSICAL || b == UNPHYSICAL) { fail = 1; break; }
            if (a == NOCONV || b == NOCONV) noconv = 1;
            R F[5];
            riemann_flux(d, P.riemann, WL, UL, WR, UR, F, P.ori);
            int fi = (kk * ext[1] + jj) * ext[0] + ii;
            for (int v = 0; v < 5; ++v) Fd[d][(size_t)v * nf[d] + fi] = F[v];
          }
    }
    if (badin) { result = BLK_BAD_INPUT; break; }
    if (!fail) {
      // Conservative update (Eq. conservative form) and the unphysical check
      // of Eq. (Unphysical result) on every updated cell.
      R coef = dt / dh;
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            R div[5];
            for (int v = 0; v < 5; ++v) div[v] = R(0.0);
            for (int d = 0; d < 3; ++d) {
              if (!act[d]) continue;
              int ext[3] = {n[0], n[1], n[2]};
              ext[d] = n[d] + 1;
              int p0[3] = {i, j, k};
              int p1[3] = {i, j, k};
              p1[d] += 1;
              int f0 = (p0[2] * ext[1] + p0[1]) * ext[0] + p0[0];
              int f1 = (p1[2] * ext[1] + p1[1]) * ext[0] + p1[0];
              for (int v = 0; v < 5; ++v)
                div[v] = div[v] + (Fd[d][(size_t)v * nf[d] + f1] - Fd[d][(size_t)v * nf[d] + f0]);
            }
            int c = B.idx(i, j, k);
            int o = (k * n[1] + j) * n[0] + i;
            R Un[5];
            for (int v = 0; v < 5; ++v) {
              Un[v] = in[(size_t)v * nc + c] - coef * div[v];
              out[(size_t)v * nint + o] = Un[v];
            }
            R m2;
            R A = A_of_cons(Un, &m2, P.ori);
            if (!(val(Un[0]) > 0.0) || !(val(A) > kEpsUnphysical)) fail = 1;
          }
    }
    if (!fail) break;
    if (theta == 0.0) { result = BLK_UNPHYSICAL; break; }
    ++attempt;
    theta = theta * P.retry_factor;
    if (theta < P.theta_floor * theta0) theta = 0.0;
  }
  if (retries_out) *retries_out = attempt;
  if (flux_out) {
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
      for (size_t q = 0; q < (size_t)5 * nf[d]; ++q) flux_out[off + q] = Fd[d][q];
      off += (size_t)5 * nf[d];
    }
  }
  if (result == BLK_OK && noconv) result = BLK_NOCONV;
  return result;
}


// ----------------------------------------------------------------------------
// VL integrator (Section 3.1: "MUSCL-Hancock and VL"; van Leer 2006, Falle
// 1991): a predictor-corrector step.
//   predictor  U*(c) = U^n(c) - dt/(2 dh) sum_d [F1(c, c+e_d) - F1(c-e_d, c)]
//              with F1 the Riemann flux between the piecewise-constant cell
//              states (first order, unsplit), then W* = con2pri(U*);
//   corrector  PLM slopes of W* (the limiter with coefficient theta), face
//              states W* -/+ dW/2 (no Hancock evolution), their conserved
//              form, the Riemann flux, and
//              U^{n+1} = U^n - dt/dh sum_d [F(face+) - F(face-)].
// The corrector's PLM stencil reaches two cells beyond the face and the
// predictor one more, so the block carries 3 ghost cells per active side.
// The limiter retry (Section 3.3) redoes the corrector with a smaller theta;
// the predictor does not depend on theta. If a predicted state is
// unphysical the corrector cannot run: the block returns BLK_UNPHYSICAL with
// NaN outputs.
// ----------------------------------------------------------------------------
template <class R> struct VlBlock {
  int n[3], g[3], N[3], act[3];
  int ori, riemann;
  R dt, dh;
  const R* in;
  std::vector<R> W;          // W^n [5][Ncells]
  std::vector<int8_t> Wst;   // -1 not computed, else con2pri status
  std::vector<R> Wh;         // W* [5][Ncells]
  std::vector<int8_t> Whst;  // -1 not computed, else status (1 = unphysical)
  int ncell() const { return N[0] * N[1] * N[2]; }
  int idx(int i, int j, int k) const {
    return ((k + g[2]) * N[1] + (j + g[1])) * N[0] + (i + g[0]);
  }
};

template <class R> int vl_prim_n(VlBlock<R>& B, int c, R W[5]) {
  const int nc = B.ncell();
  if (B.Wst[c] < 0) {
    R U[5], Wc[5];
    for (int v = 0; v < 5; ++v) U[v] = B.in[(size_t)v * nc + c];
    B.Wst[c] = (int8_t)con2pri(U, Wc, (R*)nullptr, (Con2PriInfo*)nullptr, B.ori);
    for (int v = 0; v < 5; ++v) B.W[(size_t)v * nc + c] = Wc[v];
  }
  for (int v = 0; v < 5; ++v) W[v] = B.W[(size_t)v * nc + c];
  return B.Wst[c];
}

// Predicted primitive state W* of cell (i,j,k); returns 0 ok, 1 unphysical
// predicted state, 2 unphysical input in its stencil.
template <class R> int vl_half(VlBlock<R>& B, int i, int j, int k, R out[5]) {
  const int nc = B.ncell();
  const int c = B.idx(i, j, k);
  if (B.Whst[c] < 0) {
    R Wc[5], Uc[5];
    int st = vl_prim_n(B, c, Wc);
    for (int v = 0; v < 5; ++v) Uc[v] = B.in[(size_t)v * nc + c];
    R div[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
    for (int d = 0; d < 3 && st != UNPHYSICAL; ++d) {
      if (!B.act[d]) continue;
      int e[3] = {0, 0, 0};
      e[d] = 1;
      const int cm = B.idx(i - e[0], j - e[1], k - e[2]);
      const int cp = B.idx(i + e[0], j + e[1], k + e[2]);
      R Wm[5], Wp[5], Um[5], Up[5], Fm[5], Fp[5];
      int sm = vl_prim_n(B, cm, Wm), sp = vl_prim_n(B, cp, Wp);
      if (sm == UNPHYSICAL || sp == UNPHYSICAL) { st = UNPHYSICAL; break; }
      for (int v = 0; v < 5; ++v) {
        Um[v] = B.in[(size_t)v * nc + cm];
        Up[v] = B.in[(size_t)v * nc + cp];
      }
      riemann_flux(d, B.riemann, Wm, Um, Wc, Uc, Fm, B.ori);
      riemann_flux(d, B.riemann, Wc, Uc, Wp, Up, Fp, B.ori);
      for (int v = 0; v < 5; ++v) div[v] = div[v] + (Fp[v] - Fm[v]);
    }
    if (st == UNPHYSICAL) {
      B.Whst[c] = 2;
    } else {
      R half = R(0.5) * B.dt / B.dh;
      R Uh[5], Wh[5];
      for (int v = 0; v < 5; ++v) Uh[v] = Uc[v] - half * div[v];
      int s2 = con2pri(Uh, Wh, (R*)nullptr, (Con2PriInfo*)nullptr, B.ori);
      B.Whst[c] = (int8_t)(s2 == UNPHYSICAL ? 1 : 0);
      for (int v = 0; v < 5; ++v) B.Wh[(size_t)v * nc + c] = Wh[v];
    }
  }
  for (int v = 0; v < 5; ++v) out[v] = B.Wh[(size_t)v * nc + c];
  return B.Whst[c];
}

template <class R>
int advance_block_vl(const R* in, R* out, R* flux_out, const int n[3], const int act[3], R dt,
                     R dh, const Params& P, int* retries_out) {
  VlBlock<R> B;
  for (int d = 0; d < 3; ++d) {
    B.n[d] = n[d];
    B.act[d] = act[d];
    B.g[d] = act[d] ? 3 : 0;
    B.N[d] = n[d] + 2 * B.g[d];
  }
  B.in = in;
  B.ori = P.ori;
  B.riemann = P.riemann;
  B.dt = dt;
  B.dh = dh;
  const int nc = B.ncell();
  B.W.assign((size_t)5 * nc, R(0.0));
  B.Wst.assign(nc, -1);
  B.Wh.assign((size_t)5 * nc, R(0.0));
  B.Whst.assign(nc, -1);
  const int nint = n[0] * n[1] * n[2];
  int nf[3];
  for (int d = 0; d < 3; ++d) nf[d] = act[d] ? (nint / n[d]) * (n[d] + 1) : 0;
  std::vector<R> Fd[3];
  for (int d = 0; d < 3; ++d) Fd[d].assign((size_t)5 * nf[d], R(0.0));
  const double theta0 = P.theta;
  double theta = theta0;
  int attempt = 0;
  int result = BLK_OK;
  int predicted_bad = 0, badin = 0;
  for (;;) {
    int fail = 0;
    for (int d = 0; d < 3 && !fail && !predicted_bad && !badin; ++d) {
      if (!act[d]) continue;
      int ext[3] = {n[0], n[1], n[2]};
      ext[d] = n[d] + 1;
      int e[3] = {0, 0, 0};
      e[d] = 1;
      for (int kk = 0; kk < ext[2] && !fail && !predicted_bad && !badin; ++kk)
        for (int jj = 0; jj < ext[1] && !fail && !predicted_bad && !badin; ++jj)
          for (int ii = 0; ii < ext[0]; ++ii) {
            // face between cl = (ii,jj,kk) - e_d and cr = (ii,jj,kk)
            const int il = ii - e[0], jl = jj - e[1], kl = kk - e[2];
            R Wl[5], Wll[5], Wr[5], Wrr[5], Wlm[5], Wrp[5];
            int s[4];
            s[0] = vl_half(B, il - e[0], jl - e[1], kl - e[2], Wll);
            s[1] = vl_half(B, il, jl, kl, Wl);
            s[2] = vl_half(B, ii, jj, kk, Wr);
            s[3] = vl_half(B, ii + e[0], jj + e[1], kk + e[2], Wrr);
            if (s[0] == 2 || s[1] == 2 || s[2] == 2 || s[3] == 2) { badin = 1; break; }
            if (s[0] || s[1] || s[2] || s[3]) { predicted_bad = 1; break; }
            for (int v = 0; v < 5; ++v) {
              R dWl = limited_slope(Wl[v] - Wll[v], Wr[v] - Wl[v], R(theta));
              R dWr = limited_slope(Wr[v] - Wl[v], Wrr[v] - Wr[v], R(theta));
              Wlm[v] = Wl[v] + R(0.5) * dWl;   // left state: + face of cl
              Wrp[v] = Wr[v] - R(0.5) * dWr;   // right state: - face of cr
            }
            R UL[5], UR[5], F[5];
            if (prim2con(Wlm, UL, B.ori) != OK || prim2con(Wrp, UR, B.ori) != OK) {
              fail = 1;
              break;
            }
            riemann_flux(d, P.riemann, Wlm, UL, Wrp, UR, F, B.ori);
            const int fi = (kk * ext[1] + jj) * ext[0] + ii;
            for (int v = 0; v < 5; ++v) Fd[d][(size_t)v * nf[d] + fi] = F[v];
          }
    }
    if (badin) { result = BLK_BAD_INPUT; break; }
    if (predicted_bad) { result = BLK_UNPHYSICAL; break; }
    if (!fail) {
      R coef = dt / dh;
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            R div[5];
            for (int v = 0; v < 5; ++v) div[v] = R(0.0);
            for (int d = 0; d < 3; ++d) {
              if (!act[d]) continue;
              int ext[3] = {n[0], n[1], n[2]};
              ext[d] = n[d] + 1;
              int p0[3] = {i, j, k};
              int p1[3] = {i, j, k};
              p1[d] += 1;
              int f0 = (p0[2] * ext[1] + p0[1]) * ext[0] + p0[0];
              int f1 = (p1[2] * ext[1] + p1[1]) * ext[0] + p1[0];
              for (int v = 0; v < 5; ++v)
                div[v] = div[v] + (Fd[d][(size_t)v * nf[d] + f1] - Fd[d][(size_t)v * nf[d] + f0]);
            }
            const int c = B.idx(i, j, k);
            const int o = (k * n[1] + j) * n[0] + i;
            R Un[5];
            for (int v = 0; v < 5; ++v) {
              Un[v] = in[(size_t)v * nc + c] - coef * div[v];
              out[(size_t)v * nint + o] = Un[v];
            }
            R m2;
            R A = A_of_cons(Un, &m2, P.ori);
            if (!(val(Un[0]) > 0.0) || !(val(A) > kEpsUnphysical)) fail = 1;
          }
    }
    if (!fail) break;
    if (theta == 0.0) { result = BLK_UNPHYSICAL; break; }
    ++attempt;
    theta = theta * P.retry_factor;
    if (theta < P.theta_floor * theta0) theta = 0.0;
  }
  if (badin || predicted_bad)
    for (size_t q = 0; q < (size_t)5 * nint; ++q) out[q] = R(NAN);
  if (retries_out) *retries_out = attempt;
  if (flux_out) {
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
      for (size_t q = 0; q < (size_t)5 * nf[d]; ++q) flux_out[off + q] = Fd[d][q];
      off += (size_t)5 * nf[d];
    }
  }
  return result;
}


// ----------------------------------------------------------------------------
// Exact solution of the 1-D relativistic Riemann problem with the TM EoS
// (Appendix C). Double precision only; this is not on the hot path.
// ----------------------------------------------------------------------------

// Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's
// method on the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2).
struct GaussLegendre {
  static constexpr int n = 16;
  double x[n], w[n];
  GaussLegendre() {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double z1 = z;
        z = z1 - p1 / dp;
        if (std::fabs(z - z1) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};
const GaussLegendre& gauss_legendre() { static GaussLegendre g; return g; }

// Integrand of the rarefaction rapidity integral in u = ln T: along an
// isentrope of the TM gas, d ln rho = (1.5/T + 2.25/sqrt(1 + 2.25 T^2)) dT
// (from dh = dp/rho with p = rho T, i.e. Eq. entropy), and the Riemann
// invariant Eq. (Riemann invariant) gives d asinh(U) = +/- c_s d ln rho.
// Polytropic EoS: p/rho^Gamma = const, d ln rho = dT / ((Gamma-1) T).
double rapidity_integrand(double u) {
  double T = std::exp(u);
  double cs = std::sqrt(cs2_of_T(T));
  if (g_eos.gamma_law) return cs / (g_eos.gam - 1.0);
  return cs * (1.5 + 2.25 * T / std::sqrt(1.0 + 2.25 * T * T));
}

double gl_panel(double a, double b) {
  const GaussLegendre& g = gauss_legendre();
  double c = 0.5 * (a + b), r = 0.5 * (b - a), s = 0.0;
  for (int i = 0; i < GaussLegendre::n; ++i) s += g.w[i] * rapidity_integrand(c + r * g.x[i]);
  return s * r;
}

double gl_adapt(double a, double b, double whole, double tol, int depth) {
  double m = 0.5 * (a + b);
  double l = gl_panel(a, m), r = gl_panel(m, b);
  if (std::fabs(l + r - whole) <= tol || depth >= 12) return l + r;
  return gl_adapt(a, m, l, 0.5 * tol, depth + 1) + gl_adapt(m, b, r, 0.5 * tol, depth + 1);
}

// I(T1, T2) = integral from T1 to T2 of c_s (1.5/T + 2.25/sqrt(1+2.25T^2)) dT.
double rapidity_integral(double T1, double T2) {
  if (T1 == T2) return 0.0;
  double a = std::log(T1), b = std::log(T2);
  double sign = 1.0;
  if (a > b) { std::swap(a, b); sign = -1.0; }
  double whole = 0.0;
  // Coarse panels of width <= 1 in ln T, each refined adaptively.
  int np = std::max(1, (int)std::ceil(b - a));
  double acc = 0.0;
  for (int q = 0; q < np; ++q) {
    double lo = a + (b - a) * q / np, hi = a + (b - a) * (q + 1) / np;
    whole = gl_panel(lo, hi);
    acc += gl_adapt(lo, hi, whole, 1e-300 + 2e-15 * std::fabs(whole), 0);
  }
  return sign * acc;
}

struct RState {
  double rho, U, p, T, h, cs, phi;
};

RState make_state(double rho, double U, double p) {
  RState s;
  s.rho = rho; s.U = U; s.p = p;
  s.T = p / rho;
  s.h = 1.0 + htilde_of_T(s.T);
  s.cs = std::sqrt(cs2_of_T(s.T));
  s.phi = std::asinh(U);
  return s;
}

// Density on the isentrope through state K at temperature T (Eq. entropy,
// p (h - T) / rho^{5/3} = const with p = rho T): rho = rho_K [T (h-T) /
// (T_K (h_K - T_K))]^{3/2}.
double isentrope_rho(const RState& K, double T) {
  if (g_eos.gamma_law) return K.rho * std::pow(T / K.T, 1.0 / (g_eos.gam - 1.0));
  double h = 1.0 + htilde_of_T(T);
  return K.rho * std::pow(T * (h - T) / (K.T * (K.h - K.T)), 1.5);
}

// Temperature on the isentrope through K where the pressure equals p.
double isentrope_T_at_p(const RState& K, double p) {
  double lo = std::log(K.T) - 120.0, hi = std::log(K.T) + 120.0;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double T = std::exp(mid);
    if (isentrope_rho(K, T) * T < p) lo = mid; else hi = mid;
  }
  return std::exp(0.5 * (lo + hi));
}

struct WaveCurve {
  int shock;       // 1 shock, 0 rarefaction (or no wave)
  double phi;      // rapidity behind the wave
  double rho;      // density behind the wave
  double Ushock;   // shock four-velocity (shock only)
  double Tstar;    // temperature behind the wave
};

// Shock branch (Appendix C, U_S): solve the Taub adiabat Eq. (TaubAdiabatic)
// for the downstream temperature, then the mass flux Eq. (mass flux) and
// the Lorentz boosts Eq. (Ushock) and Eq. (Udown); s = -1 left, +1 right.
// (In Eq. Ushock the second +/- must be +: it is the velocity composition of
// U_up with the upstream speed J/rho_up relative to the shock.)
WaveCurve shock_curve(const RState& K, double ps, int s) {
  auto G = [&](double Td) {
    double hd = 1.0 + htilde_of_T(Td);
    double rhod = ps / Td;
    return K.h * K.h - hd * hd - (hd / rhod + K.h / K.rho) * (K.p - ps);
  };
  double lo = std::log(K.T), hi = lo + 1.0;
  int guard = 0;
  while (G(std::exp(hi)) > 0.0 && guard++ < 400) hi += 2.0;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (G(std::exp(mid)) > 0.0) lo = mid; else hi = mid;
  }
  // final polish by bisection in T itself
  double tlo = std::exp(lo), thi = std::exp(hi);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (tlo + thi);
    if (mid <= tlo || mid >= thi) break;
    if (G(mid) > 0.0) tlo = mid; else thi = mid;
  }
  double Td = (std::fabs(G(tlo)) < std::fabs(G(thi))) ? tlo : thi;
  double hd = 1.0 + htilde_of_T(Td);
  double rhod = ps / Td;
  double J = std::sqrt((ps - K.p) / (K.h / K.rho - hd / rhod));
  // Eq. (Ushock) and Eq. (Udown) are Lorentz boosts by the shock-frame
  // speeds J/rho_up and J/rho_down; they are applied as the equivalent
  // rapidity additions, which avoid the cancellation of products of order
  // gamma^2 when the upstream gas is ultra-relativistic.
  double ju = J / K.rho, jd = J / rhod;
  double phi_sh = K.phi + s * std::asinh(ju);
  double phi_d = phi_sh - s * std::asinh(jd);
  WaveCurve w;
  w.shock = 1; w.phi = phi_d; w.rho = rhod; w.Ushock = std::sinh(phi_sh); w.Tstar = Td;
  return w;
}

// Rarefaction branch (Appendix C, U_R): isentrope Eq. (entropy) plus the
// Riemann invariant Eq. (Riemann invariant) integrated in T.
WaveCurve rarefaction_curve(const RState& K, double ps, int s) {
  double Ts = isentrope_T_at_p(K, ps);
  WaveCurve w;
  w.shock = 0;
  w.Tstar = Ts;
  w.rho = isentrope_rho(K, Ts);
  w.phi = K.phi - s * rapidity_integral(Ts, K.T);
  w.Ushock = 0.0;
  return w;
}

WaveCurve wave_curve(const RState& K, double ps, int s) {
  if (ps > K.p) return shock_curve(K, ps, s);
  if (ps < K.p) return rarefaction_curve(K, ps, s);
  WaveCurve w;
  w.shock = 0; w.phi = K.phi; w.rho = K.rho; w.Ushock = 0.0; w.Tstar = K.T;
  return w;
}

struct ExactSolution {
  RState L, R;
  double pstar;
  WaveCurve wl, wr;
};

// p* from equality of the contact rapidities (Eq. p*, written as
// phi_CL(p*) = phi_CR(p*), which is Relative(U_CL, U_CR) = 0), bracketed and
// bisected in ln p and then in p.
ExactSolution solve_exact(const RState& L, const RState& R) {
  auto g = [&](double p) { return wave_curve(L, p, -1).phi - wave_curve(R, p, +1).phi; };
  double lo = std::log(std::min(L.p, R.p)) - 1.0;
  double hi = std::log(std::max(L.p, R.p)) + 1.0;
  int guard = 0;
  while (g(std::exp(lo)) < 0.0 && guard++ < 200) lo -= 2.0;
  guard = 0;
  while (g(std::exp(hi)) > 0.0 && guard++ < 200) hi += 2.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (g(std::exp(mid)) > 0.0) lo = mid; else hi = mid;
  }
  double plo = std::exp(lo), phi_ = std::exp(hi);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (plo + phi_);
    if (mid <= plo || mid >= phi_) break;
    if (g(mid) > 0.0) plo = mid; else phi_ = mid;
  }
  ExactSolution S;
  S.L = L; S.R = R;
  S.pstar = (std::fabs(g(plo)) < std::fabs(g(phi_))) ? plo : phi_;
  S.wl = wave_curve(L, S.pstar, -1);
  S.wr = wave_curve(R, S.pstar, +1);
  return S;
}

// State inside a rarefaction fan at similarity coordinate xi (Appendix C,
// step 3): find T with phi(T) - s atanh(c_s(T)) ... written per side as
// phi(T) + atanh(c_s) = atanh(xi) (left, s = -1) or phi(T) - atanh(c_s) =
// atanh(xi)... expressed as tanh(phi -/+ atanh c_s) = xi.
void fan_state(const RState& K, const WaveCurve& w, int s, double xi, double* rho, double* U,
               double* p) {
  double target = std::atanh(xi);
  auto F = [&](double T) {
    double phi = K.phi - s * rapidity_integral(T, K.T);
    return phi + s * std::atanh(std::sqrt(cs2_of_T(T)));
  };
  // Between T* and T_K. Left fan (s=-1): F(T) = phi - atanh(cs) decreases
  // with T; right fan (s=+1): F = phi + atanh(cs) increases with T.
  double lo = std::log(std::min(w.Tstar, K.T)), hi = std::log(std::max(w.Tstar, K.T));
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double v = F(std::exp(mid));
    bool go_up = (s < 0) ? (v > target) : (v < target);
    if (go_up) lo = mid; else hi = mid;
  }
  double T = std::exp(0.5 * (lo + hi));
  double phi = K.phi - s * rapidity_integral(T, K.T);
  *rho = isentrope_rho(K, T);
  *U = std::sinh(phi);
  *p = *rho * T;
}

void sample_exact(const ExactSolution& S, double xi, double* rho, double* U, double* p) {
  const RState& L = S.L;
  const RState& R = S.R;
  double phis = S.wl.phi;  // == S.wr.phi up to the root tolerance
  double vc = std::tanh(0.5 * (S.wl.phi + S.wr.phi));
  // left wave
  if (S.wl.shock) {
    double vs = S.wl.Ushock / std::sqrt(1.0 + S.wl.Ushock * S.wl.Ushock);
    if (xi < vs) { *rho = L.rho; *U = L.U; *p = L.p; return; }
  } else if (S.pstar < L.p) {
    double head = std::tanh(L.phi - std::atanh(L.cs));
    double tail = std::tanh(phis - std::atanh(std::sqrt(cs2_of_T(S.wl.Tstar))));
    if (xi < head) { *rho = L.rho; *U = L.U; *p = L.p; return; }
    if (xi < tail) { fan_state(L, S.wl, -1, xi, rho, U, p); return; }
  } else if (xi < vc) { *rho = L.rho; *U = L.U; *p = L.p; return; }
  if (xi < vc) { *rho = S.wl.rho; *U = std::sinh(S.wl.phi); *p = S.pstar; return; }
  // right wave
  if (S.wr.shock) {
    double vs = S.wr.Ushock / std::sqrt(1.0 + S.wr.Ushock * S.wr.Ushock);
    if (xi > vs) { *rho = R.rho; *U = R.U; *p = R.p; return; }
  } else if (S.pstar < R.p) {
    double head = std::tanh(R.phi + std::atanh(R.cs));
    double tail = std::tanh(S.wr.phi + std::atanh(std::sqrt(cs2_of_T(S.wr.Tstar))));
    if (xi > head) { *rho = R.rho; *U = R.U; *p = R.p; return; }
    if (xi > tail) { fan_state(R, S.wr, +1, xi, rho, U, p); return; }
  } else { *rho = R.rho; *U = R.U; *p = R.p; return; }
  *rho = S.wr.rho; *U = std::sinh(S.wr.phi); *p = S.pstar;
}

}  // namespace

// ============================================================================
// C interface for ctypes. Arrays are float64, C-contiguous.
// ============================================================================
extern "C" {

// EoS selection for the calls that follow on this thread: kind 0 = TM,
// kind 1 = polytropic with the given Gamma (1 < Gamma <= 5/3). Returns 0, or
// BADARG.
int or_set_eos(int kind, double gam) {
  if (kind == 0) { g_eos.gamma_law = 0; return OK; }
  if (kind != 1 || !(gam > 1.0) || !(gam <= 5.0 / 3.0 + 1e-12)) return BADARG;
  g_eos.gamma_law = 1;
  g_eos.gam = gam;
  return OK;
}
double or_htilde_of_T(double T) { return htilde_of_T(T); }
double or_T_of_htilde(double ht) { return T_of_htilde(ht); }
double or_dT_dhtilde(double ht) { return dT_dhtilde(ht); }
double or_cs2_of_T(double T) { return cs2_of_T(T); }
double or_f_of_htilde(double ht, double m2) { return f_of_htilde(ht, T_of_htilde(ht), m2); }
double or_df_dhtilde(double ht, double m2) {
  return df_dhtilde(ht, T_of_htilde(ht), dT_dhtilde(ht), m2);
}
double or_newton_guess(double A, double m2) { return newton_guess(A, m2); }
double or_htilde_bisect(double A, double m2) { return htilde_bisect(A, m2); }
double or_limited_slope(double dl, double dr, double theta) { return limited_slope(dl, dr, theta); }

// Batched prim2con: prim [5][n] -> cons [5][n]; status [n] (nullable).
void or_prim2con(const double* prim, double* cons, int64_t n, int32_t* status, int scheme) {
  for (int64_t i = 0; i < n; ++i) {
    double W[5], U[5];
    for (int v = 0; v < 5; ++v) W[v] = prim[v * n + i];
    int st = prim2con(W, U, scheme);
    for (int v = 0; v < 5; ++v) cons[v * n + i] = U[v];
    if (status) status[i] = st;
  }
}

// Batched con2pri: cons [5][n] -> prim [5][n]; status, iters, htilde, A
// (each nullable).
void or_con2pri(const double* cons, double* prim, int64_t n, int32_t* status,
                int32_t* iters, double* htilde, double* A, int scheme) {
  for (int64_t i = 0; i < n; ++i) {
    double U[5], W[5], ht = NAN;
    for (int v = 0; v < 5; ++v) U[v] = cons[v * n + i];
    Con2PriInfo info;
    int st = con2pri(U, W, &ht, &info, scheme);
    for (int v = 0; v < 5; ++v) prim[v * n + i] = W[v];
    if (status) status[i] = st;
    if (iters) iters[i] = info.iters;
    if (htilde) htilde[i] = info.htilde;
    if (A) A[i] = info.A;
  }
}

// One physical flux / Riemann flux evaluation (for unit tests).
void or_phys_flux(int d, const double* W, const double* U, double* F, int scheme) {
  phys_flux(d, W, U, F, scheme);
}
void or_char_speeds(int d, const double* W, double* lm, double* lp) { char_speeds(d, W, lm, lp); }
int or_riemann_flux(int d, int solver, const double* WL, const double* UL, const double* WR,
                    const double* UR, double* F, int scheme) {
  return riemann_flux(d, solver, WL, UL, WR, UR, F, scheme);
}
double or_smax(const double* W, int ndim) { return smax_of_prim(W, ndim); }

// One MUSCL-Hancock step of a block with ghost zones. flux_out (nullable)
// receives the face fluxes, direction-major [d][5][faces of d].
int or_advance_block(const double* in, double* out, double* flux_out, int nx, int ny, int nz,
                     int actx, int acty, int actz, double dt, double dh, double theta,
                     double retry_factor, double theta_floor, int riemann, int32_t* retries,
                     int scheme) {
  int n[3] = {nx, ny, nz};
  int act[3] = {actx, acty, actz};
  Params P{theta, retry_factor, theta_floor, riemann, actx + acty + actz, 0.5, 0, scheme};
  int r = 0;
  int st = advance_block(in, out, flux_out, n, act, dt, dh, P, &r);
  if (retries) *retries = r;
  return st;
}

// Batched advance of npatch independent 8^3 patches with 2-cell ghosts,
// cons_in [np][5][12^3] -> cons_out [np][5][8^3]; dt_dh [np][2];
// status [np] and retries [np] (nullable).
void or_advance_patches(const double* in, double* out, int64_t npatch, const double* dt_dh,
                        double theta, double retry_factor, double theta_floor, int riemann,
                        int32_t* status, int32_t* retries, double* flux_out, int scheme) {
  const int n[3] = {8, 8, 8};
  const int act[3] = {1, 1, 1};
  Params P{theta, retry_factor, theta_floor, riemann, 3, 0.5, 0, scheme};
  const size_t nflux = (size_t)3 * 5 * 9 * 64;
  for (int64_t p = 0; p < npatch; ++p) {
    int r = 0;
    int st = advance_block(in + (size_t)p * 5 * 1728, out + (size_t)p * 5 * 512,
                           flux_out ? flux_out + (size_t)p * nflux : (double*)nullptr, n, act,
                           dt_dh[2 * p], dt_dh[2 * p + 1], P, &r);
    if (status) status[p] = st;
    if (retries) retries[p] = r;
  }
}

// VL block step (3 ghost cells on active sides), arguments as or_advance_block.
int or_advance_block_vl(const double* in, double* out, double* flux_out, int nx, int ny, int nz,
                        int actx, int acty, int actz, double dt, double dh, double theta,
                        double retry_factor, double theta_floor, int riemann, int32_t* retries,
                        int scheme) {
  int n[3] = {nx, ny, nz};
  int act[3] = {actx, acty, actz};
  Params P{theta, retry_factor, theta_floor, riemann, actx + acty + actz, 0.5, 0, scheme};
  int r = 0;
  int st = advance_block_vl(in, out, flux_out, n, act, dt, dh, P, &r);
  if (retries) *retries = r;
  return st;
}

// Batched VL advance of 8^3 patches with 3-cell ghosts, cons_in [np][5][14^3].
void or_advance_patches_vl(const double* in, double* out, int64_t npatch, const double* dt_dh,
                           double theta, double retry_factor, double theta_floor, int riemann,
                           int32_t* status, int32_t* retries, double* flux_out, int scheme) {
  const int n[3] = {8, 8, 8};
  const int act[3] = {1, 1, 1};
  Params P{theta, retry_factor, theta_floor, riemann, 3, 0.5, 0, scheme};
  const size_t nflux = (size_t)3 * 5 * 9 * 64;
  for (int64_t p = 0; p < npatch; ++p) {
    int r = 0;
    int st = advance_block_vl(in + (size_t)p * 5 * 2744, out + (size_t)p * 5 * 512,
                              flux_out ? flux_out + (size_t)p * nflux : (double*)nullptr, n, act,
                              dt_dh[2 * p], dt_dh[2 * p + 1], P, &r);
    if (status) status[p] = st;
    if (retries) retries[p] = r;
  }
}

// CFL time step over cells cons [5][n] (Eq. time_step_sound_speed): returns
// min_i C dh / S_max,i (cfl_mode 0) or C dh (cfl_mode 1, speed of light);
// NaN if any cell is unphysical.
double or_cfl_dt(const double* cons, int64_t n, double dh, double cfl, int ndim, int cfl_mode,
                 int scheme) {
  if (cfl_mode == 1) return cfl * dh;
  double smax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double U[5], W[5];
    for (int v = 0; v < 5; ++v) U[v] = cons[v * n + i];
    int st = con2pri(U, W, (double*)nullptr, (Con2PriInfo*)nullptr, scheme);
    if (st == UNPHYSICAL) return NAN;
    smax = std::max(smax, smax_of_prim(W, ndim));
  }
  return cfl * dh / smax;
}

// Algorithmic operation count of one block advance (adds+subs, muls, divs,
// sqrts), using the counting instantiation of the same code.
void or_count_advance_block(const double* in, int nx, int ny, int nz, int actx, int acty,
                            int actz, double dt, double dh, double theta, int riemann,
                            uint64_t* counts) {
  int n[3] = {nx, ny, nz};
  int act[3] = {actx, acty, actz};
  Params P{theta, 0.75, 1e-2, riemann, actx + acty + actz, 0.5, 0, 0};
  int nin = 1;
  for (int d = 0; d < 3; ++d) nin *= n[d] + (act[d] ? 4 : 0);
  std::vector<OpCount> cin((size_t)5 * nin), cout((size_t)5 * nx * ny * nz);
  for (size_t q = 0; q < cin.size(); ++q) cin[q] = OpCount(in[q]);
  g_tally = OpTally();
  int r = 0;
  advance_block(cin.data(), cout.data(), (OpCount*)nullptr, n, act, OpCount(dt), OpCount(dh), P, &r);
  counts[0] = g_tally.add;
  counts[1] = g_tally.mul;
  counts[2] = g_tally.div;
  counts[3] = g_tally.sqrt;
}

// The same count for one VL block advance (3 ghost cells on active sides).
void or_count_advance_block_vl(const double* in, int nx, int ny, int nz, int actx, int acty,
                               int actz, double dt, double dh, double theta, int riemann,
                               uint64_t* counts) {
  int n[3] = {nx, ny, nz};
  int act[3] = {actx, acty, actz};
  Params P{theta, 0.75, 1e-2, riemann, actx + acty + actz, 0.5, 0, 0};
  int nin = 1;
  for (int d = 0; d < 3; ++d) nin *= n[d] + (act[d] ? 6 : 0);
  std::vector<OpCount> cin((size_t)5 * nin), cout((size_t)5 * nx * ny * nz);
  for (size_t q = 0; q < cin.size(); ++q) cin[q] = OpCount(in[q]);
  g_tally = OpTally();
  int r = 0;
  advance_block_vl(cin.data(), cout.data(), (OpCount*)nullptr, n, act, OpCount(dt), OpCount(dh), P,
                   &r);
  counts[0] = g_tally.add;
  counts[1] = g_tally.mul;
  counts[2] = g_tally.div;
  counts[3] = g_tally.sqrt;
}

// Operation count of the signal-speed CFL bound of n cells (con2pri + S_max).
void or_count_cfl(const double* cons, int64_t n, int ndim, uint64_t* counts) {
  g_tally = OpTally();
  for (int64_t i = 0; i < n; ++i) {
    OpCount U[5], W[5];
    for (int v = 0; v < 5; ++v) U[v] = OpCount(cons[v * n + i]);
    con2pri(U, W, (OpCount*)nullptr, (Con2PriInfo*)nullptr);
    smax_of_prim(W, ndim);
  }
  counts[0] = g_tally.add;
  counts[1] = g_tally.mul;
  counts[2] = g_tally.div;
  counts[3] = g_tally.sqrt;
}

// Exact TM Riemann solution (Appendix C) sampled at x[n] for time t with the
// initial discontinuity at x0. info (nullable, 10 doubles): p*, U*_L, U*_R,
// rho*_L, rho*_R, left shock flag, right shock flag, U_shock_L, U_shock_R,
// T*_L.
void or_exact_riemann(double rhoL, double UL, double pL, double rhoR, double UR, double pR,
                      double x0, double t, const double* x, int64_t n, double* rho, double* U,
                      double* p, double* info) {
  RState L = make_state(rhoL, UL, pL), R = make_state(rhoR, UR, pR);
  ExactSolution S = solve_exact(L, R);
  for (int64_t i = 0; i < n; ++i) sample_exact(S, (x[i] - x0) / t, &rho[i], &U[i], &p[i]);
  if (info) {
    info[0] = S.pstar;
    info[1] = std::sinh(S.wl.phi);
    info[2] = std::sinh(S.wr.phi);
    info[3] = S.wl.rho;
    info[4] = S.wr.rho;
    info[5] = S.wl.shock;
    info[6] = S.wr.shock;
    info[7] = S.wl.Ushock;
    info[8] = S.wr.Ushock;
    info[9] = S.wl.Tstar;
  }
}

double or_rapidity_integral(double T1, double T2) { return rapidity_integral(T1, T2); }

}  // extern "C"
