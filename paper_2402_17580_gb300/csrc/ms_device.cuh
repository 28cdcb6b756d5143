// Device-side phase model and moving-source temperature for sm_103a.
//
// Every function is templated on the arithmetic type AT of the rates and the
// temperature (float: SFU ex2.approx / lg2.approx / rsqrt.approx /
// rcp.approx, with exp(x) = 2^(x log2 e) and x^p = 2^(p log2 x); double: the
// device's FP64 exp2 / log2 / rsqrt, for the full-FP64 spot-check path) and on
// the fraction type FT that carries the stored state and the Euler
// accumulation (float, double, or the compensated pair KF).
//
// Paper passages (arXiv 2402.17580):
//   X_alpha^eq                   Sec. 2.2, eq:equilibrium_phase_as
//   X_am,0^eq, X_am^eq           Sec. 2.2, eq:equilibrium_phase_am0 / eq:equilibrium_phase_am
//   rates r1, r2, r3             Sec. 2.2, eq:beta_to_alpha_s, eq:alpha_m_to_alpha_s,
//                                eq:alpha_s_to_beta; k_as, k_beta after them
//   martensite                   eq:inst_martensite_formation, eq:inst_martensite_dissolution
//   regularisation               Sec. 2.2 (T_reg = 100 K)
//   explicit step                Sec. 3.1, eq:explicit_integration + eq:explicit_correction
//   initiation                   Appendix A, eq:analytical_solution_beta
//   liquid fraction              Sec. 2.1, eq:liquid_fraction
#pragma once

#include <cstdint>
#include <type_traits>

namespace ms {

// Constants derived on the host from ms_params, in the arithmetic type.
template <typename AT>
struct ModelConstT {
  AT T_s, T_l, inv_mushy;           // eq:liquid_fraction
  AT T_as_start, T_as_end;          // Table 2
  AT T_am_start, T_inf;             // Table 2
  AT kaeq_l2;                       // k_alpha_eq * log2(e)
  AT kam_l2;                        // k_am_eq * log2(e)
  AT k1, k2, k3_l2;                 // Table 3, k3 * log2(e)
  AT f;                             // Table 3
  AT c_as, c_b, inv_c_as, inv_c_b;
  AT pa, qa, pb, qb;                // (c -+ 1) / c for alpha_s and beta
  AT T_cap0, inv_T_reg;             // T_as_start + T_reg, 1 / T_reg
  AT init_exit, init_exit_floor;    // App. A exit rule (reading A5)
  AT T_thr;                         // active-set threshold
  int martensite_literal;           // reading A3
  int init_ba_steps;                // reading A6
  AT fp_eps_abs, fp_eps_rel;        // implicit scheme: WRMS tolerances (Sec. 3)
  int fp_max_iter;                  // implicit scheme: iteration cap
};
using ModelConst = ModelConstT<float>;

// Compensated FP32 fraction (MS_KAHAN): an unevaluated sum hi + lo of two
// floats (double-float).  Sums and differences are error-free transforms
// (TwoSum, then FastTwoSum to renormalise), products carry the FMA error term,
// so the Euler accumulation keeps ~44 bits where plain FP32 keeps 24.
struct KF {
  float hi, lo;
  __host__ __device__ KF() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ KF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit KF(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
  __host__ __device__ explicit KF(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ explicit KF(int v) : hi(float(v)), lo(0.0f) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
};

__host__ __device__ __forceinline__ KF kf_fast_two_sum(float a, float b) {
  const float s = a + b;
  return KF(s, b - (s - a));
}
__host__ __device__ __forceinline__ KF operator+(KF a, KF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
  return kf_fast_two_sum(s, e);
}
__host__ __device__ __forceinline__ KF operator-(KF a) { return KF(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ KF operator-(KF a, KF b) { return a + (-b); }
__host__ __device__ __forceinline__ KF operator*(KF a, KF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  return kf_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ KF operator/(KF a, KF b) {
  const float q1 = a.hi / b.hi;
  const KF r = a - b * KF(q1);
  return kf_fast_two_sum(q1, r.hi / b.hi);
}
__host__ __device__ __forceinline__ KF& operator*=(KF& a, KF b) { return a = a * b; }
__host__ __device__ __forceinline__ bool operator<(KF a, KF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ bool operator>(KF a, KF b) { return b < a; }
__host__ __device__ __forceinline__ bool operator<=(KF a, KF b) { return !(b < a); }
__host__ __device__ __forceinline__ bool operator>=(KF a, KF b) { return !(a < b); }
__host__ __device__ __forceinline__ bool operator==(KF a, KF b) { return a.hi == b.hi && a.lo == b.lo; }

// ----------------------------------------------------------- math per type
__device__ __forceinline__ float sfu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp2 and log2 on the FMA pipe (the paper's polynomial transcendentals,
// Sec. 3.3, for FP32): an IEEE-754 range reduction, a polynomial fitted by
// weighted least squares on Chebyshev nodes (paper_2402_17580_gb300/
// fit_poly.py prints the coefficients) evaluated with Estrin's scheme, and the
// exponent written back into the bits.  No conversion instruction: integers
// move through the 1.5 * 2^23 rounding constant.
//   fma_ex2: x = n + f, n = round(x), |f| <= 1/2; 2^f by a degree-6 polynomial
//            (relative error <= 1e-7 in FP32); 0 below 2^-126 like
//            ex2.approx.ftz, 2^127.99 at most.
//   fma_lg2: x = 2^e m, m in [sqrt(1/2), sqrt(2)), t = m - 1; log2(1 + t) =
//            t q(t) with q of degree 8 (absolute error <= 6e-8 on t q);
//            -inf for 0 and subnormals (ftz), NaN below 0, inf for inf.
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float fma_ex2(float x) {
  const float xc = fminf(x, 127.99f);
  const float tn = xc + kRound;
  const float n = tn - kRound;
  const float f = xc - n;
  const float f2 = f * f;
  const float f4 = f2 * f2;
  const float a = fmaf(6.931472056e-01f, f, 1.000000001e+00f);
  const float b = fmaf(5.550328998e-02f, f, 2.402264661e-01f);
  const float c = fmaf(1.339986036e-03f, f, 9.618519534e-03f);
  const float d = fmaf(1.533757683e-04f, f2, c);
  const float p = fmaf(f4, d, fmaf(f2, b, a));
  const int ni = __float_as_int(tn) - 0x4B400000;
  const float r = __int_as_float(__float_as_int(p) + (ni << 23));
  return xc < -126.0f ? 0.0f : r;
}
__device__ __forceinline__ float fma_lg2(float x) {
  const int i = __float_as_int(x);
  const int e = (i - 0x3F3504F3) >> 23;
  const float t = __int_as_float(i - (e << 23)) - 1.0f;
  const float ef = __int_as_float(e + 0x4B400000) - kRound;
  const float t2 = t * t;
  const float t4 = t2 * t2;
  const float q0 = fmaf(-7.213474818e-01f, t, 1.442695004e+00f);
  const float q1 = fmaf(-3.606921079e-01f, t, 4.809107678e-01f);
  const float q2 = fmaf(-2.391949061e-01f, t, 2.879017533e-01f);
  const float q3 = fmaf(-2.057056070e-01f, t, 2.161191295e-01f);
  const float q23 = fmaf(1.228052831e-01f, t4, fmaf(t2, q3, q2));
  const float q = fmaf(t4, q23, fmaf(t2, q1, q0));
  const float r = fmaf(t, q, ef);
  return x >= 1.17549435e-38f ? (x < INFINITY ? r : x)
                              : (x >= 0.0f ? -INFINITY : __int_as_float(0x7fffffff));
}

template <typename AT>
struct Fn;
template <>
struct Fn<float> {
#ifdef MS_FMA_TRANSCENDENTALS
  // the translation unit of the FMA-pipe variant (MS_FLAG_FMA_TRANSCENDENTALS)
  static __device__ __forceinline__ float ex2(float x) { return fma_ex2(x); }
  static __device__ __forceinline__ float lg2(float x) { return fma_lg2(x); }
#else
  static __device__ __forceinline__ float ex2(float x) { return sfu_ex2(x); }
  static __device__ __forceinline__ float lg2(float x) { return sfu_lg2(x); }
#endif
  static __device__ __forceinline__ float rsqrt(float x) { return sfu_rsqrt(x); }
  static __device__ __forceinline__ float rcp(float x) { return sfu_rcp(x); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float min(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
};
template <>
struct Fn<double> {
  static __device__ __forceinline__ double ex2(double x) { return ::exp2(x); }
  static __device__ __forceinline__ double lg2(double x) { return ::log2(x); }
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double max(double a, double b) { return ::fmax(a, b); }
  static __device__ __forceinline__ double min(double a, double b) { return ::fmin(a, b); }
  static __device__ __forceinline__ double abs(double a) { return ::fabs(a); }
};

constexpr float XMAX = 0.9f;  // bound on X_alpha used throughout Sec. 2.2

// An equilibrium value in the fraction type.  Its plateau 0.9 maps to FT(0.9)
// (from the double 0.9), the value a state set to 0.9 holds, so that states
// on the bound compare equal to the plateau also when FT is wider than AT
// (MS_F64ACC, MS_KAHAN: FT(0.9f) would sit 2.4e-8 below FT(0.9)).
template <typename AT, typename FT>
__device__ __forceinline__ FT eq_ft(AT v) {
  return v == AT(0.9) ? FT(0.9) : FT(v);
}

// ------------------------------------------------- transcendental counts
// The hot kernel's roofline counts the transcendental operations that the
// model's formulas require on the branch each point takes: ex2 (exp) and the
// slower class of lg2 (log, powers as 2^(p log2 x)) and rcp (division).  The
// model functions take a counter; NoCount compiles to
// nothing, SfuCount packs both classes into one word (ex2 in the low 16 bits,
// one add per branch) that the kernel drains per tile, before either half can
// reach 2^16 (at most 512 steps x 4 points x 12 operations of a class).
struct NoCount {
  __device__ __forceinline__ void add(unsigned, unsigned) {}
};
struct SfuCount {
  unsigned packed = 0;
  __device__ __forceinline__ void add(unsigned ex2, unsigned slow) { packed += ex2 | (slow << 16); }
};

// ------------------------------------------------------------ equilibria
// eq:equilibrium_phase_as
template <typename AT, typename OC = NoCount>
__device__ __forceinline__ AT xalpha_eq(const ModelConstT<AT>& m, AT T, OC&& oc = OC()) {
  if (T < m.T_as_end) return AT(0.9);
  if (T <= m.T_as_start) {
    oc.add(1, 0);
    return AT(1) - Fn<AT>::ex2(m.kaeq_l2 * (T - m.T_as_start));
  }
  return AT(0);
}

// eq:equilibrium_phase_am0, third branch at T > T_am,start and capped at 0.9
template <typename AT, typename OC = NoCount>
__device__ __forceinline__ AT xam0_eq(const ModelConstT<AT>& m, AT T, OC&& oc = OC()) {
  if (T < m.T_inf) return AT(0.9);
  if (T <= m.T_am_start) {
    oc.add(1, 0);
    return Fn<AT>::min(AT(1) - Fn<AT>::ex2(m.kam_l2 * (T - m.T_am_start)), AT(0.9));
  }
  return AT(0);
}

// eq:liquid_fraction
template <typename AT>
__device__ __forceinline__ AT liquid_fraction(const ModelConstT<AT>& m, AT T) {
  if (T < m.T_s) return AT(0);
  if (T > m.T_l) return AT(1);
  return (T - m.T_s) * m.inv_mushy;
}

// k_as(T) = k1 / (1 + exp(-k3 (T - k2)))
template <typename AT>
__device__ __forceinline__ AT k_alpha_s(const ModelConstT<AT>& m, AT T) {
  return m.k1 * Fn<AT>::rcp(AT(1) + Fn<AT>::ex2(m.k3_l2 * (m.k2 - T)));
}

// log2(1 + 2^y) without overflow
template <typename AT>
__device__ __forceinline__ AT softplus2(AT y) {
  return y > AT(0) ? y + Fn<AT>::lg2(AT(1) + Fn<AT>::ex2(-y))
                   : Fn<AT>::lg2(AT(1) + Fn<AT>::ex2(y));
}

// One step of eq:analytical_solution_beta in log2 form.  With xi = X / D,
// u = (xi / (1 - xi))^(1/c) grows by D k dt / c per step at constant k, and
// X^{n+1} = D / (1 + w^-c), w = u + D k dt / c.  lX is log2 X^n (-inf for
// X = 0); returns log2 X^{n+1}.  The log form keeps values far below the FP32
// range (X~ ~ 1e-70 after one step at 1200 K) representable.
template <typename AT, typename OC = NoCount>
__device__ __forceinline__ AT logistic_step_log2(AT lX, AT D, AT k, AT c, AT inv_c, AT dt,
                                                 OC&& oc = OC()) {
  const AT lD = Fn<AT>::lg2(D);
  AT u = AT(0);
  oc.add(1, 3);  // lg2 D, lg2 w, softplus2's 2^y and lg2
  if (lX > AT(-1.0e30)) {
    oc.add(2, 1);
    const AT lxi = lX - lD;
    const AT xi = Fn<AT>::ex2(lxi);
    u = Fn<AT>::ex2((lxi - Fn<AT>::lg2(AT(1) - xi)) * inv_c);
  }
  const AT w = Fn<AT>::fma(D * k * dt, inv_c, u);
  return lD - softplus2<AT>(Fn<AT>::mul_rn(-c, Fn<AT>::lg2(w)));
}

// ---------------------------------------------------------- correction g
// eq:explicit_correction: clamp negatives, rescale X_alpha > 0.9 keeping the
// ratio, alpha_s regularisation above T_as,start (clamped at 0), martensite
// dissolution if X_alpha > X_alpha^eq, martensite formation below T_am,start.
template <typename AT, typename FT, typename OC = NoCount>
__device__ __forceinline__ void correct(const ModelConstT<AT>& m, AT T, FT& xas, FT& xam,
                                        OC&& oc = OC()) {
  xas = xas > FT(0) ? xas : FT(0);
  xam = xam > FT(0) ? xam : FT(0);
  const FT xa = xas + xam;
  if (xa > FT(0.9)) {
    const FT s = FT(0.9) / xa;
    xas *= s;
    xam *= s;
  }
  if (T > m.T_as_start) {
    const AT cap = Fn<AT>::max(AT(0.9) * (m.T_cap0 - T) * m.inv_T_reg, AT(0));
    if (xas > FT(cap)) xas = FT(cap);
  }
  const FT xeq = eq_ft<AT, FT>(xalpha_eq<AT>(m, T, oc));
  if (xas + xam > xeq) {
    const FT v = xeq - xas;
    xam = v > FT(0) ? v : FT(0);
  }
  if (T < m.T_am_start) {
    const FT e = FT(xam0_eq<AT>(m, T, oc)) * (FT(0.9) - xas) * FT(1.0 / 0.9);
    if (m.martensite_literal) xam = e;
    else if (e > xam) xam = e;
  }
}

// ------------------------------------------------------------ point step
// A diffusive rate k x^p y^q as k 2^(p log2 x + q log2 y), log2 x given (it
// is shared between rates); the exponent is one explicit FMA, so every caller
// rounds it the same way.  x = 0 or y = 0 give 2^-inf = 0 (reading A14).
template <typename AT>
__device__ __forceinline__ AT pow_rate(AT k, AT p, AT lx, AT q, AT y) {
  return Fn<AT>::mul_rn(k, Fn<AT>::ex2(Fn<AT>::fma(q, Fn<AT>::lg2(y), p * lx)));
}

// The explicit Euler update x + dt d of a fraction: one FMA when the fraction
// type is the arithmetic type, else the rounded increment added in the
// fraction type.  It is written out, like the rounded product of pow_rate,
// because whether the compiler fuses a multiply into an add depends on the
// code around it: the per-point and the lockstep step would otherwise be free
// to round the same update differently.
template <typename AT, typename FT>
__device__ __forceinline__ FT euler_add(FT x, AT dt, AT d) {
  if constexpr (std::is_same<AT, FT>::value)
    return Fn<AT>::fma(dt, d, x);
  else
    return x + FT(Fn<AT>::mul_rn(dt, d));
}

// aux encodes the App. A initiation: 0 none; < 0 alpha_s -> beta in progress
// with aux = log2 X~_beta; > 0 (1.0) persisted beta -> alpha_s (init_ba_steps).
template <typename AT, typename FT, typename OC = NoCount>
__device__ __forceinline__ void point_step(const ModelConstT<AT>& m, AT T0, AT T1, AT dt,
                                           FT& xas_io, FT& xam_io, float& aux, OC&& oc = OC()) {
  const FT xas = xas_io, xam = xam_io;
  const FT xa = xas + xam;
  const AT xeq0 = xalpha_eq<AT>(m, T0, oc);
  const AT k = k_alpha_s<AT>(m, T0);
  oc.add(1, 1);  // k_as: exp and reciprocal
  const AT kb = m.f * k;

  const FT xeq0f = eq_ft<AT, FT>(xeq0);
  // App. A's alpha_s -> beta initiation needs D = 0.9 - X_alpha^eq > 0
  const bool can5 = xeq0 < AT(0.9);
  bool a5 = aux < 0.0f, a6 = aux > 0.0f;
  if (a5 && !(can5 && xa > xeq0f)) a5 = false;
  if (a6 && !(xa < xeq0f)) a6 = false;
  const bool enter5 = !a5 && !a6 && can5 && xa > xeq0f && FT(0.9) - xa <= FT(0) && xam == FT(0);

  FT nas, nam;
  AT L = AT(0);
  if (a5 || enter5) {
    // App. A: X~ = X_beta - 0.1, equilibrium D = X_beta^eq - 0.1, rate k_beta
    const AT D = AT(0.9) - xeq0;
    L = logistic_step_log2<AT>(a5 ? AT(aux) : AT(-INFINITY), D, kb, m.c_b, m.inv_c_b, dt, oc);
    oc.add(1, 0);
    nas = FT(0.9) - FT(Fn<AT>::ex2(L));
    nam = xam;
    a5 = true;
  } else if (xa < xeq0f && (xas == FT(0) || a6)) {
    // reading A6: beta -> alpha_s initiation, D = X_alpha^eq - X_am, alpha_m frozen
    const AT D = AT(xeq0f - xam);
    const AT las = xas > FT(0) ? Fn<AT>::lg2(AT(xas)) : AT(-INFINITY);
    if (xas > FT(0)) oc.add(0, 1);
    AT r2 = AT(0);
    if (xam > FT(0)) {
      oc.add(1, 1);
      r2 = pow_rate<AT>(k, m.pa, las, m.qa, AT(xam));
    }
    const AT lX = logistic_step_log2<AT>(las, D, k, m.c_as, m.inv_c_as, dt, oc);
    oc.add(1, 0);
    nas = euler_add<AT, FT>(FT(Fn<AT>::ex2(lX)), dt, r2);
    nam = euler_add<AT, FT>(xam, dt, -r2);
    if (m.init_ba_steps) a6 = true;
  } else {
    // eq:explicit_integration with the rates at T^n.  r1 and r3 exclude each
    // other and share one lg2 / lg2 / ex2 triple.
    const bool lo = xa < xeq0f, hi = xa > xeq0f;
    AT d_as = AT(0), d_am = AT(0);
    AT las = AT(0);
    if (lo || xam > FT(0)) las = Fn<AT>::lg2(AT(xas));
    if (lo) {
      oc.add(1, 2);  // lg2 X_as, lg2 (X_eq - X_a), ex2
      d_as = pow_rate<AT>(k, m.pa, las, m.qa, AT(xeq0f - xa));
    } else if (hi) {
      const FT gap = FT(0.9) - xa;
      const AT lg = gap > FT(0) ? Fn<AT>::lg2(AT(gap)) : AT(-INFINITY);
      oc.add(1, gap > FT(0) ? 2 : 1);
      d_as = pow_rate<AT>(-kb, m.pb, lg, m.qb, AT(xa - xeq0f));
    }
    if (xam > FT(0)) {
      oc.add(1, lo ? 1 : 2);  // lg2 X_am, ex2, and lg2 X_as unless r1 took it
      const AT r2 = pow_rate<AT>(k, m.pa, las, m.qa, AT(xam));
      d_as += r2;
      d_am = -r2;
    }
    nas = euler_add<AT, FT>(xas, dt, d_as);
    nam = euler_add<AT, FT>(xam, dt, d_am);
  }

  const FT before = nas;
  correct<AT, FT>(m, T1, nas, nam, oc);

  if (a5) {
    const AT xt = Fn<AT>::ex2(L);
    if (nas < before) a5 = false;  // the regularisation cap won
    else if (xt * dt > m.init_exit && xt >= m.init_exit_floor) a5 = false;
  } else if (a6) {
    const AT xs = AT(nas);
    if (xs * dt > m.init_exit && xs >= m.init_exit_floor) a6 = false;
  }
  aux = a5 ? float(L) : (a6 ? 1.0f : 0.0f);
  xas_io = nas;
  xam_io = nam;
}

// ------------------------------------------------- implicit scheme (Sec. 3)
// Diffusive rates m_diff(T, m) of eq:diff_inst_split: r1 (beta -> alpha_s)
// and r3 (alpha_s -> beta) exclude each other, r2 (alpha_m -> alpha_s) adds;
// powers as 2^(p log2 x), so 0^p = 0 (reading A14).
template <typename AT, typename FT>
__device__ __forceinline__ void diff_rates(const ModelConstT<AT>& m, AT T, FT xas, FT xam, AT& das,
                                           AT& dam) {
  const FT xa = xas + xam;
  const FT xeq = eq_ft<AT, FT>(xalpha_eq<AT>(m, T));
  const AT k = k_alpha_s<AT>(m, T);
  const bool lo = xa < xeq, hi = xa > xeq;
  das = AT(0);
  dam = AT(0);
  AT las = AT(0);
  if (lo || xam > FT(0)) las = Fn<AT>::lg2(AT(xas));
  if (lo) {
    das = k * Fn<AT>::ex2(m.pa * las + m.qa * Fn<AT>::lg2(AT(xeq - xa)));
  } else if (hi) {
    const FT gap = FT(0.9) - xa;
    const AT lg = gap > FT(0) ? Fn<AT>::lg2(AT(gap)) : AT(-INFINITY);
    das = -(m.f * k) * Fn<AT>::ex2(m.pb * lg + m.qb * Fn<AT>::lg2(AT(xa - xeq)));
  }
  if (xam > FT(0)) {
    const AT r2 = k * Fn<AT>::ex2(m.pa * las + m.qa * Fn<AT>::lg2(AT(xam)));
    das += r2;
    dam = -r2;
  }
}

// One Crank-Nicolson step from T0 to T1 (eq:implicit_integration +
// eq:implicit_correction) by the fixed-point iteration eq:implicit_fp_iteration
// in the order of the paper's implicit algorithm: m_0 = g(T1, m^n), then
// m_{i+1} = g(T1, m^n + dt/2 (mdot(T1, m_i) + mdot(T0, m^n))) until the WRMS
// norm of dt/2 (mdot(T1, m_{i+1}) - mdot(T1, m_i)), weights
// 1 / (eps_abs + |m_{i+1,j}| eps_rel), is below 1.  Adds the iterations to
// iters and returns false if the cap was reached.
template <typename AT, typename FT>
__device__ __forceinline__ bool cn_step(const ModelConstT<AT>& m, AT T0, AT T1, AT dt, FT& xas_io,
                                        FT& xam_io, unsigned& iters) {
  const FT xas = xas_io, xam = xam_io;
  AT das0, dam0;
  diff_rates<AT, FT>(m, T0, xas, xam, das0, dam0);
  FT mas = xas, mam = xam;
  correct<AT, FT>(m, T1, mas, mam);
  AT das, dam;
  diff_rates<AT, FT>(m, T1, mas, mam, das, dam);
  const AT h = AT(0.5) * dt;
  bool conv = false;
  for (int it = 0; it < m.fp_max_iter; ++it) {
    FT nas = xas + FT(h * (das + das0));
    FT nam = xam + FT(h * (dam + dam0));
    correct<AT, FT>(m, T1, nas, nam);
    AT das1, dam1;
    diff_rates<AT, FT>(m, T1, nas, nam, das1, dam1);
    const AT ras = h * (das1 - das) / (m.fp_eps_abs + Fn<AT>::abs(AT(nas)) * m.fp_eps_rel);
    const AT ram = h * (dam1 - dam) / (m.fp_eps_abs + Fn<AT>::abs(AT(nam)) * m.fp_eps_rel);
    mas = nas;
    mam = nam;
    das = das1;
    dam = dam1;
    ++iters;
    if (AT(0.5) * (ras * ras + ram * ram) < AT(1)) {
      conv = true;
      break;
    }
  }
  xas_io = mas;
  xam_io = mam;
  return conv;
}

// One implicit step of one point: n_sub substeps with the temperature linear
// in time between T0 and T1; in each substep an App. A initiation (aux, or
// its entry conditions) takes the explicit closed-form step, otherwise
// cn_step.
template <typename AT, typename FT>
__device__ __forceinline__ void point_step_implicit(const ModelConstT<AT>& m, AT T0, AT T1, AT dt,
                                                    int n_sub, FT& xas, FT& xam, float& aux,
                                                    unsigned& iters, unsigned& unconverged) {
  const AT h = dt / AT(n_sub);
  for (int s = 0; s < n_sub; ++s) {
    const AT Ta = T0 + (T1 - T0) * (AT(s) / AT(n_sub));
    const AT Tb = T0 + (T1 - T0) * (AT(s + 1) / AT(n_sub));
    const FT xa = xas + xam;
    const AT xeq0 = xalpha_eq<AT>(m, Ta);
    const FT xeq0f = eq_ft<AT, FT>(xeq0);
    const bool can5 = xeq0 < AT(0.9);
    const bool init = (aux < 0.0f && can5 && xa > xeq0f) || (aux > 0.0f && xa < xeq0f) ||
                      (can5 && xa > xeq0f && FT(0.9) - xa <= FT(0) && xam == FT(0)) ||
                      (xa < xeq0f && xas == FT(0));
    if (init) {
      point_step<AT, FT>(m, Ta, Tb, h, xas, xam, aux);
    } else {
      aux = 0.0f;
      if (!cn_step<AT, FT>(m, Ta, Tb, h, xas, xam, iters)) ++unconverged;
    }
  }
}

// A point may skip a step (active set, reading A9) when both temperatures are
// below T_thr and martensite formation at T1 would be a no-op, and (reading
// A9b) on the alpha_s plateau's fixed point X_as = 0.9, X_am = 0 while both
// are below T_as,end, where the step is the identity.
template <typename AT, typename FT>
__device__ __forceinline__ bool step_is_noop(const ModelConstT<AT>& m, AT T0, AT T1, FT xas,
                                             FT xam, float aux) {
  if (aux != 0.0f) return false;
  if (xas == FT(0.9) && xam == FT(0) && T0 < m.T_as_end && T1 < m.T_as_end) return true;
  if (!(T0 < m.T_thr && T1 < m.T_thr)) return false;
  if (!(T1 < m.T_am_start)) return true;
  const FT e = FT(xam0_eq<AT>(m, T1)) * (FT(0.9) - xas) * FT(1.0 / 0.9);
  return xam >= e;
}

// ------------------------------------------------------ moving point source
// One source of the table for one time level (see ms_heat_source in ms.h),
// in the source's own frame: along = x . u, across = x . (u_y, -u_x).
// 16-byte aligned: the FP32 kernels read an entry with two float4 loads.
template <typename AT>
struct alignas(16) SrcEntryT {
  AT s_xi;        // source position projected on u
  AT s_pp;        // source position projected on (u_y, -u_x)
  AT ux, uy;      // direction
  AT cR;          // -v / (2 alpha) * log2(e)
  AT lC;          // log2(A P / (2 pi k) * interlayer scale); -inf when 0
  AT hcR;         // -cR / 2 (the Newton correction of R + xi, source_term_x)
  AT pad1;
};
using SrcEntry = SrcEntryT<float>;

// SrcLevelT::axis: every source of the level moves along +-x (u_y == 0);
// LEVEL_AXIS_NEAR also says that the far field can serve none of them in any
// row tile (the source table's test against the specimen's whole x-range),
// so the kernels sum them point by point without classifying them.
constexpr int LEVEL_AXIS = 1;
constexpr int LEVEL_AXIS_NEAR = 3;

template <typename AT>
struct alignas(16) SrcLevelT {
  int n;          // started sources of the current layer at this level
  int axis;       // 0, LEVEL_AXIS or LEVEL_AXIS_NEAR
  AT z_surf;      // current layer surface (all its sources sit on it)
  AT T0, T_max;
};
using SrcLevel = SrcLevelT<float>;

// Contribution of one source to a point with squared depth below the surface
// dz2 (plus a tiny constant, which keeps R > 0 and sends R = 0 to the T_max
// cap):  A P / (2 pi k R) exp(-v (R + xi) / (2 alpha)).
// Behind the source (xi < 0) R + xi cancels: R carries the rounding of r2
// and of the approximate 1/sqrt, and a far receding source would lose its
// exponent to it.  So d = R + xi from the approximate R is refined by one
// Newton step on f(d) = d (d - 2 xi) - perp^2, which is 0 at the exact
// d = R + xi since (R + xi)(R - xi) = R^2 - xi^2 = perp^2:
//   d <- d - f(d) / f'(d),  f'(d) = 2 (d - xi) = 2 R ~ 2 / rinv.
// f(d) is one FMA of exact-or-once-rounded operands, so the refined d keeps
// its relative accuracy on both sides of the source with no reciprocal and no
// branch.  The correction is folded into the exponent:
//   cR d = cR d0 + hcR * (rinv f(d0)),  hcR = -cR / 2.
// In FP32: 10 instructions, 2 on the SFU, the last an FMA that adds the term
// to the caller's sum acc (written out, so that every path sums the sources
// with the same roundings); the offsets add 1 per point in a row tile
// (source_term_x) and 5 in the general form (source_term).
//
// The offsets are xi = px u_x + (py u_y - s_xi) and pp = px u_y + (py (-u_x)
// - s_pp); the bracketed parts and, when u_y == 0, perp^2 do not depend on
// px, so points that share py and pz may compute them once (source_offsets,
// source_term_x) and get the same bits.
template <typename AT>
__device__ __forceinline__ AT source_term_x(const SrcEntryT<AT>& e, AT xi, AT perp2, AT acc) {
  const AT r2 = Fn<AT>::fma(xi, xi, perp2);
  const AT rinv = Fn<AT>::rsqrt(r2);
  const AT d = Fn<AT>::fma(r2, rinv, xi);                                  // R + xi, approximate
  const AT f = Fn<AT>::fma(d, Fn<AT>::fma(AT(-2), xi, d), -perp2);        // d (d - 2 xi) - perp^2
  const AT a = Fn<AT>::fma(e.hcR, rinv * f, Fn<AT>::fma(e.cR, d, e.lC));  // cR (R + xi) + lC
  return Fn<AT>::fma(rinv, Fn<AT>::ex2(a), acc);
}

// The parts of xi and pp that do not depend on px.
template <typename AT>
__device__ __forceinline__ void source_offsets(const SrcEntryT<AT>& e, AT py, AT& c_xi, AT& c_pp) {
  c_xi = Fn<AT>::fma(py, e.uy, -e.s_xi);
  c_pp = Fn<AT>::fma(py, -e.ux, -e.s_pp);
}

template <typename AT>
__device__ __forceinline__ AT source_term(const SrcEntryT<AT>& e, AT px, AT py, AT dz2, AT acc) {
  AT c_xi, c_pp;
  source_offsets<AT>(e, py, c_xi, c_pp);
  const AT xi = Fn<AT>::fma(px, e.ux, c_xi);
  const AT pp = Fn<AT>::fma(px, e.uy, c_pp);
  return source_term_x<AT>(e, xi, Fn<AT>::fma(pp, pp, dz2), acc);
}

}  // namespace ms
