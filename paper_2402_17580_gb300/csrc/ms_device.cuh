// Device-side phase model and moving-source temperature for sm_103a.
//
// Arithmetic of the rates and transcendentals is FP32 on the SFU
// (ex2.approx / lg2.approx / rsqrt.approx / rcp.approx): exp(x) = 2^(x log2 e),
// x^p = 2^(p log2 x).  The fraction type FT (float or double) carries the
// stored state and the Euler accumulation.
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

namespace ms {

// FP32 constants derived on the host from ms_params.
struct ModelConst {
  float T_s, T_l, inv_mushy;        // eq:liquid_fraction
  float T_as_start, T_as_end;       // Table 2
  float T_am_start, T_inf;          // Table 2
  float kaeq_l2;                    // k_alpha_eq * log2(e)
  float kam_l2;                     // k_am_eq * log2(e)
  float k1, k2, k3_l2;              // Table 3, k3 * log2(e)
  float f;                          // Table 3
  float c_as, c_b, inv_c_as, inv_c_b;
  float pa, qa, pb, qb;             // (c -+ 1) / c for alpha_s and beta
  float T_cap0, inv_T_reg;          // T_as_start + T_reg, 1 / T_reg
  float init_exit, init_exit_floor; // App. A exit rule (reading A5)
  float T_thr;                      // active-set threshold
  int martensite_literal;           // reading A3
  int init_ba_steps;                // reading A6
};

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

constexpr float XMAX = 0.9f;        // bound on X_alpha used throughout Sec. 2.2
constexpr float INV_XMAX = 1.0f / 0.9f;

// ------------------------------------------------------------ SFU wrappers
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

// ------------------------------------------------------------ equilibria
// eq:equilibrium_phase_as
__device__ __forceinline__ float xalpha_eq(const ModelConst& m, float T) {
  if (T < m.T_as_end) return XMAX;
  if (T <= m.T_as_start) return 1.0f - sfu_ex2(m.kaeq_l2 * (T - m.T_as_start));
  return 0.0f;
}

// eq:equilibrium_phase_am0, third branch at T > T_am,start and capped at 0.9
__device__ __forceinline__ float xam0_eq(const ModelConst& m, float T) {
  if (T < m.T_inf) return XMAX;
  if (T <= m.T_am_start) return fminf(1.0f - sfu_ex2(m.kam_l2 * (T - m.T_am_start)), XMAX);
  return 0.0f;
}

// eq:liquid_fraction
__device__ __forceinline__ float liquid_fraction(const ModelConst& m, float T) {
  if (T < m.T_s) return 0.0f;
  if (T > m.T_l) return 1.0f;
  return (T - m.T_s) * m.inv_mushy;
}

// k_as(T) = k1 / (1 + exp(-k3 (T - k2)))
__device__ __forceinline__ float k_alpha_s(const ModelConst& m, float T) {
  return m.k1 * sfu_rcp(1.0f + sfu_ex2(m.k3_l2 * (m.k2 - T)));
}

// log2(1 + 2^y) without overflow
__device__ __forceinline__ float softplus2(float y) {
  return y > 0.0f ? y + sfu_lg2(1.0f + sfu_ex2(-y)) : sfu_lg2(1.0f + sfu_ex2(y));
}

// One step of eq:analytical_solution_beta in log2 form.  With xi = X / D,
// u = (xi / (1 - xi))^(1/c) grows by D k dt / c per step at constant k, and
// X^{n+1} = D / (1 + w^-c), w = u + D k dt / c.  lX is log2 X^n (-inf for
// X = 0); returns log2 X^{n+1}.  The log form keeps values far below the FP32
// range (X~ ~ 1e-70 after one step at 1200 K) representable.
__device__ __forceinline__ float logistic_step_log2(float lX, float D, float k, float c,
                                                    float inv_c, float dt) {
  const float lD = sfu_lg2(D);
  float u = 0.0f;
  if (lX > -1.0e30f) {
    const float lxi = lX - lD;
    const float xi = sfu_ex2(lxi);
    u = sfu_ex2((lxi - sfu_lg2(1.0f - xi)) * inv_c);
  }
  const float w = fmaf(D * k * dt, inv_c, u);
  return lD - softplus2(-c * sfu_lg2(w));
}

// ---------------------------------------------------------- correction g
// eq:explicit_correction: clamp negatives, rescale X_alpha > 0.9 keeping the
// ratio, alpha_s regularisation above T_as,start (clamped at 0), martensite
// dissolution if X_alpha > X_alpha^eq, martensite formation below T_am,start.
template <typename FT>
__device__ __forceinline__ void correct(const ModelConst& m, float T, FT& xas, FT& xam) {
  xas = xas > FT(0) ? xas : FT(0);
  xam = xam > FT(0) ? xam : FT(0);
  const FT xa = xas + xam;
  if (xa > FT(0.9)) {
    const FT s = FT(0.9) / xa;
    xas *= s;
    xam *= s;
  }
  if (T > m.T_as_start) {
    const float cap = fmaxf(XMAX * (m.T_cap0 - T) * m.inv_T_reg, 0.0f);
    if (xas > FT(cap)) xas = FT(cap);
  }
  const float xeq = xalpha_eq(m, T);
  if (xas + xam > FT(xeq)) {
    const FT v = FT(xeq) - xas;
    xam = v > FT(0) ? v : FT(0);
  }
  if (T < m.T_am_start) {
    const FT e = FT(xam0_eq(m, T)) * (FT(0.9) - xas) * FT(1.0 / 0.9);
    if (m.martensite_literal) xam = e;
    else if (e > xam) xam = e;
  }
}

// ------------------------------------------------------------ point step
// aux encodes the App. A initiation: 0 none; < 0 alpha_s -> beta in progress
// with aux = log2 X~_beta; > 0 (1.0) persisted beta -> alpha_s (init_ba_steps).
template <typename FT>
__device__ __forceinline__ void point_step(const ModelConst& m, float T0, float T1, float dt,
                                           FT& xas_io, FT& xam_io, float& aux) {
  const FT xas = xas_io, xam = xam_io;
  const FT xa = xas + xam;
  const float xeq0 = xalpha_eq(m, T0);
  const float k = k_alpha_s(m, T0);
  const float kb = m.f * k;

  bool a5 = aux < 0.0f, a6 = aux > 0.0f;
  if (a5 && !(xa > FT(xeq0))) a5 = false;
  if (a6 && !(xa < FT(xeq0))) a6 = false;
  const bool enter5 = !a5 && !a6 && xa > FT(xeq0) && FT(0.9) - xa <= FT(0) && xam == FT(0);

  FT nas, nam;
  float L = 0.0f;
  if (a5 || enter5) {
    // App. A: X~ = X_beta - 0.1, equilibrium D = X_beta^eq - 0.1, rate k_beta
    const float D = XMAX - xeq0;
    L = logistic_step_log2(a5 ? aux : -INFINITY, D, kb, m.c_b, m.inv_c_b, dt);
    nas = FT(0.9) - FT(sfu_ex2(L));
    nam = xam;
    a5 = true;
  } else if (xa < FT(xeq0) && (xas == FT(0) || a6)) {
    // reading A6: beta -> alpha_s initiation, D = X_alpha^eq - X_am, alpha_m frozen
    const float D = float(FT(xeq0) - xam);
    const float las = xas > FT(0) ? sfu_lg2(float(xas)) : -INFINITY;
    float r2 = 0.0f;
    if (xam > FT(0)) r2 = k * sfu_ex2(m.pa * las + m.qa * sfu_lg2(float(xam)));
    const float lX = logistic_step_log2(las, D, k, m.c_as, m.inv_c_as, dt);
    nas = FT(sfu_ex2(lX)) + FT(dt * r2);
    nam = xam - FT(dt * r2);
    if (m.init_ba_steps) a6 = true;
  } else {
    // eq:explicit_integration with the rates at T^n.  r1 and r3 exclude each
    // other and share one lg2 / lg2 / ex2 triple.
    const bool lo = xa < FT(xeq0), hi = xa > FT(xeq0);
    float d_as = 0.0f, d_am = 0.0f;
    float las = 0.0f;
    if (lo || xam > FT(0)) las = sfu_lg2(float(xas));
    if (lo) {
      d_as = k * sfu_ex2(m.pa * las + m.qa * sfu_lg2(float(FT(xeq0) - xa)));
    } else if (hi) {
      const FT gap = FT(0.9) - xa;
      const float lg = gap > FT(0) ? sfu_lg2(float(gap)) : -INFINITY;
      d_as = -kb * sfu_ex2(m.pb * lg + m.qb * sfu_lg2(float(xa - FT(xeq0))));
    }
    if (xam > FT(0)) {
      const float r2 = k * sfu_ex2(m.pa * las + m.qa * sfu_lg2(float(xam)));
      d_as += r2;
      d_am = -r2;
    }
    nas = xas + FT(dt * d_as);
    nam = xam + FT(dt * d_am);
  }

  const FT before = nas;
  correct<FT>(m, T1, nas, nam);

  if (a5) {
    const float xt = sfu_ex2(L);
    if (nas < before) a5 = false;  // the regularisation cap won
    else if (xt * dt > m.init_exit && xt >= m.init_exit_floor) a5 = false;
  } else if (a6) {
    const float xs = float(nas);
    if (xs * dt > m.init_exit && xs >= m.init_exit_floor) a6 = false;
  }
  aux = a5 ? L : (a6 ? 1.0f : 0.0f);
  xas_io = nas;
  xam_io = nam;
}

// A point may skip a step (active set, reading A9) when both temperatures are
// below T_thr and martensite formation at T1 would be a no-op.
template <typename FT>
__device__ __forceinline__ bool step_is_noop(const ModelConst& m, float T0, float T1, FT xas,
                                             FT xam, float aux) {
  if (!(T0 < m.T_thr && T1 < m.T_thr) || aux != 0.0f) return false;
  if (!(T1 < m.T_am_start)) return true;
  const FT e = FT(xam0_eq(m, T1)) * (FT(0.9) - xas) * FT(1.0 / 0.9);
  return xam >= e;
}

// ------------------------------------------------------ moving point source
// One source of the table for one time level (see ms_heat_source in ms.h),
// in the source's own frame: along = x . u, across = x . (u_y, -u_x).
struct SrcEntry {
  float s_xi;        // source position projected on u
  float s_pp;        // source position projected on (u_y, -u_x)
  float ux, uy;      // direction
  float cR;          // -v / (2 alpha) * log2(e)
  float lC;          // log2(A P / (2 pi k) * interlayer scale); -inf when 0
  float pad0, pad1;
};

struct SrcLevel {
  int n;             // started sources of the current layer at this level
  int axis;          // 1: every started source moves along +-(u0x, u0y)
  float z_surf;      // current layer surface (all its sources sit on it)
  float T0, T_max;
  float u0x, u0y;    // common axis when axis == 1
  float pad;
};

// 1 / (1 + a) for a in [0, 1] on the FMA pipe: a least-squares quartic
// (relative error 3e-4) refined by one Newton step (1.7e-7).  The
// MS_RCP_MODE = 1 tuning build uses it for every second source, to share the
// reciprocals between the SFU and the FMA pipe.
__device__ __forceinline__ float rcp1p_fma(float a) {
  float y = fmaf(fmaf(fmaf(fmaf(0.15224367380142212f, a, -0.5328531265258789f), a,
                           0.8658891320228577f), a, -0.9848334193229675f), a,
                 0.999702513217926f);
  const float e = fmaf(-a, y, 1.0f - y);  // 1 - (1 + a) y
  return fmaf(y, e, y);
}

// Contribution of one source to a point whose offset from the source is xi
// along the source's direction and whose squared distance from the path's
// line is perp2 (the squared depth below the surface plus 1e-30 is part of
// perp2, which keeps R > 0 and sends R = 0 to the T_max cap):
//   A P / (2 pi k R) exp(-v (R + xi) / (2 alpha)).
// Behind the source (xi < 0) R + xi cancels; it is computed there as
// perp^2 / (R + |xi|), algebraically equal and free of cancellation, so far
// receding sources keep full FP32 accuracy.
template <bool FMA_RCP>
__device__ __forceinline__ float source_term_frame(float xi, float perp2, float cR, float lC) {
  const float r2 = fmaf(xi, xi, perp2);
  const float rinv = sfu_rsqrt(r2);
  const float w = fmaf(r2, rinv, fabsf(xi));          // R + |xi|
  const float inv_w = FMA_RCP ? rcp1p_fma(fabsf(xi) * rinv) * rinv : sfu_rcp(w);
  const float rpx = xi >= 0.0f ? w : perp2 * inv_w;
  return rinv * sfu_ex2(fmaf(cR, rpx, lC));
}

// General frame: the point (px, py) projected on the source's own axes.
template <bool FMA_RCP>
__device__ __forceinline__ float source_term(const SrcEntry& e, float px, float py, float dz2) {
  const float xi = fmaf(px, e.ux, fmaf(py, e.uy, -e.s_xi));
  const float pp = fmaf(px, e.uy, fmaf(py, -e.ux, -e.s_pp));
  return source_term_frame<FMA_RCP>(xi, fmaf(pp, pp, dz2), e.cR, e.lC);
}

// Common-axis frame: pa, pb are the point's coordinates along and across the
// level's axis u0; the entry holds the sign s of u . u0 in ux, s times the
// source's along-axis coordinate in s_xi and its across-axis coordinate in s_pp.
template <bool FMA_RCP>
__device__ __forceinline__ float source_term_axis(const SrcEntry& e, float pa, float pb,
                                                  float dz2) {
  const float xi = fmaf(e.ux, pa, -e.s_xi);
  const float pp = pb - e.s_pp;
  return source_term_frame<FMA_RCP>(xi, fmaf(pp, pp, dz2), e.cR, e.lC);
}

}  // namespace ms
