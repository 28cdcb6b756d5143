/*
 * FP64 CPU oracle of the Ti-6Al-4V phase model (Proell et al., arXiv 2402.17580).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no source, header, constant table or helper with the CUDA path.
 *
 * Plain, slow, obviously correct: one point at a time, double precision,
 * libm exp/log/pow/sqrt, the steps in the paper's order.  OpenMP only splits
 * the independent points (Sec. 3: the model is decoupled in space).
 *
 * Paper passages followed (section / equation label of the LaTeX source):
 *   liquid fraction g(T)                   Sec. 2.1, eq:liquid_fraction
 *   X_sol = 1 - g, X_liq = g               Sec. 2.2 (after eq:phase_continuity_*)
 *   X_alpha^eq(T)                          Sec. 2.2, eq:equilibrium_phase_as
 *   X_alpha_m,0^eq(T)                      Sec. 2.2, eq:equilibrium_phase_am0
 *   X_alpha_m^eq(T, X_as)                  Sec. 2.2, eq:equilibrium_phase_am
 *   diffusive rates                        Sec. 2.2, eq:beta_to_alpha_s,
 *                                          eq:alpha_m_to_alpha_s, eq:alpha_s_to_beta
 *   k_as(T), k_beta(T)                     Sec. 2.2 (rate constants after the rates)
 *   instantaneous martensite               Sec. 2.2, eq:inst_martensite_formation,
 *                                          eq:inst_martensite_dissolution
 *   alpha_s regularisation (T_reg)         Sec. 2.2 (after eq:inst_martensite_dissolution)
 *   Table 2 / Table 3 constants            tab:micro_parameters, tab:micro_parameters_diffusion
 *   split m_diff + m_inst                  Sec. 3.1, eq:diff_inst_split
 *   explicit Euler + correction g          Sec. 3.1, eq:explicit_integration,
 *                                          eq:explicit_correction (and the text after it)
 *   X_beta post-processing                 Sec. 3.1, eq:time_integration_beta_postprocess
 *   analytical initiation                  Appendix A, eq:analytical_solution_beta
 *   temperature cap T_max = T_v + 1000 K   Sec. 2.1 (after eq:bc_evaporation)
 *
 * Readings where the paper is silent, garbled or inconsistent (each one is
 * listed with its justification in the design notes at the repository root):
 *   A1  eq:equilibrium_phase_am0's third branch reads "T > T_as,start"; taken as
 *       T > T_am,start so the function is defined everywhere and continuous at
 *       T_am,start.
 *   A2  piecewise definitions kept literally; X_am,0^eq additionally capped at 0.9.
 *   A3  instantaneous martensite formation is formation-only by default:
 *       X_am <- max(X_am, X_am^eq); flag MARTENSITE_LITERAL gives X_am <- X_am^eq.
 *   A4  the regularisation cap applies for T > T_as,start and is clamped at 0,
 *       so X_as = 0 for T >= T_as,start + T_reg.
 *   A5  alpha_s -> beta initiation (App. A): entered when X_alpha > X_alpha^eq,
 *       0.9 - X_alpha <= 0 and X_am == 0; X~_beta is tracked in its own
 *       variable; left when X~_beta * dt > init_exit and X~_beta >= init_exit_floor,
 *       when X_alpha <= X_alpha^eq, or when the cap lowers X_as.
 *   A6  beta -> alpha_s initiation: the same closed form with D = X_alpha^eq - X_am,
 *       k~ = D k_as, c = c_as, xi = X_as / D; one step whenever X_as == 0 and
 *       X_alpha < X_alpha^eq (flag INIT_BA_STEPS keeps it with the A5 exit rule).
 *   A7  Rosenthal source at distance 0: T = T_max.
 *   A8  rates at T^n, correction g at T^{n+1}.
 *   A11 rescaling by 0.9 / X_alpha when X_alpha > 0.9.
 *   A13 sum of the four fractions is 1; melting forces X_as = X_am = 0.
 *   A14 0^p = 0 for p > 0.
 *
 * The moving heat source (superposed Rosenthal point sources) is the synthetic
 * temperature driver of the workloads, not part of the paper's method; its
 * formula is the classical thick-plate moving point source,
 *   T - T0 = A P / (2 pi k R) * exp(-v (R + xi) / (2 alpha)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- parameter vector (indices shared with oracle/__init__.py only) ---- */
enum {
  P_T_S = 0,        /* solidus temperature, Table 1/2: 1878 K              */
  P_T_L,            /* liquidus temperature, Table 1/2: 1928 K             */
  P_T_AS_START,     /* Table 2: 1273 K                                       */
  P_T_AS_END,       /* Table 2: 935 K                                        */
  P_T_AM_START,     /* Table 2: 848 K                                        */
  P_T_INF,          /* Table 2: 293 K                                        */
  P_K_ALPHA_EQ,     /* Table 2: 0.0068 1/K                                   */
  P_K_AM_EQ,        /* Table 2: 0.00415 1/K                                  */
  P_C_AS,           /* Table 3: 2.51                                         */
  P_C_B,            /* Table 3: 11.0                                         */
  P_K1,             /* Table 3: 0.294 1/s                                    */
  P_K2,             /* Table 3: 850 K                                        */
  P_K3,             /* Table 3: 0.0337 1/K                                   */
  P_F,              /* Table 3: 3.8                                          */
  P_T_REG,          /* Sec. 2.2: 100 K                                       */
  P_INIT_EXIT,      /* App. A: leave initiation once X~ * dt > 1e-15         */
  P_INIT_EXIT_FLOOR,/* reading A5: and X~ >= this floor                      */
  P_MART_LITERAL,   /* reading A3 flag (0/1)                                 */
  P_INIT_BA_STEPS,  /* reading A6 flag (0/1)                                 */
  P_INTEGRATOR,     /* 0 explicit (eq:explicit_integration), 1 implicit
                       Crank-Nicolson (eq:implicit_integration), Sec. 3       */
  P_DT_SUB,         /* implicit: largest substep, Sec. 3: 0.01 s (<= 0: none) */
  P_FP_EPS_ABS,     /* implicit: WRMS absolute tolerance, Sec. 3: 1e-10       */
  P_FP_EPS_REL,     /* implicit: WRMS relative tolerance, Sec. 3: 1e-3        */
  P_FP_MAX_ITER,    /* implicit: cap on the fixed-point iterations            */
  P_COUNT
};

#define XMAX 0.9 /* the 0.9 bound on X_alpha that the paper uses throughout Sec. 2.2 */

enum { MODE_NONE = 0, MODE_AS_TO_B = 1, MODE_B_TO_AS = 2 };

/* eq:liquid_fraction */
static double liquid_fraction(const double *p, double T) {
  if (T < p[P_T_S]) return 0.0;
  if (T > p[P_T_L]) return 1.0;
  return (T - p[P_T_S]) / (p[P_T_L] - p[P_T_S]);
}

/* eq:equilibrium_phase_as */
static double xalpha_eq(const double *p, double T) {
  if (T < p[P_T_AS_END]) return XMAX;
  if (T <= p[P_T_AS_START]) return 1.0 - exp(-p[P_K_ALPHA_EQ] * (p[P_T_AS_START] - T));
  return 0.0;
}

/* eq:equilibrium_phase_am0 with readings A1 (upper branch at T_am,start) and A2 (cap 0.9) */
static double xam0_eq(const double *p, double T) {
  if (T < p[P_T_INF]) return XMAX;
  if (T <= p[P_T_AM_START]) {
    double v = 1.0 - exp(-p[P_K_AM_EQ] * (p[P_T_AM_START] - T));
    return v < XMAX ? v : XMAX;
  }
  return 0.0;
}

/* eq:equilibrium_phase_am */
static double xam_eq(const double *p, double T, double xas) {
  return xam0_eq(p, T) * (XMAX - xas) / XMAX;
}

/* k_as(T) = k1 / (1 + exp(-k3 (T - k2))), Sec. 2.2 */
static double k_alpha_s(const double *p, double T) {
  return p[P_K1] / (1.0 + exp(-p[P_K3] * (T - p[P_K2])));
}

/* x^e for x >= 0 and e > 0, with 0^e = 0 (reading A14) */
static double powpos(double x, double e) { return x > 0.0 ? pow(x, e) : 0.0; }

/* Diffusive part m_diff(T, m) of eq:diff_inst_split, built from
 * eq:beta_to_alpha_s (r1), eq:alpha_m_to_alpha_s (r2), eq:alpha_s_to_beta (r3). */
static void rates(const double *p, double T, double xas, double xam, double *das, double *dam) {
  double xeq = xalpha_eq(p, T);
  double k = k_alpha_s(p, T), kb = p[P_F] * k;
  double xa = xas + xam;
  double ca = p[P_C_AS], cb = p[P_C_B];
  double r1 = 0.0, r2 = 0.0, r3 = 0.0;
  if (xa < xeq) r1 = k * powpos(xas, (ca - 1.0) / ca) * powpos(xeq - xa, (ca + 1.0) / ca);
  if (xam > 0.0) r2 = k * powpos(xas, (ca - 1.0) / ca) * powpos(xam, (ca + 1.0) / ca);
  if (xa > xeq) r3 = kb * powpos(XMAX - xa, (cb - 1.0) / cb) * powpos(xa - xeq, (cb + 1.0) / cb);
  *das = r1 + r2 - r3;
  *dam = -r2;
}

/* One step of the closed form eq:analytical_solution_beta for the generalised
 * logistic ODE  d(xi)/dt = k~ xi^((c-1)/c) (1-xi)^((c+1)/c),  xi = X / D,
 * k~ = D k, exact for constant k~ (App. A):
 *   X^{n+1} = D [1 + (c / (D k dt + c (xi_n / (1 - xi_n))^(1/c)))^c]^(-1). */
static double logistic_step(double X, double D, double k, double c, double dt) {
  double xi = X / D;
  double u = xi > 0.0 ? pow(xi / (1.0 - xi), 1.0 / c) : 0.0;
  double w = c / (D * k * dt + c * u);
  return D / (1.0 + pow(w, c));
}

/* Correction function g(T, m) of eq:explicit_correction: clamp, rescale
 * (A11), regularisation (A4), instantaneous dissolution
 * (eq:inst_martensite_dissolution), instantaneous formation
 * (eq:inst_martensite_formation, reading A3). */
static void correct(const double *p, double T, double *xas_io, double *xam_io) {
  double xas = *xas_io, xam = *xam_io;
  if (xas < 0.0) xas = 0.0;
  if (xam < 0.0) xam = 0.0;
  double xa = xas + xam;
  if (xa > XMAX) {
    double s = XMAX / xa;
    xas *= s;
    xam *= s;
  }
  if (T > p[P_T_AS_START]) {
    double cap = XMAX * (p[P_T_AS_START] + p[P_T_REG] - T) / p[P_T_REG];
    if (cap < 0.0) cap = 0.0;
    if (xas > cap) xas = cap;
  }
  double xeq = xalpha_eq(p, T);
  if (xas + xam > xeq) {
    double v = xeq - xas;
    xam = v > 0.0 ? v : 0.0;
  }
  if (T < p[P_T_AM_START]) {
    double e = xam_eq(p, T, xas);
    if (p[P_MART_LITERAL] != 0.0) xam = e;
    else if (e > xam) xam = e;
  }
  *xas_io = xas;
  *xam_io = xam;
}

/* One explicit step n -> n+1 of one point (eq:explicit_integration followed by
 * eq:explicit_correction), rates at T0 = T^n and g at T1 = T^{n+1} (A8),
 * with the App. A initiations (A5, A6). */
static void point_step(const double *p, double T0, double T1, double dt,
                       double *xas_io, double *xam_io, double *xt_io, int32_t *mode_io) {
  double xas = *xas_io, xam = *xam_io, xt = *xt_io;
  int32_t mode = *mode_io;
  double xa = xas + xam;
  double xeq0 = xalpha_eq(p, T0);
  double k = k_alpha_s(p, T0), kb = p[P_F] * k;
  double nas, nam;

  if (mode == MODE_AS_TO_B && !(xa > xeq0)) mode = MODE_NONE;
  if (mode == MODE_B_TO_AS && !(xa < xeq0)) mode = MODE_NONE;
  if (mode == MODE_NONE && xa > xeq0 && XMAX - xa <= 0.0 && xam == 0.0) {
    mode = MODE_AS_TO_B;
    xt = 0.0;
  }

  if (mode == MODE_AS_TO_B) {
    /* App. A: shifted beta fraction X~ = X_beta - 0.1, equilibrium
     * D = X_beta^eq - 0.1 = (1 - X_alpha^eq) - 0.1, rate k_beta. */
    double D = (1.0 - xeq0) - 0.1;
    xt = logistic_step(xt, D, kb, p[P_C_B], dt);
    nas = XMAX - xt;
    nam = xam;
  } else if (xa < xeq0 && (xas == 0.0 || mode == MODE_B_TO_AS)) {
    /* reading A6: beta -> alpha_s initiation, alpha_m frozen over the step */
    double D = xeq0 - xam;
    double ca = p[P_C_AS];
    double r2 = xam > 0.0 ? k * powpos(xas, (ca - 1.0) / ca) * powpos(xam, (ca + 1.0) / ca) : 0.0;
    nas = logistic_step(xas, D, k, ca, dt) + dt * r2;
    nam = xam - dt * r2;
    if (p[P_INIT_BA_STEPS] != 0.0) mode = MODE_B_TO_AS;
  } else {
    double das, dam;
    rates(p, T0, xas, xam, &das, &dam);
    nas = xas + dt * das;
    nam = xam + dt * dam;
  }

  double before = nas;
  correct(p, T1, &nas, &nam);

  if (mode == MODE_AS_TO_B) {
    if (nas < before) mode = MODE_NONE; /* the regularisation cap won */
    else if (xt * dt > p[P_INIT_EXIT] && xt >= p[P_INIT_EXIT_FLOOR]) mode = MODE_NONE;
  } else if (mode == MODE_B_TO_AS) {
    if (nas * dt > p[P_INIT_EXIT] && nas >= p[P_INIT_EXIT_FLOOR]) mode = MODE_NONE;
  }
  *xas_io = nas;
  *xam_io = nam;
  *xt_io = mode == MODE_AS_TO_B ? xt : 0.0;
  *mode_io = mode;
}

/* One Crank-Nicolson step (eq:implicit_integration + eq:implicit_correction)
 * of the diffusive rates from T0 to T1, solved by the fixed-point iteration
 * eq:implicit_fp_iteration in the order of the paper's implicit algorithm:
 * rates at (T0, m^n); m_0 = g(T1, m^n) (reading I1); then
 *   m_{i+1} = g(T1, m^n + dt/2 (mdot(T1, m_i) + mdot(T0, m^n)))
 * until the WRMS norm of dt/2 (mdot(T1, m_{i+1}) - mdot(T1, m_i)) is below 1,
 * with w_j = 1 / (eps_abs + |m_{i+1,j}| eps_rel) (reading A10; the norm is
 * taken without the root, as the paper writes it).  Returns the iterations
 * done; *converged is 0 if the cap was reached. */
static int cn_step(const double *p, double T0, double T1, double dt, double *xas_io,
                   double *xam_io, int *converged) {
  const double xas = *xas_io, xam = *xam_io;
  double das0, dam0;
  rates(p, T0, xas, xam, &das0, &dam0);
  double mas = xas, mam = xam;
  correct(p, T1, &mas, &mam);
  double das, dam;
  rates(p, T1, mas, mam, &das, &dam);
  const int max_iter = (int)p[P_FP_MAX_ITER];
  int it = 0;
  *converged = 0;
  while (it < max_iter) {
    double nas = xas + 0.5 * dt * (das + das0);
    double nam = xam + 0.5 * dt * (dam + dam0);
    correct(p, T1, &nas, &nam);
    double das1, dam1;
    rates(p, T1, nas, nam, &das1, &dam1);
    const double ras = 0.5 * dt * (das1 - das) / (p[P_FP_EPS_ABS] + fabs(nas) * p[P_FP_EPS_REL]);
    const double ram = 0.5 * dt * (dam1 - dam) / (p[P_FP_EPS_ABS] + fabs(nam) * p[P_FP_EPS_REL]);
    const double e = 0.5 * (ras * ras + ram * ram);
    mas = nas;
    mam = nam;
    das = das1;
    dam = dam1;
    ++it;
    if (e < 1.0) {
      *converged = 1;
      break;
    }
  }
  *xas_io = mas;
  *xam_io = mam;
  return it;
}

/* Substeps of a step of size dt (Sec. 3): ceil(dt / dt_sub), at least 1; the
 * small offset keeps an exact multiple (0.1 / 0.01) from rounding up. */
static int64_t n_substeps(const double *p, double dt) {
  if (!(p[P_DT_SUB] > 0.0)) return 1;
  const double r = ceil(dt / p[P_DT_SUB] - 1e-9);
  return r < 1.0 ? 1 : (int64_t)r;
}

/* One implicit step n -> n+1 of one point: subcycles of at most dt_sub with
 * the temperature linear in time between T0 and T1 (reading I3); in each
 * substep the App. A closed-form initiation takes precedence exactly as in
 * the explicit step (Crank-Nicolson cannot leave X_as = 0 or X_alpha = 0.9
 * either, reading I2), otherwise cn_step. */
static void point_step_implicit(const double *p, double T0, double T1, double dt,
                                double *xas, double *xam, double *xt, int32_t *mode,
                                int64_t *iters, int64_t *unconverged) {
  const int64_t ns = n_substeps(p, dt);
  const double h = dt / (double)ns;
  for (int64_t s = 0; s < ns; ++s) {
    const double Ta = T0 + (T1 - T0) * ((double)s / (double)ns);
    const double Tb = T0 + (T1 - T0) * ((double)(s + 1) / (double)ns);
    const double xa = *xas + *xam, xeq0 = xalpha_eq(p, Ta);
    int init = 0;
    if (*mode == MODE_AS_TO_B && xa > xeq0) init = 1;
    if (*mode == MODE_B_TO_AS && xa < xeq0) init = 1;
    if (xa > xeq0 && XMAX - xa <= 0.0 && *xam == 0.0) init = 1;
    if (xa < xeq0 && *xas == 0.0) init = 1;
    if (init) {
      point_step(p, Ta, Tb, h, xas, xam, xt, mode);
    } else {
      int conv;
      *mode = MODE_NONE;
      *xt = 0.0;
      const int it = cn_step(p, Ta, Tb, h, xas, xam, &conv);
      if (iters) *iters += it;
      if (unconverged && !conv) *unconverged += 1;
    }
  }
}

/* One step with the configured integrator. */
static void advance(const double *p, double T0, double T1, double dt, double *xas, double *xam,
                    double *xt, int32_t *mode) {
  if (p[P_INTEGRATOR] != 0.0)
    point_step_implicit(p, T0, T1, dt, xas, xam, xt, mode, NULL, NULL);
  else
    point_step(p, T0, T1, dt, xas, xam, xt, mode);
}

/* ------------------------- exported: model pieces ------------------------- */

double orc_liquid_fraction(const double *p, double T) { return liquid_fraction(p, T); }
double orc_xalpha_eq(const double *p, double T) { return xalpha_eq(p, T); }
double orc_xam0_eq(const double *p, double T) { return xam0_eq(p, T); }
double orc_xam_eq(const double *p, double T, double xas) { return xam_eq(p, T, xas); }
double orc_k_alpha_s(const double *p, double T) { return k_alpha_s(p, T); }
double orc_logistic_step(double X, double D, double k, double c, double dt) {
  return logistic_step(X, D, k, c, dt);
}
void orc_rates(const double *p, double T, double xas, double xam, double *das, double *dam) {
  rates(p, T, xas, xam, das, dam);
}
void orc_correct(const double *p, double T, double *xas, double *xam) { correct(p, T, xas, xam); }
int orc_cn_step(const double *p, double T0, double T1, double dt, double *xas, double *xam,
                int *converged) {
  return cn_step(p, T0, T1, dt, xas, xam, converged);
}
int64_t orc_n_substeps(const double *p, double dt) { return n_substeps(p, dt); }

/* X_beta and X_liq from the state and the temperature:
 * eq:time_integration_beta_postprocess with X_sol = 1 - g(T). */
void orc_fractions(const double *p, int64_t n, const double *xas, const double *xam,
                   const double *T, double *xbeta, double *xliq) {
  for (int64_t i = 0; i < n; ++i) {
    double g = liquid_fraction(p, T[i]);
    xbeta[i] = (1.0 - g) - xas[i] - xam[i];
    if (xliq) xliq[i] = g;
  }
}

/* n_steps explicit steps of n independent points with given temperature
 * histories: T[s * n + i] is T^{s} of point i, s = 0 .. n_steps (Algorithm 1
 * with the local step of Algorithm 2). */
void orc_run_temps(const double *p, int64_t n, int64_t n_steps, double dt, const double *T,
                   double *xas, double *xam, double *xt, int32_t *mode) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t s = 0; s < n_steps; ++s)
      advance(p, T[s * n + i], T[(s + 1) * n + i], dt, &xas[i], &xam[i], &xt[i], &mode[i]);
  }
}

/* --------------------- synthetic moving heat source ---------------------- */
/* spec: A, k, alpha, T0, T_max, t_offset, z_tol
 * track (8 doubles): x0, y0, ux, uy, v, P, t_start, layer
 * layer (4 doubles): z_surface, t_begin, t_scan_end, t_end */
enum { S_A = 0, S_K, S_ALPHA, S_T0, S_TMAX, S_TOFF, S_ZTOL, S_COUNT };
enum { TR_X0 = 0, TR_Y0, TR_UX, TR_UY, TR_V, TR_P, TR_TS, TR_LAYER, TR_COUNT };
enum { LY_Z = 0, LY_TB, LY_TSE, LY_TE, LY_COUNT };

static int32_t layer_at(const double *layers, int32_t n_layers, double tl) {
  int32_t l = 0;
  for (int32_t j = 0; j < n_layers; ++j)
    if (layers[j * LY_COUNT + LY_TB] <= tl) l = j;
  return l;
}

/* temperature of one point at specimen-local time tl; *active = 0 when the
 * point lies above the current layer's surface (not yet deposited). */
static double source_temperature(const double *spec, const double *tracks, int32_t n_tracks,
                                 const double *layers, int32_t n_layers, double x, double y,
                                 double z, double tl, int *active) {
  int32_t l = layer_at(layers, n_layers, tl);
  const double *L = layers + (int64_t)l * LY_COUNT;
  *active = z <= L[LY_Z] + spec[S_ZTOL];
  double scale = 1.0;
  if (tl > L[LY_TSE]) {
    double span = L[LY_TE] - L[LY_TSE];
    scale = span > 0.0 ? 1.0 - (tl - L[LY_TSE]) / span : 0.0;
    if (scale < 0.0) scale = 0.0;
  }
  double sum = 0.0;
  for (int32_t j = 0; j < n_tracks; ++j) {
    const double *tr = tracks + (int64_t)j * TR_COUNT;
    if ((int32_t)tr[TR_LAYER] != l || tl < tr[TR_TS]) continue;
    double travel = tr[TR_V] * (tl - tr[TR_TS]);
    double dx = x - (tr[TR_X0] + tr[TR_UX] * travel);
    double dy = y - (tr[TR_Y0] + tr[TR_UY] * travel);
    double dz = z - L[LY_Z];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    if (R == 0.0) return spec[S_TMAX]; /* reading A7 */
    double xi = dx * tr[TR_UX] + dy * tr[TR_UY];
    double q = spec[S_A] * tr[TR_P] / (2.0 * M_PI * spec[S_K] * R);
    sum += q * exp(-tr[TR_V] * (R + xi) / (2.0 * spec[S_ALPHA]));
  }
  double T = spec[S_T0] + scale * sum;
  return T < spec[S_TMAX] ? T : spec[S_TMAX];
}

/* temperatures at global time t of n points (used by pins and tests) */
void orc_temperature(const double *spec, const double *tracks, int32_t n_tracks,
                     const double *layers, int32_t n_layers, int64_t n, const double *x,
                     const double *y, const double *z, double t, double *T, int32_t *active) {
  for (int64_t i = 0; i < n; ++i) {
    int a;
    T[i] = source_temperature(spec, tracks, n_tracks, layers, n_layers, x[i], y[i], z[i],
                              t - spec[S_TOFF], &a);
    if (active) active[i] = a;
  }
}

/* Steps n0 .. n0 + n_steps - 1 (time level t_n = n * dt) of n points at the
 * given coordinates under the moving source.  The final temperature is
 * returned in T_last (for X_beta and X_liq).  Points above the current layer
 * surface are not advanced. */
void orc_run_track(const double *p, const double *spec, const double *tracks, int32_t n_tracks,
                   const double *layers, int32_t n_layers, int64_t n, const double *x,
                   const double *y, const double *z, int64_t n0, int64_t n_steps, double dt,
                   double *xas, double *xam, double *xt, int32_t *mode, double *T_last) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    int a0, a1;
    double T0 = source_temperature(spec, tracks, n_tracks, layers, n_layers, x[i], y[i], z[i],
                                   (double)n0 * dt - spec[S_TOFF], &a0);
    for (int64_t s = 0; s < n_steps; ++s) {
      double t1 = (double)(n0 + s + 1) * dt - spec[S_TOFF];
      double T1 = source_temperature(spec, tracks, n_tracks, layers, n_layers, x[i], y[i], z[i],
                                     t1, &a1);
      if (a1) advance(p, T0, T1, dt, &xas[i], &xam[i], &xt[i], &mode[i]);
      T0 = T1;
    }
    if (T_last) T_last[i] = T0;
  }
}

/* The window form of the hybrid path (an extension of Sec. 3, not in the
 * paper) for a network whose output is zero, so that the window machinery is
 * checked apart from the network's arithmetic.  Steps are taken in windows of
 * window x stride levels from n0; the window's samples are its levels
 * stride, 2 stride, ..., window x stride.  A full-length window whose start
 * temperature and samples all stay more than band_half away from
 * T_am,start, T_as,end, T_as,start and T_as,start + T_reg and at or below
 * T_s - band_half, whose consecutive samples (the start included) differ by
 * at most band_half, with (for stride > 1) no three consecutive samples
 * whose parabola has its vertex within two spacings of the middle one and
 * a minimum below T_am,start or a maximum above T_as,end (there the
 * correction g depends on the path's extreme, which can lie between
 * samples), with no App. A initiation running at its start and the
 * point below the surface on every level, applies only the correction g at
 * its samples in turn (no diffusion); every other window takes the explicit
 * steps at every level.  n_mlp[i] counts the first kind of window per point.
 * Before either, a point on the alpha_s plateau's fixed point (X_as = 0.9,
 * X_am = 0, no initiation) whose start and sample temperatures all stay
 * below T_as,end keeps its state over a full-length window: there
 * X_alpha^eq = 0.9, no rate acts and the correction changes nothing, so the
 * explicit steps are the identity (the hybrid kernel skips such windows);
 * n_fixed[i] (if given) counts them.  Points form groups of `group`
 * consecutive points (the hybrid kernel's 128-point tiles): when a window
 * sends any point of a group with a level below the surface to the
 * explicit steps, every point of the group that would apply g only takes
 * the explicit steps too (group = 1: each point decides alone). */
static int in_band(const double *p, double T, double h) {
  if (!(T <= p[P_T_S] - h)) return 1;
  if (fabs(T - p[P_T_AM_START]) < h || fabs(T - p[P_T_AS_END]) < h) return 1;
  if (fabs(T - p[P_T_AS_START]) < h || fabs(T - (p[P_T_AS_START] + p[P_T_REG])) < h) return 1;
  return 0;
}

/* The parabola through three equally spaced samples a, b, c: its vertex lies
 * at (a - c) / (2 k) spacings from b, k = a - 2 b + c, with the value
 * b - (c - a)^2 / (8 k).  True when the vertex lies within two spacings of b
 * and is a minimum below T_am,start (k > 0) or a maximum above T_as,end
 * (k < 0). */
static int extreme_near(const double *p, double a, double b, double c) {
  const double k = a - 2.0 * b + c, s = c - a;
  if (k == 0.0 || !(fabs(s) <= 4.0 * fabs(k))) return 0;
  const double v = b - s * s / (8.0 * k);
  return k > 0.0 ? v < p[P_T_AM_START] : v > p[P_T_AS_END];
}

void orc_run_track_windows(const double *p, const double *spec, const double *tracks,
                           int32_t n_tracks, const double *layers, int32_t n_layers, int64_t n,
                           const double *x, const double *y, const double *z, int64_t n0,
                           int64_t n_steps, double dt, int32_t window, int32_t stride,
                           double band_half, int64_t group, double *xas, double *xam, double *xt,
                           int32_t *mode, int64_t *n_mlp, int64_t *n_fixed) {
  const int64_t len = (int64_t)window * stride;
  const int64_t n_groups = (n + group - 1) / group;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t gi = 0; gi < n_groups; ++gi) {
    const int64_t i0 = gi * group, m = n - i0 < group ? n - i0 : group;
    const size_t ld = (size_t)len + 1;
    double *T = malloc(sizeof(double) * ld * (size_t)m), *Tn = malloc(sizeof(double) * (size_t)m);
    int *act = malloc(sizeof(int) * ld * (size_t)m), *kind = malloc(sizeof(int) * (size_t)m);
    for (int64_t k = 0; k < m; ++k) {
      int a0;
      const int64_t i = i0 + k;
      Tn[k] = source_temperature(spec, tracks, n_tracks, layers, n_layers, x[i], y[i], z[i],
                                 (double)n0 * dt - spec[S_TOFF], &a0);
      if (n_mlp) n_mlp[i] = 0;
      if (n_fixed) n_fixed[i] = 0;
    }
    for (int64_t w0 = 0; w0 < n_steps; w0 += len) {
      const int64_t K = n_steps - w0 < len ? n_steps - w0 : len;
      int any_explicit = 0;
      for (int64_t k = 0; k < m; ++k) {   /* kind: 0 idle, 1 fixed, 2 g only, 3 explicit */
        const int64_t i = i0 + k;
        double *Ti = T + ld * k;
        int *ai = act + ld * k, all_act = 1, any_act = 0;
        Ti[0] = Tn[k];
        for (int64_t l = 1; l <= K; ++l) {
          double tl = (double)(n0 + w0 + l) * dt - spec[S_TOFF];
          Ti[l] = source_temperature(spec, tracks, n_tracks, layers, n_layers, x[i], y[i], z[i],
                                     tl, &ai[l]);
          all_act &= ai[l];
          any_act |= ai[l];
        }
        /* the tests on the start and the samples */
        int band = in_band(p, Ti[0], band_half), cool = Ti[0] < p[P_T_AS_END];
        for (int64_t l = stride; K == len && l <= K; l += stride) {
          band |= in_band(p, Ti[l], band_half) || !(fabs(Ti[l] - Ti[l - stride]) <= band_half);
          if (stride > 1 && l >= 2 * stride)
            band |= extreme_near(p, Ti[l - 2 * stride], Ti[l - stride], Ti[l]);
          cool &= Ti[l] < p[P_T_AS_END];
        }
        if (!any_act)
          kind[k] = 0;
        else if (K == len && cool && mode[i] == MODE_NONE && xas[i] == 0.9 && xam[i] == 0.0)
          kind[k] = 1;
        else if (K == len && all_act && !band && mode[i] == MODE_NONE)
          kind[k] = 2;
        else
          kind[k] = 3;
        any_explicit |= kind[k] == 3;
        Tn[k] = Ti[K];
      }
      for (int64_t k = 0; k < m; ++k) {
        const int64_t i = i0 + k;
        const double *Ti = T + ld * k;
        const int *ai = act + ld * k;
        if (kind[k] == 1) {
          if (n_fixed) ++n_fixed[i];
        } else if (kind[k] == 2 && !any_explicit) {
          for (int64_t l = stride; l <= K; l += stride) correct(p, Ti[l], &xas[i], &xam[i]);
          if (n_mlp) ++n_mlp[i];
        } else if (kind[k] != 0) {
          for (int64_t l = 1; l <= K; ++l)
            if (ai[l]) advance(p, Ti[l - 1], Ti[l], dt, &xas[i], &xam[i], &xt[i], &mode[i]);
        }
      }
    }
    free(T);
    free(Tn);
    free(act);
    free(kind);
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the point loops (the timed CPU baseline also runs on one core). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_param_count(void) { return P_COUNT; }
