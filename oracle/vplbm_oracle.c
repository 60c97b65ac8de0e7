/*
 * vplbm_oracle.c -- plain, slow FP64 CPU implementation of the volume-penalized
 * lattice Boltzmann method (VP-LBM) of Liberge & Beghein, "About fluid forces
 * computation for Volume Penalization coupled with Lattice Boltzmann method"
 * (arXiv 2110.00967), with its two fluid-force estimators (MEM and SIM) and the
 * rigid-body equations of its sedimentation case.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU baseline
 * of the benchmark may load it.  It shares no code, header or table with the
 * CUDA path and never calls it.
 *
 * Conventions (all from Sec. 2.2 of the paper unless stated):
 *   - D2Q9, dt = dx = 1, c_s^2 = 1/3; node (i, j), x = i, y = j, i fastest.
 *   - populations f[a][j][i], a = 0..8, stored as f[(a*ny + j)*nx + i].
 *   - the stored state between steps is the PRE-collision field f^n
 *     (what Eq. eqBd produces on its left-hand side).
 *   - one time step: moments + penalized velocity (Eqs. updatestep,
 *     updatestep2, updatestep3, updatestepm), equilibrium, Guo forcing,
 *     BGK or TRT collision (Eq. TRT), MEM on the post-collision field
 *     (Eq. MMEL, Eq. fluidtorque), streaming (Eq. eqBd) and the boundary
 *     conditions of Sec. 3.1 / 3.2.  SIM (Eq. defFf and the stress formula
 *     of Sec. 2.3.2) is evaluated on the pre-collision field of the step.
 *
 * Readings of the paper taken here (where it is silent or inconsistent):
 *   R1 Guo forcing term F_a = w_a[(c_a - u)/cs2 + (c_a.u) c_a/cs4].G with G
 *      the force density rho*F; in TRT the paper multiplies all of F_a by
 *      (1 - 1/(2 tau+)) (Eq. TRT).  A second mode applies (1 - 1/(2 tau-)) to
 *      the antisymmetric part instead ("split").
 *   R2 the penalization force density is G = -rho (chi/eta)(u - u_s) (the
 *      sign of Eq. (1) and Eq. updatestep2).
 *   R3 G is evaluated in the rearranged form -(chi/eta)(j - rho u_s)/(1 + k),
 *      k = chi dt/(2 eta), which is algebraically identical to the literal one.
 *   R5 MEM uses the post-collision populations; x_Gamma is the link midpoint.
 *   R6 SIM copies f from the first fluid node met when walking from the
 *      nearest node of the integration point along the lattice direction
 *      closest to n; a point exactly half-way between nodes averages sigma
 *      over both candidates (keeps mirror-symmetric bodies symmetric).
 *   R7 the tau in the SIM stress is tau+.
 *  R10 convective outlet velocity U_c = |u_in|;  R11 inlet wall density 1.
 *  R20 a first-order SIM variant extrapolates the stress linearly to the
 *      integration point from the first two fluid nodes along the sampling
 *      direction (the paper copies it from the first, R6).
 *  R21 the "free flow" outlet of the sedimentation case (Sec. 3.2) is a
 *      zero normal gradient: the populations entering the last column from
 *      beyond the edge copy those of the column before it, after streaming.
 *  R19 the volume-integral force of Eq. Angotforce is the penalization
 *      force reversed, sum over solid nodes of rho (chi/eta)(u - u_s) (the
 *      printed formula has lost the 1/eta and writes the limit as eta to
 *      infinity); the paper reports that it fails, it is a diagnostic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* threads used by the row loops of the collision and streaming passes; the
 * result does not depend on it (no reduction runs in parallel) */
int orc_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- lattice (Fig. d2q9 and the velocity formula of Sec. 2.2) ------------ */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WGT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* boundary kinds, per side x_lo, x_hi, y_lo, y_hi */
enum { BC_PERIODIC = 0, BC_INLET = 1, BC_OUTLET = 2, BC_SYMMETRY = 3, BC_NOSLIP = 4, BC_OUTLET_FREE = 5 };
enum { COLL_BGK = 0, COLL_TRT = 1 };
enum { FORCING_PAPER = 0, FORCING_SPLIT = 1 };
enum { BODY_NONE = 0, BODY_DISK = 1, BODY_NACA = 2 };

typedef struct {
  int32_t nx, ny;
  int32_t bc[4];
  int32_t collision;
  int32_t forcing;
  double tau_plus;
  double lambda_trt;
  double eta;
  double u_in[2];
  double body_force[2]; /* uniform force density on every node */
} orc_config;

typedef struct {
  int32_t kind;
  int32_t moving; /* 1: integrate Eqs. dep1 / theta2 */
  int32_t n_sim;  /* SIM integration points */
  int32_t pad;
  double length;    /* disk diameter D or chord C */
  double thickness; /* NACA 4-digit thickness t (0.12 for NACA 0012) */
  double xg, yg;    /* disk centre / NACA pivot point (the body reference point) */
  double theta;     /* disk: rotation angle; NACA: angle of attack, nose up */
  double pivot_frac;
  double u[2];      /* rigid translational velocity */
  double omega;     /* rigid angular velocity */
  double density_ratio; /* rho_s / rho */
  double gravity[2];
} orc_body;

void orc_lattice(int32_t *cx, int32_t *cy, int32_t *opp, double *w) {
  for (int a = 0; a < Q; ++a) {
    cx[a] = CX[a];
    cy[a] = CY[a];
    opp[a] = OPP[a];
    w[a] = WGT[a];
  }
}

static inline size_t idx(const orc_config *cfg, int a, int i, int j) {
  return ((size_t)a * cfg->ny + j) * cfg->nx + i;
}

/* ---- equilibrium (Sec. 2.2, BGK paragraph) ------------------------------- */
void orc_feq(double rho, double ux, double uy, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int a = 0; a < Q; ++a) {
    double cu = CX[a] * ux + CY[a] * uy;
    /* uu:(c c - cs2 I) = (c.u)^2 - cs2 |u|^2 */
    feq[a] = WGT[a] * rho * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
  }
}

/* ---- Guo forcing term for force density G (ref. guo_discrete_2002) ------- */
void orc_guo(double ux, double uy, double gx, double gy, double *fa) {
  for (int a = 0; a < Q; ++a) {
    double cu = CX[a] * ux + CY[a] * uy;
    double cg = CX[a] * gx + CY[a] * gy;
    double lin = ((CX[a] - ux) * gx + (CY[a] - uy) * gy) / CS2;
    fa[a] = WGT[a] * (lin + cu * cg / (CS2 * CS2));
  }
}

/* ---- body geometry ------------------------------------------------------- */
static double naca_half_thickness(double t, double xi) {
  /* NACA 4-digit symmetric thickness law, in chords */
  return 5.0 * t *
         (0.2969 * sqrt(xi) - 0.1260 * xi - 0.3516 * (xi * xi) +
          0.2843 * (xi * xi * xi) - 0.1015 * (xi * xi * xi * xi));
}

/* chi of Eq. fcar at the lattice node (i, j): 1 inside the body, boundary
 * included.  For the airfoil, (cos a, sin a) of the angle are taken once by
 * the caller of the raster. */
static int inside_body(const orc_body *b, double ca, double sa, int i, int j) {
  double dx = (double)i - b->xg;
  double dy = (double)j - b->yg;
  if (b->kind == BODY_DISK) {
    double r = 0.5 * b->length;
    return dx * dx + dy * dy <= r * r;
  }
  if (b->kind == BODY_NACA) {
    /* airfoil frame: chord direction t = (cos a, -sin a) (nose up for a > 0),
       normal n = (sin a, cos a); xi from the leading edge, zeta along n */
    double xi = (dx * ca - dy * sa) / b->length + b->pivot_frac;
    double zeta = (dx * sa + dy * ca) / b->length;
    if (!(xi >= 0.0 && xi <= 1.0)) return 0;
    return fabs(zeta) <= naca_half_thickness(b->thickness, xi);
  }
  return 0;
}

int orc_raster(const orc_body *b, int32_t nx, int32_t ny, uint8_t *chi) {
  double ca = cos(b->theta), sa = sin(b->theta);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) chi[(size_t)j * nx + i] = (uint8_t)inside_body(b, ca, sa, i, j);
  return 0;
}

/* rigid-body velocity u_s = U + Omega x (x - x_G) at the point (x, y) */
static void solid_velocity(const orc_body *b, double x, double y, double *us) {
  if (b == NULL || b->kind == BODY_NONE) {
    us[0] = us[1] = 0.0;
    return;
  }
  us[0] = b->u[0] - b->omega * (y - b->yg);
  us[1] = b->u[1] + b->omega * (x - b->xg);
}

/* ---- macroscopic fields at one node (Eqs. updatestep .. updatestepm) ----- */
/* Returns rho, u and the total force density G (penalization + body force). */
static void node_moments(const orc_config *cfg, const orc_body *b, const double *fl, int chi, int i,
                         int j, double *rho_o, double *u_o, double *g_o) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < Q; ++a) {
    rho += fl[a];
    jx += CX[a] * fl[a];
    jy += CY[a] * fl[a];
  }
  /* half of the uniform body force enters the momentum as in Eq. updatestep */
  jx += 0.5 * cfg->body_force[0];
  jy += 0.5 * cfg->body_force[1];
  double us[2] = {0.0, 0.0};
  if (chi) solid_velocity(b, (double)i, (double)j, us);
  double pen = chi ? 1.0 / cfg->eta : 0.0; /* chi / eta */
  double k = 0.5 * pen;                    /* dt/2 * chi/eta, dt = 1 */
  /* Eq. updatestepm */
  double ux = (jx + k * rho * us[0]) / (rho + k * rho);
  double uy = (jy + k * rho * us[1]) / (rho + k * rho);
  /* G = -rho chi/eta (u - u_s), rearranged (reading R3):
     rho (u - u_s) = (j - rho u_s) / (1 + k) */
  double gx = cfg->body_force[0] - pen * (jx - rho * us[0]) / (1.0 + k);
  double gy = cfg->body_force[1] - pen * (jy - rho * us[1]) / (1.0 + k);
  *rho_o = rho;
  u_o[0] = ux;
  u_o[1] = uy;
  g_o[0] = gx;
  g_o[1] = gy;
}

/* literal form of the penalization force of Eq. (1) from u of Eq. updatestepm,
 * kept to check the rearranged form */
void orc_penalization_literal(double rho, double jx, double jy, int chi, double eta, double usx,
                              double usy, double *out) {
  double pen = chi ? 1.0 / eta : 0.0;
  double k = 0.5 * pen;
  double ux = (jx + k * rho * usx) / (rho + k * rho);
  double uy = (jy + k * rho * usy) / (rho + k * rho);
  out[0] = ux;
  out[1] = uy;
  out[2] = -rho * pen * (ux - usx);
  out[3] = -rho * pen * (uy - usy);
}

/* exported for the tests: rho, u, G of one node */
void orc_node_moments(const orc_config *cfg, const orc_body *b, const double *fl, int32_t chi,
                      int32_t i, int32_t j, double *out) {
  double rho, u[2], g[2];
  node_moments(cfg, b, fl, chi, i, j, &rho, u, g);
  out[0] = rho;
  out[1] = u[0];
  out[2] = u[1];
  out[3] = g[0];
  out[4] = g[1];
}

static double tau_minus(const orc_config *cfg) {
  if (cfg->collision == COLL_BGK) return cfg->tau_plus;
  return cfg->lambda_trt / (cfg->tau_plus - 0.5) + 0.5;
}

/* ---- collision of one node: BGK or TRT (Eq. TRT) with forcing ------------ */
void orc_collide_node(const orc_config *cfg, const double *fl, double rho, double ux, double uy,
                      double gx, double gy, double *ft) {
  double feq[Q], fa[Q];
  orc_feq(rho, ux, uy, feq);
  orc_guo(ux, uy, gx, gy, fa);
  double tp = cfg->tau_plus;
  if (cfg->collision == COLL_BGK) {
    for (int a = 0; a < Q; ++a)
      ft[a] = fl[a] - (fl[a] - feq[a]) / tp + (1.0 - 1.0 / (2.0 * tp)) * fa[a];
    return;
  }
  double tm = tau_minus(cfg);
  for (int a = 0; a < Q; ++a) {
    int o = OPP[a];
    double fp = 0.5 * (fl[a] + fl[o]), fm = 0.5 * (fl[a] - fl[o]);
    double ep = 0.5 * (feq[a] + feq[o]), em = 0.5 * (feq[a] - feq[o]);
    double src;
    if (cfg->forcing == FORCING_PAPER) {
      src = (1.0 - 1.0 / (2.0 * tp)) * fa[a];
    } else {
      double sp = 0.5 * (fa[a] + fa[o]), sm = 0.5 * (fa[a] - fa[o]);
      src = (1.0 - 1.0 / (2.0 * tp)) * sp + (1.0 - 1.0 / (2.0 * tm)) * sm;
    }
    ft[a] = fl[a] - (fp - ep) / tp - (fm - em) / tm + src;
  }
}

/* ---- SIM stress (Sec. 2.3.2): sigma = -rho cs2 I - (1 - 1/(2 tau)) sum c c (f - feq) */
void orc_stress(const orc_config *cfg, const double *fl, double *sig) {
  double rho, u[2], g[2];
  node_moments(cfg, NULL, fl, 0, 0, 0, &rho, u, g);
  double feq[Q];
  orc_feq(rho, u[0], u[1], feq);
  double pxx = 0.0, pxy = 0.0, pyy = 0.0;
  for (int a = 0; a < Q; ++a) {
    double d = fl[a] - feq[a];
    pxx += CX[a] * CX[a] * d;
    pxy += CX[a] * CY[a] * d;
    pyy += CY[a] * CY[a] * d;
  }
  double s = 1.0 - 1.0 / (2.0 * cfg->tau_plus);
  sig[0] = -rho * CS2 - s * pxx;
  sig[1] = -s * pxy;
  sig[2] = -rho * CS2 - s * pyy;
}

/* ---- initial state: f = f^eq(rho = 1, u0), u0 = u_in in the fluid and the
 * rigid velocity in the solid -------------------------------------------- */
void orc_init(const orc_config *cfg, const orc_body *b, const uint8_t *chi, double *f) {
  for (int j = 0; j < cfg->ny; ++j)
    for (int i = 0; i < cfg->nx; ++i) {
      double u[2] = {cfg->u_in[0], cfg->u_in[1]};
      if (chi[(size_t)j * cfg->nx + i]) solid_velocity(b, (double)i, (double)j, u);
      double feq[Q];
      orc_feq(1.0, u[0], u[1], feq);
      for (int a = 0; a < Q; ++a) f[idx(cfg, a, i, j)] = feq[a];
    }
}

/* ---- collision of the whole lattice ------------------------------------- */
void orc_collide(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *f,
                 double *ft) {
  int nx = cfg->nx, ny = cfg->ny;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double fl[Q], out[Q], rho, u[2], g[2];
      for (int a = 0; a < Q; ++a) fl[a] = f[idx(cfg, a, i, j)];
      node_moments(cfg, b, fl, chi[(size_t)j * nx + i], i, j, &rho, u, g);
      orc_collide_node(cfg, fl, rho, u[0], u[1], g[0], g[1], out);
      for (int a = 0; a < Q; ++a) ft[idx(cfg, a, i, j)] = out[a];
    }
}

/* ---- macroscopic fields (rho, ux, uy) of a pre-collision field ------------ */
void orc_fields(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *f,
                double *rho_o, double *ux_o, double *uy_o) {
  int nx = cfg->nx, ny = cfg->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double fl[Q], rho, u[2], g[2];
      for (int a = 0; a < Q; ++a) fl[a] = f[idx(cfg, a, i, j)];
      node_moments(cfg, b, fl, chi[(size_t)j * nx + i], i, j, &rho, u, g);
      size_t n = (size_t)j * nx + i;
      rho_o[n] = rho;
      ux_o[n] = u[0];
      uy_o[n] = u[1];
    }
}

/* ---- streaming (Eq. eqBd) and boundary conditions (Sec. 3.1, 3.2) ---------
 * f_out[a](y) = ft[a](y - c_a) when that source node exists (periodic sides
 * wrap).  Otherwise the side the source lies beyond decides (x side first):
 *   inlet   : half-way bounce-back from a wall moving with u_in,
 *             f_a = ft_abar(y) + 2 w_a rho_w (c_a.u_in)/cs2, rho_w = 1
 *   no-slip : half-way bounce-back, f_a = ft_abar(y)
 *   symmetry: specular reflection at the wall half a cell beyond the edge
 *   outlet  : convective condition (Yang), f_a^{n+1}(N-1) =
 *             (f_a^n(N-1) + U_c f_a^{n+1}(N-2)) / (1 + U_c), U_c = |u_in|
 *   free outlet: zero normal gradient, f_a^{n+1}(N-1) = f_a^{n+1}(N-2)
 * f_prev is the pre-collision field of the current step (for the outlet). */
static int mirror_y(int a) {
  /* flip c_y */
  static const int m[Q] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
  return m[a];
}

void orc_stream(const orc_config *cfg, const double *ft, const double *f_prev, double *f_out) {
  int nx = cfg->nx, ny = cfg->ny;
  double uc = sqrt(cfg->u_in[0] * cfg->u_in[0] + cfg->u_in[1] * cfg->u_in[1]);
  /* pass 1: everything except outlet populations */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int a = 0; a < Q; ++a) {
        int si = i - CX[a], sj = j - CY[a];
        if (si < 0 && cfg->bc[0] == BC_PERIODIC) si += nx;
        if (si >= nx && cfg->bc[1] == BC_PERIODIC) si -= nx;
        if (sj < 0 && cfg->bc[2] == BC_PERIODIC) sj += ny;
        if (sj >= ny && cfg->bc[3] == BC_PERIODIC) sj -= ny;
        double v;
        if (si >= 0 && si < nx && sj >= 0 && sj < ny) {
          v = ft[idx(cfg, a, si, sj)];
        } else if (si < 0 || si >= nx) {
          int side = si < 0 ? 0 : 1;
          int kind = cfg->bc[side];
          if (kind == BC_OUTLET || kind == BC_OUTLET_FREE) continue; /* pass 2 */
          if (kind == BC_INLET) {
            double cu = CX[a] * cfg->u_in[0] + CY[a] * cfg->u_in[1];
            v = ft[idx(cfg, OPP[a], i, j)] + 2.0 * WGT[a] * 1.0 * cu / CS2;
          } else { /* BC_NOSLIP */
            v = ft[idx(cfg, OPP[a], i, j)];
          }
        } else {
          int side = sj < 0 ? 2 : 3;
          int kind = cfg->bc[side];
          if (kind == BC_SYMMETRY) {
            /* the population arrived by reflection from the node in the same
               row that its horizontal motion came from */
            v = ft[idx(cfg, mirror_y(a), si, j)];
          } else { /* BC_NOSLIP */
            v = ft[idx(cfg, OPP[a], i, j)];
          }
        }
        f_out[idx(cfg, a, i, j)] = v;
      }
  /* pass 2: convective outlet on the x_hi side */
  if (cfg->bc[1] == BC_OUTLET) {
    int i = nx - 1;
    for (int j = 0; j < ny; ++j)
      for (int a = 0; a < Q; ++a) {
        if (CX[a] >= 0) continue;
        f_out[idx(cfg, a, i, j)] =
            (f_prev[idx(cfg, a, i, j)] + uc * f_out[idx(cfg, a, i - 1, j)]) / (1.0 + uc);
      }
  }
  /* pass 2: free outlet on the x_hi side */
  if (cfg->bc[1] == BC_OUTLET_FREE) {
    int i = nx - 1;
    for (int j = 0; j < ny; ++j)
      for (int a = 0; a < Q; ++a)
        if (CX[a] < 0) f_out[idx(cfg, a, i, j)] = f_out[idx(cfg, a, i - 1, j)];
  }
}

/* ---- MEM (Sec. 2.3.1, Eqs. MMEL and fluidtorque) ---------------------------
 * Links are the pairs (x_f, a) with chi(x_f) = 0 and chi(x_f + c_a) = 1, both
 * inside the lattice (periodic sides wrap).  Summed j-major, then i, then a. */
void orc_mem(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *ft,
             double *out) {
  int nx = cfg->nx, ny = cfg->ny;
  double fx = 0.0, fy = 0.0, tq = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (chi[(size_t)j * nx + i]) continue;
      for (int a = 1; a < Q; ++a) {
        int si = i + CX[a], sj = j + CY[a];
        if (si < 0 || si >= nx) {
          if (cfg->bc[0] != BC_PERIODIC) continue;
          si = (si + nx) % nx;
        }
        if (sj < 0 || sj >= ny) {
          if (cfg->bc[2] != BC_PERIODIC) continue;
          sj = (sj + ny) % ny;
        }
        if (!chi[(size_t)sj * nx + si]) continue;
        /* x_Gamma: midpoint of the link (unwrapped) */
        double xgx = (double)i + 0.5 * CX[a], xgy = (double)j + 0.5 * CY[a];
        double ug[2];
        solid_velocity(b, xgx, xgy, ug);
        int o = OPP[a];
        double f_out = ft[idx(cfg, a, i, j)];
        double f_in = ft[idx(cfg, o, si, sj)];
        double lx = (CX[a] - ug[0]) * f_out - (CX[o] - ug[0]) * f_in;
        double ly = (CY[a] - ug[1]) * f_out - (CY[o] - ug[1]) * f_in;
        fx += lx;
        fy += ly;
        double rx = xgx - (b ? b->xg : 0.0), ry = xgy - (b ? b->yg : 0.0);
        tq += rx * ly - ry * lx;
      }
    }
  out[0] = fx;
  out[1] = fy;
  out[2] = tq;
}

/* ---- volume-integral force (Eq. Angotforce, Sec. 2.3) ----------------------
 * The force the penalization exerts on the fluid, reversed: over the solid
 * nodes, F = -sum G_pen = sum rho (chi/eta)(u - u_s), with u the penalized
 * velocity of Eq. updatestepm and G_pen the penalization part of the force
 * density (reading R19: the printed formula has lost its 1/eta and its limit
 * is eta -> 0).  Torque about the body reference point.  Evaluated on the
 * pre-collision field of a step, like SIM; summed j-major, then i. */
void orc_angot(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *f,
               double *out) {
  const int nx = cfg->nx, ny = cfg->ny;
  double F[2] = {0.0, 0.0}, T = 0.0;
  double fl[Q];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (!chi[(size_t)j * nx + i]) continue;
      for (int a = 0; a < Q; ++a) fl[a] = f[((size_t)a * ny + j) * nx + i];
      double rho, u[2], g[2];
      node_moments(cfg, b, fl, 1, i, j, &rho, u, g);
      const double fx = -(g[0] - cfg->body_force[0]), fy = -(g[1] - cfg->body_force[1]);
      F[0] += fx;
      F[1] += fy;
      T += (i - b->xg) * fy - (j - b->yg) * fx;
    }
  out[0] = F[0];
  out[1] = F[1];
  out[2] = T;
}

/* ---- SIM integration points: a closed polygon, counter-clockwise ---------
 * pts[k*5 + 0..4] = (x - x_G, y - y_G, n_x, n_y, S) at the edge midpoints.
 * Disk: n vertices at angles 2 pi k / n on the circle.
 * NACA: m = (n - 1)/2 cosine-spaced stations xi_k = (1 - cos(pi k / m))/2 on
 * each surface, upper surface from the trailing edge to the leading edge,
 * lower surface back, closed by the trailing-edge segment (n = 849 gives the
 * point count of Sec. 3.1). */
int orc_sim_points(const orc_body *b, int32_t n, double *pts) {
  int nv;
  double *vx, *vy;
  if (b->kind == BODY_DISK) {
    if (n < 3) return -1;
    nv = n;
    vx = malloc(sizeof(double) * nv);
    vy = malloc(sizeof(double) * nv);
    double r = 0.5 * b->length;
    for (int k = 0; k < nv; ++k) {
      double th = 2.0 * M_PI * (double)k / (double)nv;
      vx[k] = r * cos(th);
      vy[k] = r * sin(th);
    }
  } else if (b->kind == BODY_NACA) {
    if (n < 5 || n % 2 == 0) return -1;
    int m = (n - 1) / 2;
    /* upper surface TE .. LE (m + 1 vertices), lower surface after the LE
       up to the TE (m vertices) */
    vx = malloc(sizeof(double) * (2 * m + 1));
    vy = malloc(sizeof(double) * (2 * m + 1));
    double ca = cos(b->theta), sa = sin(b->theta);
    int v = 0;
    /* airfoil-frame vertex (xi, zeta) in chords -> offset from the pivot */
    for (int k = m; k >= 0; --k) { /* upper surface, TE to LE */
      double xi = 0.5 * (1.0 - cos(M_PI * (double)k / (double)m));
      double zt = naca_half_thickness(b->thickness, xi);
      double s = (xi - b->pivot_frac) * b->length, z = zt * b->length;
      vx[v] = s * ca + z * sa;
      vy[v] = -s * sa + z * ca;
      ++v;
    }
    for (int k = 1; k <= m; ++k) { /* lower surface, LE to TE */
      double xi = 0.5 * (1.0 - cos(M_PI * (double)k / (double)m));
      double zt = -naca_half_thickness(b->thickness, xi);
      double s = (xi - b->pivot_frac) * b->length, z = zt * b->length;
      vx[v] = s * ca + z * sa;
      vy[v] = -s * sa + z * ca;
      ++v;
    }
    /* v == 2m + 1 here: the lower TE vertex is the last one; the closing
       edge goes from it back to vertex 0 (upper TE) */
    nv = v;
    if (nv != n) {
      free(vx);
      free(vy);
      return -1;
    }
  } else {
    return -1;
  }
  for (int k = 0; k < nv; ++k) {
    int k2 = (k + 1) % nv;
    double ex = vx[k2] - vx[k], ey = vy[k2] - vy[k];
    double len = sqrt(ex * ex + ey * ey);
    pts[5 * k + 0] = 0.5 * (vx[k] + vx[k2]);
    pts[5 * k + 1] = 0.5 * (vy[k] + vy[k2]);
    /* outward normal of a counter-clockwise polygon: the edge turned clockwise */
    pts[5 * k + 2] = ey / len;
    pts[5 * k + 3] = -ex / len;
    pts[5 * k + 4] = len;
  }
  free(vx);
  free(vy);
  return 0;
}

/* lattice direction closest to the normal n: argmax c_a.n / |c_a|, ties to
 * the lowest a */
int orc_sim_direction(double nx_, double ny_) {
  int best = 1;
  double bv = -1e300;
  for (int a = 1; a < Q; ++a) {
    double len = (a <= 4) ? 1.0 : sqrt(2.0);
    double v = (CX[a] * nx_ + CY[a] * ny_) / len;
    if (v > bv) {
      bv = v;
      best = a;
    }
  }
  return best;
}

/* ---- SIM force (Eq. defFf and its quadrature form) -------------------------
 * For each point x_i: the nearest lattice node (a coordinate exactly half-way
 * between two nodes has both as candidates); from each candidate walk
 * q_k = q_0 + k c_a*, k = 0..3, to the first fluid node inside the lattice;
 * sigma at x_i is the mean of sigma over the candidates' fluid nodes, computed
 * from their pre-collision populations.  Sums S_i sigma n_i and
 * (x_i - x_G) x (S_i sigma n_i) in point order.  nodes[p] gets the fluid node
 * of the first candidate (-1 when a point has none).  Returns the number of
 * points without a fluid node (0 on success); those points are left out. */
static int sim_walk(const orc_config *cfg, const uint8_t *chi, int a, int qi, int qj, int *oi,
                    int *oj) {
  for (int k = 0; k <= 3; ++k) {
    int ii = qi + k * CX[a], jj = qj + k * CY[a];
    if (ii < 0 || ii >= cfg->nx || jj < 0 || jj >= cfg->ny) return 0;
    if (!chi[(size_t)jj * cfg->nx + ii]) {
      *oi = ii;
      *oj = jj;
      return 1;
    }
  }
  return 0;
}

/* SIM force and torque (Eq. defFf) with the stress of Sec. 2.3.2 sampled at
 * each integration point either as the paper describes it (order 0, reading
 * R6: the stress of the first fluid node q met along the lattice direction c
 * closest to the normal), or extrapolated linearly to the point along that
 * direction (order 1, reading R20): sigma(x_i) = sigma(q) + t (sigma(q + c) -
 * sigma(q)) with t = (x_i - q).c / |c|^2, falling back to order 0 where q + c
 * is solid or outside the lattice.  Tie points average over both nodes.
 * pt_sigma, when given, receives each point's (xx, xy, yy) stress. */
int orc_sim_order(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *f,
                  int32_t n, const double *pts, int32_t order, double *out, int32_t *nodes,
                  double *pt_sigma) {
  int nx = cfg->nx, ny = cfg->ny, missing = 0;
  double fx = 0.0, fy = 0.0, tq = 0.0;
  for (int p = 0; p < n; ++p) {
    const double *pt = pts + 5 * p;
    double x = b->xg + pt[0], y = b->yg + pt[1];
    int a = orc_sim_direction(pt[2], pt[3]);
    double rx = floor(x + 0.5), ry = floor(y + 0.5);
    int cxs[2] = {(int)rx, (int)rx - 1}, cys[2] = {(int)ry, (int)ry - 1};
    int ncx = (rx == x + 0.5) ? 2 : 1, ncy = (ry == y + 0.5) ? 2 : 1;
    double sig[3] = {0.0, 0.0, 0.0};
    int ok = 1, first = -1;
    for (int u = 0; u < ncy && ok; ++u)
      for (int v = 0; v < ncx && ok; ++v) {
        int qi, qj;
        if (!sim_walk(cfg, chi, a, cxs[v], cys[u], &qi, &qj)) {
          ok = 0;
          break;
        }
        if (first < 0) first = qj * nx + qi;
        double fl[Q], s3[3];
        for (int c = 0; c < Q; ++c) fl[c] = f[idx(cfg, c, qi, qj)];
        orc_stress(cfg, fl, s3);
        const int ni = qi + CX[a], nj = qj + CY[a];
        if (order == 1 && ni >= 0 && ni < nx && nj >= 0 && nj < ny && !chi[(size_t)nj * nx + ni]) {
          double s3n[3];
          for (int c = 0; c < Q; ++c) fl[c] = f[idx(cfg, c, ni, nj)];
          orc_stress(cfg, fl, s3n);
          const double t = ((x - qi) * CX[a] + (y - qj) * CY[a]) / (double)(CX[a] * CX[a] + CY[a] * CY[a]);
          for (int k = 0; k < 3; ++k) s3[k] += t * (s3n[k] - s3[k]);
        }
        sig[0] += s3[0];
        sig[1] += s3[1];
        sig[2] += s3[2];
      }
    if (nodes) nodes[p] = ok ? first : -1;
    if (!ok) {
      ++missing;
      continue;
    }
    double cnt = (double)(ncx * ncy);
    sig[0] /= cnt;
    sig[1] /= cnt;
    sig[2] /= cnt;
    if (pt_sigma) {
      pt_sigma[3 * p] = sig[0];
      pt_sigma[3 * p + 1] = sig[1];
      pt_sigma[3 * p + 2] = sig[2];
    }
    double tx = pt[4] * (sig[0] * pt[2] + sig[1] * pt[3]);
    double ty = pt[4] * (sig[1] * pt[2] + sig[2] * pt[3]);
    fx += tx;
    fy += ty;
    tq += pt[0] * ty - pt[1] * tx;
  }
  out[0] = fx;
  out[1] = fy;
  out[2] = tq;
  return missing;
}

int orc_sim(const orc_config *cfg, const orc_body *b, const uint8_t *chi, const double *f,
            int32_t n, const double *pts, double *out, int32_t *nodes) {
  return orc_sim_order(cfg, b, chi, f, n, pts, 0, out, nodes, NULL);
}

/* ---- rigid body, Eqs. dep1 and theta2, explicit trapezoid in time -------- */
void orc_rigid_update(orc_body *b, const double *force) {
  double r = 0.5 * b->length;
  double m = b->density_ratio * M_PI * r * r; /* fluid density 1 */
  double inertia = 0.5 * m * r * r;
  double buoy = 1.0 - 1.0 / b->density_ratio;
  double ax = force[0] / m + buoy * b->gravity[0];
  double ay = force[1] / m + buoy * b->gravity[1];
  double u0x = b->u[0], u0y = b->u[1], w0 = b->omega;
  b->u[0] = u0x + ax;
  b->u[1] = u0y + ay;
  b->omega = w0 + force[2] / inertia;
  b->xg += 0.5 * (u0x + b->u[0]);
  b->yg += 0.5 * (u0y + b->u[1]);
  b->theta += 0.5 * (w0 + b->omega);
}

/* ---- full time loop -------------------------------------------------------
 * f: pre-collision field f^0 in, f^nsteps out.  chi: mask of the body at the
 * start, updated when the body moves.  estimator (0 MEM, 1 SIM) drives the
 * rigid body when b->moving.  Histories (3 doubles per step) may be NULL;
 * body_hist gets (x_G, y_G, theta, u_x, u_y, omega) after each step. */
int orc_run(const orc_config *cfg, orc_body *b, double *f, uint8_t *chi, int32_t nsteps,
            int32_t estimator, int32_t n_sim, const double *sim_pts, double *mem_hist,
            double *sim_hist, double *body_hist) {
  size_t nn = (size_t)Q * cfg->nx * cfg->ny;
  double *ft = malloc(sizeof(double) * nn);
  double *fn = malloc(sizeof(double) * nn);
  if (!ft || !fn) {
    free(ft);
    free(fn);
    return -1;
  }
  int bad = 0;
  for (int s = 0; s < nsteps; ++s) {
    double mem[3] = {0, 0, 0}, sim[3] = {0, 0, 0};
    if (n_sim > 0 && sim_pts) bad += orc_sim(cfg, b, chi, f, n_sim, sim_pts, sim, NULL);
    orc_collide(cfg, b, chi, f, ft);
    orc_mem(cfg, b, chi, ft, mem);
    orc_stream(cfg, ft, f, fn);
    memcpy(f, fn, sizeof(double) * nn);
    if (mem_hist) memcpy(mem_hist + 3 * (size_t)s, mem, sizeof mem);
    if (sim_hist) memcpy(sim_hist + 3 * (size_t)s, sim, sizeof sim);
    if (b && b->moving) {
      orc_rigid_update(b, estimator == 1 ? sim : mem);
      orc_raster(b, cfg->nx, cfg->ny, chi);
    }
    if (body_hist && b) {
      double *bh = body_hist + 6 * (size_t)s;
      bh[0] = b->xg;
      bh[1] = b->yg;
      bh[2] = b->theta;
      bh[3] = b->u[0];
      bh[4] = b->u[1];
      bh[5] = b->omega;
    }
  }
  free(ft);
  free(fn);
  return bad;
}
