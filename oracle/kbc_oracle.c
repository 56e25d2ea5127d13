/*
 * kbc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU statement of the entropic
 * multi-relaxation-time lattice Boltzmann (KBC) step that the CUDA library
 * computes.  It exists to check the CUDA path: only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header or table with the CUDA library.
 *
 * Paper: Dorschner, Chikatamarla, Karlin, "Fluid-structure interaction with
 * the entropic lattice Boltzmann method" (arXiv 1710.02375).
 *   - evolution / over-relaxation ............ Eq. (f_equations)
 *   - kinematic / shear / higher split ........ Eq. (popSplit)
 *   - mirror state ............................ Eq. (f_mirr)
 *   - entropic equilibrium .................... Eqs. (feq_min), (conservationLaws)
 *   - stabiliser gamma ........................ Eq. (gamma_min_approx)
 *   - viscosity ............................... Eq. (visc)
 *
 * Readings of points the paper leaves open (each is pinned by a test):
 *   - Lattices D2Q9 / D3Q27 are tensor products of D1Q3 with weights 2/3
 *     (c = 0) and 1/6 (c = +-1).
 *   - The minimiser of Eq. (feq_min) under Eq. (conservationLaws) is taken in
 *     its closed product form (Ansumali, Karlin, Oettinger 2003):
 *       feq_i = rho prod_a w(c_ia) (2 - S_a) ((2 u_a + S_a)/(1 - u_a))^c_ia,
 *       S_a = sqrt(1 + 3 u_a^2).
 *   - k = {rho, j}; s = trace-free (deviatoric) part of the second moments;
 *     h = everything else (trace, third and fourth order moments).
 *   - gamma = 2 (plain BGK with omega = 2 beta) when <dh|dh> <= 1e-30.
 *   - gamma is held in [0, 2/beta]: Eq. (gamma_min_approx) is the vertex of
 *     the quadratic entropy norm of f', a convex parabola in gamma, and the
 *     post-collision higher-order part is (1 - beta gamma) dh, which grows
 *     outside that range.  The paper gives the estimate without bounds; the
 *     clip is the minimum of the same norm over the non-growing rates.  (Seen
 *     unbounded in a channel start-up: gamma up to 6.7 at outlet nodes next
 *     to the walls, which grew round-off differences a hundred-thousand-fold
 *     within a few dozen steps.)
 *
 * Population layout (the library's interface layout as well): structure of
 * arrays f[i][z][y][x], direction index i = (cz+1)*9 + (cy+1)*3 + (cx+1) for
 * D3Q27 and i = (cy+1)*3 + (cx+1) for D2Q9; the opposite of i is Q-1-i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXQ 27

typedef struct {
  int Q, D;
  int c[OR_MAXQ][3];
  double w[OR_MAXQ];
} or_lattice;

static int make_lattice(int lat, or_lattice *L) {
  const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}; /* index c+1 */
  if (lat == 9) {
    L->Q = 9; L->D = 2;
    for (int cy = -1; cy <= 1; ++cy)
      for (int cx = -1; cx <= 1; ++cx) {
        int i = (cy + 1) * 3 + (cx + 1);
        L->c[i][0] = cx; L->c[i][1] = cy; L->c[i][2] = 0;
        L->w[i] = w1[cx + 1] * w1[cy + 1];
      }
    return 0;
  }
  if (lat == 27) {
    L->Q = 27; L->D = 3;
    for (int cz = -1; cz <= 1; ++cz)
      for (int cy = -1; cy <= 1; ++cy)
        for (int cx = -1; cx <= 1; ++cx) {
          int i = (cz + 1) * 9 + (cy + 1) * 3 + (cx + 1);
          L->c[i][0] = cx; L->c[i][1] = cy; L->c[i][2] = cz;
          L->w[i] = w1[cx + 1] * w1[cy + 1] * w1[cz + 1];
        }
    return 0;
  }
  return -1;
}

/* ---- exported lattice tables (for tests) ---- */
int or_lattice_tables(int lat, int *c /*[Q][3]*/, double *w /*[Q]*/) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
  return L.Q;
}

/* Entropic equilibrium, Eq. (feq_min) under Eq. (conservationLaws), in the
 * closed product form.  u has 3 components; for D2Q9 u[2] is ignored. */
static void equilibrium(const or_lattice *L, double rho, const double *u, double *feq) {
  for (int i = 0; i < L->Q; ++i) {
    double p = rho;
    for (int a = 0; a < L->D; ++a) {
      double S = sqrt(1.0 + 3.0 * u[a] * u[a]);
      int ci = L->c[i][a];
      double w1 = (ci == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
      double f = w1 * (2.0 - S);
      if (ci == 1) f *= (2.0 * u[a] + S) / (1.0 - u[a]);
      if (ci == -1) f *= (1.0 - u[a]) / (2.0 * u[a] + S);
      p *= f;
    }
    feq[i] = p;
  }
}

int or_equilibrium(int lat, double rho, const double *u, double *feq) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  equilibrium(&L, rho, u, feq);
  return 0;
}

/* Zeroth, first and second moments of a population vector. */
static void moments(const or_lattice *L, const double *f, double *rho, double *j, double P[3][3]) {
  *rho = 0.0;
  for (int a = 0; a < 3; ++a) {
    j[a] = 0.0;
    for (int b = 0; b < 3; ++b) P[a][b] = 0.0;
  }
  for (int i = 0; i < L->Q; ++i) {
    *rho += f[i];
    for (int a = 0; a < 3; ++a) {
      j[a] += L->c[i][a] * f[i];
      for (int b = 0; b < 3; ++b) P[a][b] += L->c[i][a] * L->c[i][b] * f[i];
    }
  }
}

/* Shear part of a population vector with second-moment tensor dP: the
 * population carrying exactly the trace-free part of dP and no other natural
 * moment (Eq. popSplit, s-part). */
static void shear_part(const or_lattice *L, const double dP[3][3], double *s) {
  for (int i = 0; i < L->Q; ++i) {
    const int *c = L->c[i];
    int nnz = (c[0] != 0) + (c[1] != 0) + (c[2] != 0);
    double v = 0.0;
    if (L->D == 2) {
      double N = dP[0][0] - dP[1][1];
      if (nnz == 1) v = (c[0] != 0) ? N / 4.0 : -N / 4.0;
      else if (nnz == 2) v = c[0] * c[1] * dP[0][1] / 4.0;
    } else {
      double Nxz = dP[0][0] - dP[2][2], Nyz = dP[1][1] - dP[2][2];
      if (nnz == 1) {
        if (c[0] != 0) v = (2.0 * Nxz - Nyz) / 6.0;
        else if (c[1] != 0) v = (2.0 * Nyz - Nxz) / 6.0;
        else v = -(Nxz + Nyz) / 6.0;
      } else if (nnz == 2) {
        if (c[2] == 0) v = c[0] * c[1] * dP[0][1] / 4.0;
        else if (c[1] == 0) v = c[0] * c[2] * dP[0][2] / 4.0;
        else v = c[1] * c[2] * dP[1][2] / 4.0;
      }
    }
    s[i] = v;
  }
}

/* One KBC collision at one node, Eqs. (f_equations), (f_mirr),
 * (gamma_min_approx).  mode 0: KBC; mode 1: gamma fixed to 2 (BGK).
 * Outputs (optional, may be NULL): gamma, ds[Q], dh[Q], feq[Q]. */
static void collide(const or_lattice *L, double beta, int mode, const double *f, double *fout,
                    double *gamma_out, double *ds_out, double *dh_out, double *feq_out) {
  const int Q = L->Q;
  double rho, j[3], P[3][3], u[3], feq[OR_MAXQ];
  moments(L, f, &rho, j, P);
  for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
  equilibrium(L, rho, u, feq);

  double rho_e, j_e[3], Peq[3][3], dP[3][3];
  moments(L, feq, &rho_e, j_e, Peq);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) dP[a][b] = P[a][b] - Peq[a][b];

  double ds[OR_MAXQ], dh[OR_MAXQ];
  shear_part(L, dP, ds);
  for (int i = 0; i < Q; ++i) dh[i] = (f[i] - feq[i]) - ds[i]; /* dk = 0 */

  double sh = 0.0, hh = 0.0;
  for (int i = 0; i < Q; ++i) {
    sh += ds[i] * dh[i] / feq[i];
    hh += dh[i] * dh[i] / feq[i];
  }
  double gamma = 2.0;
  if (mode == 0 && hh > 1e-30) {
    gamma = 1.0 / beta - (2.0 - 1.0 / beta) * sh / hh;
    /* the quadratic entropy norm is a convex parabola in gamma; its minimum
     * over the rates at which the higher-order part does not grow,
     * |1 - beta gamma| <= 1, is the vertex clipped to [0, 2/beta] */
    if (gamma > 2.0 / beta) gamma = 2.0 / beta;
    if (gamma < 0.0) gamma = 0.0;
  }

  for (int i = 0; i < Q; ++i) {
    /* f_mirr = k + (2 s_eq - s) + ((1 - gamma) h + gamma h_eq) = f - 2 ds - gamma dh */
    double fmirr = f[i] - 2.0 * ds[i] - gamma * dh[i];
    fout[i] = (1.0 - beta) * f[i] + beta * fmirr;
  }
  if (gamma_out) *gamma_out = gamma;
  if (ds_out) memcpy(ds_out, ds, sizeof(double) * Q);
  if (dh_out) memcpy(dh_out, dh, sizeof(double) * Q);
  if (feq_out) memcpy(feq_out, feq, sizeof(double) * Q);
}

int or_collide(int lat, double beta, int mode, const double *f, double *fout, double *gamma,
               double *ds, double *dh, double *feq) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  collide(&L, beta, mode, f, fout, gamma, ds, dh, feq);
  return 0;
}

static inline long idx3(int x, int y, int z, int nx, int ny) {
  return ((long)z * ny + y) * nx + x;
}
static inline int wrap(int a, int n) { return ((a % n) + n) % n; }

/* Initialise a state to the equilibrium of given macroscopic fields.
 * rho[n], u[3][n] (n = nx*ny*nz, x fastest). */
int or_init_equilibrium(int lat, int nx, int ny, int nz, const double *rho, const double *u,
                        double *f) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  long n = (long)nx * ny * nz;
  double feq[OR_MAXQ];
  for (long k = 0; k < n; ++k) {
    double uk[3] = {u[k], u[n + k], (L.D == 3) ? u[2 * n + k] : 0.0};
    equilibrium(&L, rho[k], uk, feq);
    for (int i = 0; i < L.Q; ++i) f[i * n + k] = feq[i];
  }
  return 0;
}

/* Density and velocity of a state: rho[n], u[3][n]. */
int or_macros(int lat, int nx, int ny, int nz, const double *f, double *rho, double *u) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  long n = (long)nx * ny * nz;
  for (long k = 0; k < n; ++k) {
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < L.Q; ++i) {
      double v = f[i * n + k];
      r += v;
      for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * v;
    }
    rho[k] = r;
    for (int a = 0; a < 3; ++a) u[a * n + k] = j[a] / r;
  }
  return 0;
}

/* Fully periodic time step: pull-stream f_i(x) = f'_i(x - c_i), then the KBC
 * collision, Eq. (f_equations).  fin and fout hold post-collision states. */
int or_step_periodic(int lat, int nx, int ny, int nz, double beta, int mode, const double *fin,
                     double *fout, double *gamma_field) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  if (L.D == 2 && nz != 1) return -1;
  long n = (long)nx * ny * nz;
  double f[OR_MAXQ], fo[OR_MAXQ], g;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long k = idx3(x, y, z, nx, ny);
        for (int i = 0; i < L.Q; ++i) {
          int xs = wrap(x - L.c[i][0], nx), ys = wrap(y - L.c[i][1], ny),
              zs = wrap(z - L.c[i][2], nz);
          f[i] = fin[i * n + idx3(xs, ys, zs, nx, ny)];
        }
        collide(&L, beta, mode, f, fo, &g, NULL, NULL, NULL);
        for (int i = 0; i < L.Q; ++i) fout[i * n + k] = fo[i];
        if (gamma_field) gamma_field[k] = g;
      }
  return 0;
}

/* nsteps periodic steps; the state is advanced in place (f has Q*n doubles,
 * work is scratch of the same size). */
int or_run_periodic(int lat, int nx, int ny, int nz, double beta, int mode, int nsteps, double *f,
                    double *work) {
  for (int t = 0; t < nsteps; ++t) {
    int rc = or_step_periodic(lat, nx, ny, nz, beta, mode, f, work, NULL);
    if (rc) return rc;
    or_lattice L;
    make_lattice(lat, &L);
    memcpy(f, work, sizeof(double) * (size_t)L.Q * nx * ny * nz);
  }
  return 0;
}

/* ======================================================================
 * Multiphase KBC (section "Extensions to fluid-structure interaction in
 * multiphase flow"): Eqs. (Force), (force1), (Korteweg), (eos), the
 * exact-difference forcing Eq. (force_mp) and the shifted entropic product
 * for gamma.  Fully periodic lattices, no solid (the wetting force and walls
 * are not part of this statement).
 *
 * Readings of the points the paper leaves open or prints at odds:
 *   - Mean-field force: Eqs. (force1) and (Korteweg) give
 *       F_f = d(rho c_s^2 - p) + kappa rho d(lap rho)
 *           = 2 phi d(phi) + kappa rho d(lap rho),   phi = sqrt(rho c_s^2 - p);
 *     Eq. (force2) prints the second term with a minus sign, which the
 *     divergence of the printed Korteweg stress does not give (and which makes
 *     the surface tension negative for kappa > 0); the derivation's sign is
 *     used.  phi = sqrt(max(rho c_s^2 - p, 0)).
 *   - Derivatives on the lattice (not given): the isotropic lattice stencils
 *       d_a psi(x) = 3 sum_i W_i c_ia psi(x + c_i),
 *       lap psi(x) = 6 sum_i W_i (psi(x + c_i) - psi(x)),
 *     and d(lap rho) as the gradient stencil applied to the lap rho field.
 *   - rho(x) is the density after streaming (the pulled populations); the
 *     force uses the density fields of the same time level.
 *   - Exact difference method: du = F / rho (the printed F / (rho dt) with
 *     dt = 1); the collision uses u = j / rho; after the KBC relaxation the
 *     node adds F_i = feq(rho, u + du) - feq(rho, u); the gamma of Eq.
 *     (gamma_min_approx) takes the shifted metric 1 / feq(rho, u + du) in
 *     both products (held in [0, 2/beta] as in the single-phase step).  The
 *     velocity of the fluid at the node is (j + F/2) / rho with j the
 *     momentum before the forcing, i.e. (j' - F/2) / rho after it.
 *   - eos 0: Eq. (eos) as printed; eos 1: the ideal gas p = rho c_s^2 (test
 *     switch: phi = 0).
 *   - g_ext: an optional uniform acceleration added to F / rho (test switch).
 * ====================================================================== */

static double eos_pressure(int eos, double rho) {
  if (eos == 1) return rho / 3.0;
  const double c[6] = {5.3e-2, -3.818183621928911e-2, 4.139745482116095e-3,
                       3.748484095210317e-4, -1.4552652965531227e-4, 1.2746947442749278e-5};
  double r = rho, p = 0.0;
  for (int k = 0; k < 6; ++k) {
    p += c[k] * r;
    r *= rho;
  }
  return p;
}

int or_eos(int eos, int n, const double *rho, double *p) {
  for (int k = 0; k < n; ++k) p[k] = eos_pressure(eos, rho[k]);
  return 0;
}

/* KBC collision with the exact-difference force of velocity increment du
 * and the shifted entropic metric; returns gamma. */
static double collide_forced(const or_lattice *L, double beta, int mode, const double *f,
                             const double *du, double *fout) {
  const int Q = L->Q;
  double rho, j[3], P[3][3], u[3], us[3], feq[OR_MAXQ], fsh[OR_MAXQ];
  moments(L, f, &rho, j, P);
  for (int a = 0; a < 3; ++a) {
    u[a] = j[a] / rho;
    us[a] = u[a] + du[a];
  }
  equilibrium(L, rho, u, feq);
  equilibrium(L, rho, us, fsh);
  double rho_e, j_e[3], Peq[3][3], dP[3][3];
  moments(L, feq, &rho_e, j_e, Peq);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) dP[a][b] = P[a][b] - Peq[a][b];
  double ds[OR_MAXQ], dh[OR_MAXQ];
  shear_part(L, dP, ds);
  for (int i = 0; i < Q; ++i) dh[i] = (f[i] - feq[i]) - ds[i];
  double sh = 0.0, hh = 0.0;
  for (int i = 0; i < Q; ++i) {
    sh += ds[i] * dh[i] / fsh[i];
    hh += dh[i] * dh[i] / fsh[i];
  }
  double gamma = 2.0;
  if (mode == 0 && hh > 1e-30) {
    gamma = 1.0 / beta - (2.0 - 1.0 / beta) * sh / hh;
    if (gamma > 2.0 / beta) gamma = 2.0 / beta;
    if (gamma < 0.0) gamma = 0.0;
  }
  for (int i = 0; i < Q; ++i) {
    const double fmirr = f[i] - 2.0 * ds[i] - gamma * dh[i];
    fout[i] = (1.0 - beta) * f[i] + beta * fmirr + (fsh[i] - feq[i]);
  }
  return gamma;
}

/* One periodic multiphase step.  fin / fout: post-collision states [Q][n].
 * force (may be NULL): the total force F[3][n] used in the step. */
int or_step_multiphase(int lat, int nx, int ny, int nz, double beta, int mode, double kappa,
                       int eos, const double *g_ext, const double *fin, double *fout,
                       double *force) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  if (L.D == 2 && nz != 1) return -1;
  const long n = (long)nx * ny * nz;
  const int Q = L.Q;
  double *rho = (double *)malloc(sizeof(double) * n);
  double *phi = (double *)malloc(sizeof(double) * n);
  double *lap = (double *)malloc(sizeof(double) * n);
  if (!rho || !phi || !lap) {
    free(rho); free(phi); free(lap);
    return -2;
  }
  /* density after streaming */
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i)
          r += fin[i * n + idx3(wrap(x - L.c[i][0], nx), wrap(y - L.c[i][1], ny),
                                 wrap(z - L.c[i][2], nz), nx, ny)];
        const long k = idx3(x, y, z, nx, ny);
        rho[k] = r;
        const double s = r / 3.0 - eos_pressure(eos, r);
        phi[k] = sqrt(s > 0.0 ? s : 0.0);
      }
  /* lap rho */
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = idx3(x, y, z, nx, ny);
        double acc = 0.0;
        for (int i = 0; i < Q; ++i)
          acc += L.w[i] * (rho[idx3(wrap(x + L.c[i][0], nx), wrap(y + L.c[i][1], ny),
                                    wrap(z + L.c[i][2], nz), nx, ny)] - rho[k]);
        lap[k] = 6.0 * acc;
      }
  double f[OR_MAXQ], fo[OR_MAXQ];
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = idx3(x, y, z, nx, ny);
        double dphi[3] = {0, 0, 0}, dlap[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          const long kn = idx3(wrap(x + L.c[i][0], nx), wrap(y + L.c[i][1], ny),
                               wrap(z + L.c[i][2], nz), nx, ny);
          for (int a = 0; a < L.D; ++a) {
            dphi[a] += 3.0 * L.w[i] * L.c[i][a] * phi[kn];
            dlap[a] += 3.0 * L.w[i] * L.c[i][a] * lap[kn];
          }
        }
        double F[3] = {0, 0, 0}, du[3] = {0, 0, 0};
        for (int a = 0; a < L.D; ++a) {
          F[a] = 2.0 * phi[k] * dphi[a] + kappa * rho[k] * dlap[a];
          if (g_ext) F[a] += rho[k] * g_ext[a];
          du[a] = F[a] / rho[k];
        }
        if (force)
          for (int a = 0; a < 3; ++a) force[a * n + k] = F[a];
        for (int i = 0; i < Q; ++i)
          f[i] = fin[i * n + idx3(wrap(x - L.c[i][0], nx), wrap(y - L.c[i][1], ny),
                                   wrap(z - L.c[i][2], nz), nx, ny)];
        collide_forced(&L, beta, mode, f, du, fo);
        for (int i = 0; i < Q; ++i) fout[i * n + k] = fo[i];
      }
  free(rho); free(phi); free(lap);
  return 0;
}

/* ======================================================================
 * Multiphase step between two planar walls (section "Extensions to
 * fluid-structure interaction in multiphase flow": the wetting force F_s
 * and Grad's boundary condition in the multiphase model).
 *
 * The walls lie half a cell outside the faces normal to axis wa (q = 1/2,
 * at rest); the other axes are periodic.  Readings:
 *   - Grad fill of the missing populations of a wall node, as in the
 *     single-phase step with face walls: u_t = mean over the missing set of
 *     q u(x_b + c_i) / (1 + q), rho_t = sum of the known pulled populations
 *     plus the node's own stored f'_opp(i), grad u by finite differences
 *     (central, else one-sided second order through x_b, else first
 *     order), Pi = rho c_s^2 I + rho u u - rho c_s^2/(2 beta)(grad u +
 *     grad u^T), f*_i of Eq. (grad).  The velocities u(x, t-1) are the
 *     fluid velocities of the stored state, (j' - F_prev/2) / rho' (F_prev
 *     the force of the step that produced it; zero for a state set from
 *     outside).  The filled populations are pre-collision ones, whose
 *     momentum under the exact difference method is rho u - F/2: the
 *     target velocity is the interpolated fluid velocity minus
 *     F_prev(x_b) / (2 rho_t).  (Targeting the fluid velocity itself lets
 *     a wall-normal force at the wall node, e.g. the wetting force, inject
 *     mass every step: the fill returns the equilibrium share of rho_t
 *     while the outgoing populations carry the force's momentum.)
 *   - The fields rho, phi and lap rho of the stencils take, at the nodes
 *     beyond a wall, the value of the node across the wall (the mirror
 *     image at a wall half a cell out).
 *   - Wetting force F_s = kappa_w rho sum_i w_i s(x + c_i) c_i with w_i the
 *     lattice weights W_i (the paper leaves w_i open) and s = 1 for the
 *     nodes beyond a wall.
 *   F = 2 phi d(phi) + kappa rho d(lap rho) + F_s + rho g.
 * fin / fout: post-collision states [Q][n]; fprev (may be NULL): F_prev
 * [3][n]; force (may be NULL): the F of this step [3][n].
 * ====================================================================== */

/* node index with wrap on the periodic axes and the mirror across the walls
 * of axis wa */
static long mp_wall_idx(int x, int y, int z, const int *n, int wa, int *beyond) {
  int p[3] = {x, y, z};
  *beyond = 0;
  for (int a = 0; a < 3; ++a) {
    if (a == wa) {
      if (p[a] < 0) { p[a] = -1 - p[a]; *beyond = 1; }
      if (p[a] >= n[a]) { p[a] = 2 * n[a] - 1 - p[a]; *beyond = 1; }
    } else {
      p[a] = wrap(p[a], n[a]);
    }
  }
  return idx3(p[0], p[1], p[2], n[0], n[1]);
}

static double mp_grad_pop(const or_lattice *L, int i, double rho, const double *u,
                          const double Pi[3][3]) {
  const double cs2 = 1.0 / 3.0;
  double cu = 0.0, contr = 0.0;
  for (int a = 0; a < 3; ++a) cu += L->c[i][a] * u[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      contr += (Pi[a][b] - (a == b ? rho * cs2 : 0.0)) *
               (L->c[i][a] * L->c[i][b] - (a == b ? cs2 : 0.0));
  return L->w[i] * (rho + rho * cu / cs2 + contr / (2.0 * cs2 * cs2));
}

int or_step_multiphase_wall(int lat, int nx, int ny, int nz, double beta, int mode, double kappa,
                            int eos, const double *g_ext, double kappa_w, int wa,
                            const double *fin, const double *fprev, double *fout, double *force) {
  or_lattice L;
  if (make_lattice(lat, &L)) return -1;
  if (L.D == 2 && nz != 1) return -1;
  if (wa < 0 || wa >= L.D) return -1;
  const int n3[3] = {nx, ny, nz};
  if (n3[wa] < 3) return -1;
  const long n = (long)nx * ny * nz;
  const int Q = L.Q;
  double *f = (double *)malloc(sizeof(double) * Q * n);
  double *uo = (double *)malloc(sizeof(double) * 3 * n);
  double *rho = (double *)malloc(sizeof(double) * n);
  double *phi = (double *)malloc(sizeof(double) * n);
  double *lap = (double *)malloc(sizeof(double) * n);
  if (!f || !uo || !rho || !phi || !lap) {
    free(f); free(uo); free(rho); free(phi); free(lap);
    return -2;
  }
  /* fluid velocity of the stored state */
  for (long k = 0; k < n; ++k) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      r += fin[i * n + k];
      for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * fin[i * n + k];
    }
    for (int a = 0; a < 3; ++a) uo[a * n + k] = (j[a] - (fprev ? 0.5 * fprev[a * n + k] : 0.0)) / r;
  }
  /* pulled populations; Grad fill at the wall nodes */
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int p0[3] = {x, y, z};
        const long k = idx3(x, y, z, nx, ny);
        int miss[OR_MAXQ], nmiss = 0;
        for (int i = 0; i < Q; ++i) {
          int bey;
          const long ks = mp_wall_idx(x - L.c[i][0], y - L.c[i][1], z - L.c[i][2], n3, wa, &bey);
          miss[i] = bey;
          nmiss += bey;
          if (!bey) f[i * n + k] = fin[i * n + ks];
        }
        if (!nmiss) continue;
        double rho_t = 0.0, ut[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          if (!miss[i]) { rho_t += f[i * n + k]; continue; }
          rho_t += fin[(Q - 1 - i) * n + k];
          int p[3] = {x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]};
          if (p[wa] >= 0 && p[wa] < n3[wa]) {
            int bey;
            const long kn = mp_wall_idx(p[0], p[1], p[2], n3, wa, &bey);
            for (int a = 0; a < 3; ++a) ut[a] += (0.5 * uo[a * n + kn] / 1.5) / nmiss;
          }
        }
        /* grad u of the stored fluid velocity */
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int b = 0; b < L.D; ++b) {
          int pp[3] = {x, y, z};
          double um[3], up[3], um2[3], up2[3];
          int inm = 1, inp = 1, inm2 = 1, inp2 = 1;
          if (b == wa) {
            inm = p0[b] - 1 >= 0; inp = p0[b] + 1 < n3[b];
            inm2 = p0[b] - 2 >= 0; inp2 = p0[b] + 2 < n3[b];
          }
          for (int s = -2; s <= 2; ++s) {
            if (!s) continue;
            pp[0] = x; pp[1] = y; pp[2] = z;
            pp[b] += s;
            if (b == wa && (pp[b] < 0 || pp[b] >= n3[b])) continue;
            int bey;
            const long kk = mp_wall_idx(pp[0], pp[1], pp[2], n3, wa, &bey);
            double *dst = s == -1 ? um : s == 1 ? up : s == -2 ? um2 : up2;
            for (int a = 0; a < 3; ++a) dst[a] = uo[a * n + kk];
          }
          for (int a = 0; a < 3; ++a) {
            const double u0 = uo[a * n + k];
            if (inm && inp) G[a][b] = 0.5 * (up[a] - um[a]);
            else if (inp) G[a][b] = inp2 ? 0.5 * (-3.0 * u0 + 4.0 * up[a] - up2[a]) : up[a] - u0;
            else if (inm) G[a][b] = inm2 ? 0.5 * (3.0 * u0 - 4.0 * um[a] + um2[a]) : u0 - um[a];
          }
        }
        /* the filled populations are pre-collision ones, whose momentum is
         * rho u - F/2 for the fluid velocity u (exact difference method) */
        if (fprev)
          for (int a = 0; a < 3; ++a) ut[a] -= 0.5 * fprev[a * n + k] / rho_t;
        double Pi[3][3];
        const double cs2 = 1.0 / 3.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            Pi[a][b] = (a == b ? rho_t * cs2 : 0.0) + rho_t * ut[a] * ut[b] -
                       rho_t * cs2 / (2.0 * beta) * (G[a][b] + G[b][a]);
        for (int i = 0; i < Q; ++i)
          if (miss[i]) f[i * n + k] = mp_grad_pop(&L, i, rho_t, ut, Pi);
      }
  /* fields */
  for (long k = 0; k < n; ++k) {
    double r = 0.0;
    for (int i = 0; i < Q; ++i) r += f[i * n + k];
    rho[k] = r;
    const double s = r / 3.0 - eos_pressure(eos, r);
    phi[k] = sqrt(s > 0.0 ? s : 0.0);
  }
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = idx3(x, y, z, nx, ny);
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) {
          int bey;
          acc += L.w[i] * (rho[mp_wall_idx(x + L.c[i][0], y + L.c[i][1], z + L.c[i][2], n3, wa,
                                           &bey)] - rho[k]);
        }
        lap[k] = 6.0 * acc;
      }
  double fo[OR_MAXQ];
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = idx3(x, y, z, nx, ny);
        double dphi[3] = {0, 0, 0}, dlap[3] = {0, 0, 0}, sw[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          int bey;
          const long kn = mp_wall_idx(x + L.c[i][0], y + L.c[i][1], z + L.c[i][2], n3, wa, &bey);
          for (int a = 0; a < L.D; ++a) {
            dphi[a] += 3.0 * L.w[i] * L.c[i][a] * phi[kn];
            dlap[a] += 3.0 * L.w[i] * L.c[i][a] * lap[kn];
            if (bey) sw[a] += L.w[i] * L.c[i][a];
          }
        }
        double F[3] = {0, 0, 0}, du[3] = {0, 0, 0};
        for (int a = 0; a < L.D; ++a) {
          F[a] = 2.0 * phi[k] * dphi[a] + kappa * rho[k] * dlap[a] + kappa_w * rho[k] * sw[a];
          if (g_ext) F[a] += rho[k] * g_ext[a];
          du[a] = F[a] / rho[k];
        }
        if (force)
          for (int a = 0; a < 3; ++a) force[a * n + k] = F[a];
        double fl[OR_MAXQ];
        for (int i = 0; i < Q; ++i) fl[i] = f[i * n + k];
        collide_forced(&L, beta, mode, fl, du, fo);
        for (int i = 0; i < Q; ++i) fout[i * n + k] = fo[i];
      }
  free(f); free(uo); free(rho); free(phi); free(lap);
  return 0;
}

/* ======================================================================
 * Two-level grid refinement (the multi-domain refinement the paper uses in
 * its validation cases; the algorithm is cited, not printed).  D2Q9.
 * Reading:
 *   - A periodic coarse grid (nxc x nyc cells, node at the cell centre) and
 *     a fine patch of nfx x nfy nodes (spacing 1/2, two fine steps per
 *     coarse step: the same lattice velocity, nu_fine = 2 nu_coarse in
 *     lattice units) covering the coarse cells [i0, i0 + nfx/2) x
 *     [j0, j0 + nfy/2), its node (p, q) at coarse-cell coordinates
 *     (i0 + (p + 1/2)/2, j0 + (q + 1/2)/2).
 *   - Coarse -> fine: a fine node whose pull reaches outside the patch gets,
 *     for those populations only (as for a boundary node), Grad's
 *     approximation, Eq. (grad), Pi = rho c_s^2 I + rho u u - rho c_s^2/(2
 *     beta_f)(grad u + grad u^T), of the coarse fields rho, u (= j / rho)
 *     and grad u (central differences, in fine units: half the coarse-unit
 *     gradient) interpolated bilinearly to the node itself and linearly in
 *     time to the fine time of the pull (t + 1/2, t + 1): the pre-collision
 *     populations the node would receive.  (Grad's form evaluated at the
 *     source node instead stands for a pre-collision state where a pulled
 *     population is post-collision; its non-equilibrium part then has
 *     nearly the opposite sign at beta near 1.)
 *   - Fine -> coarse: after the two fine steps each covered coarse cell takes
 *     Grad's approximation (beta_c) of the mean density, momentum and
 *     velocity gradient of its 2 x 2 fine children (the gradient by central
 *     differences of the fine velocity, the ghost ring holding the coarse
 *     values of time t + 1, and doubled to coarse units), then the coarse
 *     KBC collision: the stored post-collision state of that cell.
 *   - Order per coarse step: the coarse step over all cells (the covered
 *     ones hold the restricted state), two fine steps, the restriction.
 * fc: coarse post-collision state [9][nyc][nxc]; ff: fine [9][nfy][nfx].
 * ====================================================================== */

static void ref_grad_pop_all(const or_lattice *L, double rho, const double *u, const double G[2][2],
                             double beta, double *f) {
  const double cs2 = 1.0 / 3.0;
  double Pn[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      Pn[a][b] = rho * u[a] * u[b] - rho * cs2 / (2.0 * beta) * (G[a][b] + G[b][a]);
  for (int i = 0; i < L->Q; ++i) {
    double cu = 0.0, contr = 0.0;
    for (int a = 0; a < 2; ++a) cu += L->c[i][a] * u[a];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        contr += Pn[a][b] * (L->c[i][a] * L->c[i][b] - (a == b ? cs2 : 0.0));
    f[i] = L->w[i] * (rho + rho * cu / cs2 + contr / (2.0 * cs2 * cs2));
  }
}

/* rho, u and grad u (coarse units, central differences) of a periodic coarse state */
static void ref_coarse_fields(const or_lattice *L, const double *fc, int nx, int ny, double *rho,
                              double *u /*[2][n]*/, double *G /*[4][n]*/) {
  const long n = (long)nx * ny;
  for (long k = 0; k < n; ++k) {
    double r = 0.0, j[2] = {0, 0};
    for (int i = 0; i < L->Q; ++i) {
      r += fc[i * n + k];
      j[0] += L->c[i][0] * fc[i * n + k];
      j[1] += L->c[i][1] * fc[i * n + k];
    }
    rho[k] = r;
    u[k] = j[0] / r;
    u[n + k] = j[1] / r;
  }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const long k = (long)y * nx + x;
      const long xp = (long)y * nx + wrap(x + 1, nx), xm = (long)y * nx + wrap(x - 1, nx);
      const long yp = (long)wrap(y + 1, ny) * nx + x, ym = (long)wrap(y - 1, ny) * nx + x;
      for (int a = 0; a < 2; ++a) {
        G[(2 * a + 0) * n + k] = 0.5 * (u[a * n + xp] - u[a * n + xm]);
        G[(2 * a + 1) * n + k] = 0.5 * (u[a * n + yp] - u[a * n + ym]);
      }
    }
}

/* Lagrange weights of the four nodes -1, 0, 1, 2 at the offset t in [0, 1) */
static void ref_cubic_w(double t, double *w) {
  w[0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
  w[1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
  w[2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
  w[3] = (t + 1.0) * t * (t - 1.0) / 6.0;
}

/* bicubic (tensor-product Lagrange, 4 x 4 nodes) value of a periodic coarse
 * field at coarse-cell coordinates (X, Y).  (Bilinear interpolation damps a
 * Fourier mode by O(h^2 k^2) at every transfer; applied every coarse step
 * that acts as an extra diffusion of the order of the grid spacing.) */
static double ref_bilinear(const double *v, int nx, int ny, double X, double Y) {
  const double sx = X - 0.5, sy = Y - 0.5;
  const int ix = (int)floor(sx), iy = (int)floor(sy);
  double wx[4], wy[4];
  ref_cubic_w(sx - ix, wx);
  ref_cubic_w(sy - iy, wy);
  double acc = 0.0;
  for (int b = 0; b < 4; ++b)
    for (int a = 0; a < 4; ++a)
      acc += wx[a] * wy[b] * v[(long)wrap(iy - 1 + b, ny) * nx + wrap(ix - 1 + a, nx)];
  return acc;
}

int or_refine_step(int nxc, int nyc, double beta_c, double beta_f, int mode, int i0, int j0,
                   int nfx, int nfy, const double *fc_in, const double *ff_in, double *fc_out,
                   double *ff_out) {
  or_lattice L;
  if (make_lattice(9, &L)) return -1;
  if (nfx < 2 || nfy < 2 || (nfx & 1) || (nfy & 1)) return -1;
  if (nfx / 2 > nxc - 2 || nfy / 2 > nyc - 2) return -1;
  const int Q = 9;
  const long nc = (long)nxc * nyc, nf = (long)nfx * nfy;
  double *rc0 = malloc(sizeof(double) * nc), *uc0 = malloc(sizeof(double) * 2 * nc);
  double *gc0 = malloc(sizeof(double) * 4 * nc), *rc1 = malloc(sizeof(double) * nc);
  double *uc1 = malloc(sizeof(double) * 2 * nc), *gc1 = malloc(sizeof(double) * 4 * nc);
  double *fa = malloc(sizeof(double) * Q * nf), *fb = malloc(sizeof(double) * Q * nf);
  if (!rc0 || !uc0 || !gc0 || !rc1 || !uc1 || !gc1 || !fa || !fb) return -2;
  ref_coarse_fields(&L, fc_in, nxc, nyc, rc0, uc0, gc0);
  /* coarse step over all cells */
  if (or_step_periodic(9, nxc, nyc, 1, beta_c, mode, fc_in, fc_out, NULL)) return -1;
  ref_coarse_fields(&L, fc_out, nxc, nyc, rc1, uc1, gc1);
  memcpy(fa, ff_in, sizeof(double) * Q * nf);
  double f[OR_MAXQ], fo[OR_MAXQ], g;
  for (int k = 0; k < 2; ++k) {
    const double w = 0.5 * (k + 1);  /* fine time of the pull, in coarse steps after t */
    for (int q = 0; q < nfy; ++q)
      for (int p = 0; p < nfx; ++p) {
        const long kf = (long)q * nfx + p;
        int nmiss = 0;
        for (int i = 0; i < Q; ++i) {
          const int ps = p - L.c[i][0], qs = q - L.c[i][1];
          if (ps >= 0 && ps < nfx && qs >= 0 && qs < nfy) f[i] = fa[i * nf + (long)qs * nfx + ps];
          else nmiss++;
        }
        if (nmiss) {
          const double X = i0 + 0.5 * (p + 0.5), Y = j0 + 0.5 * (q + 0.5);
          double r = (1 - w) * ref_bilinear(rc0, nxc, nyc, X, Y) + w * ref_bilinear(rc1, nxc, nyc, X, Y);
          double uu[2], G[2][2], fg[OR_MAXQ];
          for (int a = 0; a < 2; ++a)
            uu[a] = (1 - w) * ref_bilinear(uc0 + a * nc, nxc, nyc, X, Y) +
                    w * ref_bilinear(uc1 + a * nc, nxc, nyc, X, Y);
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
              G[a][b] = 0.5 * ((1 - w) * ref_bilinear(gc0 + (2 * a + b) * nc, nxc, nyc, X, Y) +
                               w * ref_bilinear(gc1 + (2 * a + b) * nc, nxc, nyc, X, Y));
          ref_grad_pop_all(&L, r, uu, G, beta_f, fg);
          for (int i = 0; i < Q; ++i) {
            const int ps = p - L.c[i][0], qs = q - L.c[i][1];
            if (!(ps >= 0 && ps < nfx && qs >= 0 && qs < nfy)) f[i] = fg[i];
          }
        }
        collide(&L, beta_f, mode, f, fo, &g, NULL, NULL, NULL);
        for (int i = 0; i < Q; ++i) fb[i * nf + kf] = fo[i];
      }
    double *t = fa; fa = fb; fb = t;
  }
  memcpy(ff_out, fa, sizeof(double) * Q * nf);
  /* fine fields at t + 1: rho, u on the patch; u on the ghost ring from the coarse fields */
  const int gx = nfx + 2, gy = nfy + 2;
  double *uf = malloc(sizeof(double) * 2 * gx * gy), *rf = malloc(sizeof(double) * gx * gy);
  double *jf = malloc(sizeof(double) * 2 * gx * gy);
  if (!uf || !rf || !jf) return -2;
  for (int q = -1; q <= nfy; ++q)
    for (int p = -1; p <= nfx; ++p) {
      const long kg = (long)(q + 1) * gx + (p + 1);
      if (p >= 0 && p < nfx && q >= 0 && q < nfy) {
        const long kf = (long)q * nfx + p;
        double r = 0.0, j[2] = {0, 0};
        for (int i = 0; i < Q; ++i) {
          r += fa[i * nf + kf];
          j[0] += L.c[i][0] * fa[i * nf + kf];
          j[1] += L.c[i][1] * fa[i * nf + kf];
        }
        rf[kg] = r;
        jf[kg] = j[0];
        jf[gx * gy + kg] = j[1];
        uf[kg] = j[0] / r;
        uf[gx * gy + kg] = j[1] / r;
      } else {
        const double X = i0 + 0.5 * (p + 0.5), Y = j0 + 0.5 * (q + 0.5);
        const double r = ref_bilinear(rc1, nxc, nyc, X, Y);
        rf[kg] = r;
        for (int a = 0; a < 2; ++a) {
          uf[a * gx * gy + kg] = ref_bilinear(uc1 + a * nc, nxc, nyc, X, Y);
          jf[a * gx * gy + kg] = r * uf[a * gx * gy + kg];
        }
      }
    }
  /* restriction: the coarse-centre values by the cubic midpoint rule over the
   * fine nodes 2I-1 .. 2I+2 of each axis (weights -1, 9, 9, -1 over 16; the
   * outer ones on the ghost ring for the cells along the patch edge), the
   * velocity gradient from the midpoint values of the neighbouring fine
   * pairs (spacing 1/2 apart: one-sided pairs at the patch edge use the
   * ghost ring too) */
  static const double wm[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
  for (int J = 0; J < nfy / 2; ++J)
    for (int I = 0; I < nfx / 2; ++I) {
      double r = 0.0, j[2] = {0, 0}, G[2][2] = {{0, 0}, {0, 0}};
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          const int p = 2 * I - 1 + a, q = 2 * J - 1 + b;
          const long kg = (long)(q + 1) * gx + (p + 1);
          const double ww = wm[a] * wm[b];
          r += ww * rf[kg];
          j[0] += ww * jf[kg];
          j[1] += ww * jf[gx * gy + kg];
        }
      /* d/dx at the centre: fine-unit differences of the pairs (2I+1 - 2I) on
       * the rows, midpoint-interpolated across, doubled to coarse units */
      for (int a = 0; a < 2; ++a) {
        double dx = 0.0, dy = 0.0;
        for (int b = 0; b < 4; ++b) {
          const int q = 2 * J - 1 + b;
          const long k0 = (long)(q + 1) * gx + (2 * I + 1), k1 = k0 + 1;
          dx += wm[b] * (uf[a * gx * gy + k1] - uf[a * gx * gy + k0]);
          const int p = 2 * I - 1 + b;
          const long l0 = (long)(2 * J + 1) * gx + (p + 1), l1 = l0 + gx;
          dy += wm[b] * (uf[a * gx * gy + l1] - uf[a * gx * gy + l0]);
        }
        G[a][0] = 2.0 * dx;
        G[a][1] = 2.0 * dy;
      }
      const double uu[2] = {j[0] / r, j[1] / r};
      double fg[OR_MAXQ];
      ref_grad_pop_all(&L, r, uu, G, beta_c, fg);
      collide(&L, beta_c, mode, fg, fo, &g, NULL, NULL, NULL);
      const long kc = (long)(j0 + J) * nxc + (i0 + I);
      for (int i = 0; i < Q; ++i) fc_out[i * nc + kc] = fo[i];
    }
  free(rc0); free(uc0); free(gc0); free(rc1); free(uc1); free(gc1); free(fa); free(fb);
  free(uf); free(rf); free(jf);
  return 0;
}
