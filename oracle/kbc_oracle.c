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
