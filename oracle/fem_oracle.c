/*
 * fem_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Double-precision CPU statement of the structural step: a geometrically
 * nonlinear 2-D co-rotational Euler-Bernoulli beam (the structure model the
 * paper's flag cases reduce to), integrated with the one-step-theta scheme of
 * Eq. (timeInt) in the two-field (v, u) form, Eqs. (timeDiscrete_solid_velocity)
 * and (timeDiscrete_solid_displacement), and solved with Newton-Raphson plus
 * the constant line-search relaxation lambda = 0.7 of section "Structural
 * modeling".  Plain dense Gaussian elimination with partial pivoting.
 *
 * Readings (the paper uses Q2 continuum elements; the beam replaces them):
 *   element a-b, reference length L0, chord angle b0; current chord length L
 *   and angle b; local deformations ul = L - L0, t1 = th_a - (b - b0),
 *   t2 = th_b - (b - b0); local forces N = EA ul / L0,
 *   M1 = 2EI/L0 (2 t1 + t2), M2 = 2EI/L0 (t1 + 2 t2);
 *   internal force f = B^T (N, M1, M2) with B the derivative of (ul, t1, t2)
 *   with respect to (ux_a, uy_a, th_a, ux_b, uy_b, th_b);
 *   tangent K = B^T D B + N/L z z^T + (M1 + M2)/L^2 (r z^T + z r^T),
 *   r = (-c, -s, 0, c, s, 0), z = (s, -c, 0, -s, c, 0);
 *   mass: the consistent (Hermite) mass matrix of the linear element in the
 *   reference orientation (constant);
 *   theta-scheme: M (v1 - v0)/dt = th (F1 - f(u1)) + (1 - th)(F0 - f(u0)),
 *                 (u1 - u0)/dt = th v1 + (1 - th) v0;
 *   Newton on u1 with J = M/(th dt^2) + th K(u1), update u1 += lambda du;
 *   stop when |R| <= rtol |R0| + atol or after max_it iterations.
 * DOF layout: node j owns (3j, 3j+1, 3j+2) = (ux, uy, th); fixed DOFs are
 * given by a mask.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

typedef struct {
  int nn;             /* nodes */
  const double *X;    /* [nn][2] reference positions */
  double EA, EI, rhoA;
  const int *fixed;   /* [3 nn] 1 = Dirichlet (held at zero displacement) */
} beam_t;

/* Internal force f[3nn] and (optionally) tangent K[3nn][3nn] at displacement u. */
static void beam_internal(const beam_t *B, const double *u, double *f, double *K) {
  const int n = 3 * B->nn;
  memset(f, 0, sizeof(double) * n);
  if (K) memset(K, 0, sizeof(double) * n * n);
  for (int e = 0; e < B->nn - 1; ++e) {
    const int a = e, b = e + 1;
    const double X0x = B->X[2 * b] - B->X[2 * a], X0y = B->X[2 * b + 1] - B->X[2 * a + 1];
    const double L0 = sqrt(X0x * X0x + X0y * X0y), b0 = atan2(X0y, X0x);
    const double dx = X0x + u[3 * b] - u[3 * a], dy = X0y + u[3 * b + 1] - u[3 * a + 1];
    const double L = sqrt(dx * dx + dy * dy), bb = atan2(dy, dx);
    const double c = dx / L, s = dy / L;
    double rot = bb - b0; /* rigid rotation of the chord, wrapped to (-pi, pi] */
    while (rot > OR_PI) rot -= 2 * OR_PI;
    while (rot <= -OR_PI) rot += 2 * OR_PI;
    const double ul = L - L0, t1 = u[3 * a + 2] - rot, t2 = u[3 * b + 2] - rot;
    const double N = B->EA * ul / L0;
    const double k2 = 2.0 * B->EI / L0;
    const double M1 = k2 * (2 * t1 + t2), M2 = k2 * (t1 + 2 * t2);
    const double r[6] = {-c, -s, 0, c, s, 0};
    const double z[6] = {s, -c, 0, -s, c, 0};
    double Bm[3][6];
    for (int k = 0; k < 6; ++k) {
      Bm[0][k] = r[k];
      Bm[1][k] = -z[k] / L;
      Bm[2][k] = -z[k] / L;
    }
    Bm[1][2] += 1.0;
    Bm[2][5] += 1.0;
    const double q[3] = {N, M1, M2};
    const int dof[6] = {3 * a, 3 * a + 1, 3 * a + 2, 3 * b, 3 * b + 1, 3 * b + 2};
    for (int k = 0; k < 6; ++k)
      for (int m = 0; m < 3; ++m) f[dof[k]] += Bm[m][k] * q[m];
    if (K) {
      const double D[3][3] = {{B->EA / L0, 0, 0}, {0, 2 * k2, k2}, {0, k2, 2 * k2}};
      for (int k = 0; k < 6; ++k)
        for (int l = 0; l < 6; ++l) {
          double v = 0.0;
          for (int m = 0; m < 3; ++m)
            for (int p = 0; p < 3; ++p) v += Bm[m][k] * D[m][p] * Bm[p][l];
          v += N / L * z[k] * z[l] + (M1 + M2) / (L * L) * (r[k] * z[l] + z[k] * r[l]);
          K[dof[k] * n + dof[l]] += v;
        }
    }
  }
}

/* Consistent mass matrix M[3nn][3nn]. */
static void beam_mass(const beam_t *B, double *M) {
  const int n = 3 * B->nn;
  memset(M, 0, sizeof(double) * n * n);
  for (int e = 0; e < B->nn - 1; ++e) {
    const int a = e, b = e + 1;
    const double X0x = B->X[2 * b] - B->X[2 * a], X0y = B->X[2 * b + 1] - B->X[2 * a + 1];
    const double L = sqrt(X0x * X0x + X0y * X0y);
    const double c = X0x / L, s = X0y / L;
    /* local DOFs (u_a, v_a, th_a, u_b, v_b, th_b) */
    double Ml[6][6] = {{0}};
    const double ma = B->rhoA * L / 6.0, mb = B->rhoA * L / 420.0;
    Ml[0][0] = 2 * ma; Ml[0][3] = ma; Ml[3][0] = ma; Ml[3][3] = 2 * ma;
    const int bi[4] = {1, 2, 4, 5};
    const double Mb[4][4] = {{156, 22 * L, 54, -13 * L},
                             {22 * L, 4 * L * L, 13 * L, -3 * L * L},
                             {54, 13 * L, 156, -22 * L},
                             {-13 * L, -3 * L * L, -22 * L, 4 * L * L}};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) Ml[bi[i]][bi[j]] = mb * Mb[i][j];
    /* rotation to global: local (u, v) = R (ux, uy), R = [[c, s], [-s, c]] */
    double T[6][6] = {{0}};
    for (int k = 0; k < 2; ++k) {
      T[3 * k][3 * k] = c; T[3 * k][3 * k + 1] = s;
      T[3 * k + 1][3 * k] = -s; T[3 * k + 1][3 * k + 1] = c;
      T[3 * k + 2][3 * k + 2] = 1;
    }
    const int dof[6] = {3 * a, 3 * a + 1, 3 * a + 2, 3 * b, 3 * b + 1, 3 * b + 2};
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
        for (int k = 0; k < 6; ++k)
          for (int l = 0; l < 6; ++l) v += T[k][i] * Ml[k][l] * T[l][j];
        M[dof[i] * n + dof[j]] += v;
      }
  }
}

/* Solve A x = b in place (A destroyed), Gaussian elimination with partial
 * pivoting; returns 0 on success. */
static int dense_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
      }
      double t = b[k]; b[k] = b[p]; b[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      const double m = A[i * n + k] / A[k * n + k];
      if (m == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
      b[i] -= m * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
    b[k] = s / A[k * n + k];
  }
  return 0;
}

/* Apply Dirichlet rows/columns: unit diagonal, zero residual. */
static void apply_fixed(const beam_t *B, double *J, double *R) {
  const int n = 3 * B->nn;
  for (int i = 0; i < n; ++i) {
    if (!B->fixed[i]) continue;
    for (int j = 0; j < n; ++j) { J[i * n + j] = 0.0; J[j * n + i] = 0.0; }
    J[i * n + i] = 1.0;
    R[i] = 0.0;
  }
}

static double norm(int n, const double *v) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

/* One theta-scheme step.  u, v: [3nn] state, updated in place.  F0, F1:
 * external nodal loads at t_n and t_{n+1}.  Returns the Newton iteration
 * count (negative if not converged). */
int or_beam_step(int nn, const double *X, double EA, double EI, double rhoA, const int *fixed,
                 double dt, double theta, double lambda, double rtol, double atol, int max_it,
                 const double *F0, const double *F1, double *u, double *v) {
  beam_t B = {nn, X, EA, EI, rhoA, fixed};
  const int n = 3 * nn;
  double *M = malloc(sizeof(double) * n * n), *K = malloc(sizeof(double) * n * n);
  double *J = malloc(sizeof(double) * n * n);
  double *f0 = malloc(sizeof(double) * n), *f1 = malloc(sizeof(double) * n);
  double *u0 = malloc(sizeof(double) * n), *v0 = malloc(sizeof(double) * n);
  double *R = malloc(sizeof(double) * n), *v1 = malloc(sizeof(double) * n);
  beam_mass(&B, M);
  memcpy(u0, u, sizeof(double) * n);
  memcpy(v0, v, sizeof(double) * n);
  beam_internal(&B, u0, f0, NULL);
  int it, conv = 0;
  double r0 = -1.0;
  for (it = 0; it < max_it; ++it) {
    beam_internal(&B, u, f1, K);
    for (int i = 0; i < n; ++i) v1[i] = ((u[i] - u0[i]) / dt - (1.0 - theta) * v0[i]) / theta;
    for (int i = 0; i < n; ++i) {
      double mv = 0.0;
      for (int j = 0; j < n; ++j) mv += M[i * n + j] * (v1[j] - v0[j]);
      R[i] = mv / dt - theta * (F1[i] - f1[i]) - (1.0 - theta) * (F0[i] - f0[i]);
    }
    for (int i = 0; i < n; ++i)
      if (fixed[i]) R[i] = 0.0;
    const double rn = norm(n, R);
    if (r0 < 0) r0 = rn;
    if (rn <= rtol * r0 + atol) { conv = 1; break; }
    for (int i = 0; i < n * n; ++i) J[i] = M[i] / (theta * dt * dt) + theta * K[i];
    apply_fixed(&B, J, R);
    for (int i = 0; i < n; ++i) R[i] = -R[i];
    if (dense_solve(n, J, R)) break;
    for (int i = 0; i < n; ++i) u[i] += lambda * R[i];
  }
  for (int i = 0; i < n; ++i) {
    if (fixed[i]) { u[i] = 0.0; v[i] = 0.0; continue; }
    v[i] = ((u[i] - u0[i]) / dt - (1.0 - theta) * v0[i]) / theta;
  }
  free(M); free(K); free(J); free(f0); free(f1); free(u0); free(v0); free(R); free(v1);
  return conv ? it : -it - 1;
}

/* Static equilibrium f_int(u) = F by full Newton (lambda = 1 unless given).
 * Returns iterations (negative if not converged). */
int or_beam_static(int nn, const double *X, double EA, double EI, const int *fixed,
                   const double *F, double lambda, double rtol, double atol, int max_it,
                   double *u) {
  beam_t B = {nn, X, EA, EI, 0.0, fixed};
  const int n = 3 * nn;
  double *K = malloc(sizeof(double) * n * n), *f = malloc(sizeof(double) * n);
  double *R = malloc(sizeof(double) * n);
  int it, conv = 0;
  double r0 = -1;
  for (it = 0; it < max_it; ++it) {
    beam_internal(&B, u, f, K);
    for (int i = 0; i < n; ++i) R[i] = fixed[i] ? 0.0 : F[i] - f[i];
    const double rn = norm(n, R);
    if (r0 < 0) r0 = rn > 0 ? rn : 1.0;
    if (rn <= rtol * r0 + atol) { conv = 1; break; }
    apply_fixed(&B, K, R);
    if (dense_solve(n, K, R)) break;
    for (int i = 0; i < n; ++i) u[i] += lambda * R[i];
  }
  free(K); free(f); free(R);
  return conv ? it : -it - 1;
}

/* Internal force and tangent, exported for tests. */
int or_beam_internal(int nn, const double *X, double EA, double EI, const double *u, double *f,
                     double *K) {
  beam_t B = {nn, X, EA, EI, 0.0, NULL};
  beam_internal(&B, u, f, K);
  return 0;
}

int or_beam_mass(int nn, const double *X, double rhoA, double *M) {
  beam_t B = {nn, X, 0.0, 0.0, rhoA, NULL};
  beam_mass(&B, M);
  return 0;
}
