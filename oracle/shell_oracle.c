/*
 * shell_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Double-precision CPU statement of the 3-D structural step for the plate
 * cases: a geometrically nonlinear co-rotational flat shell of 4-node
 * quadrilaterals on a structured nx x ny node grid, integrated with the
 * one-step-theta scheme of Eq. (timeInt) in the two-field (v, u) form and
 * solved with Newton-Raphson plus the constant relaxation lambda = 0.7 of
 * section "Structural modeling".  (The paper uses Q2 continuum elements; the
 * flat shell replaces them for the plate.)
 *
 * Readings:
 *  - node n = i ny + j (i along the length, j along the width); element
 *    (i, j) has nodes (i,j), (i+1,j), (i+1,j+1), (i,j+1); six DOFs per node:
 *    translations (ux, uy, uz) and a rotation, kept as a rotation matrix R_n
 *    (R_n = I in the reference state);
 *  - element frame: e3 along (x3 - x1) x (x4 - x2), e1 along the part of
 *    (x2 + x3 - x1 - x4) normal to e3, e2 = e3 x e1, origin at the mean of
 *    the four nodes;
 *  - local deformations: translations d_t = R_e^T (x - c) - (reference local
 *    position), rotations d_r = log(R_e^T R_n R_e0) (axial vector);
 *  - local element: linear, constant stiffness from the reference geometry:
 *    plane-stress membrane (bilinear, 2x2 Gauss), Mindlin plate bending
 *    (2x2 Gauss) with MITC4 transverse shear (covariant strains tied at the
 *    edge midpoints, shear factor 5/6), drilling stiffness 1e-3 D on the
 *    rotation about e3, D = E h^3 / (12 (1 - nu^2)); rotation about local x
 *    tilts the normal towards -y, about local y towards +x;
 *  - internal force f = T^T P^T K_l d (T: rotation of each node's
 *    translation and rotation triplets into the element frame; P: projector
 *    removing the rigid motion of the element frame, whose spin follows from
 *    the frame definition); tangent T^T P^T K_l P T (without the geometric
 *    terms of the projector's variation; Newton with the constant relaxation
 *    converges linearly either way);
 *  - mass: lumped, rho h A / 4 per node and element for the translations,
 *    rho h^3/12 A / 4 for the three rotations;
 *  - theta-scheme with rotations: the step's rotation vector phi_n
 *    (R_n^{k+1} = exp(phi_n) R_n^k) plays the role of the rotational
 *    displacement increment, angular velocities that of the rotational
 *    velocities; Newton corrections of phi are added;
 *  - stop when |R| <= rtol |R0| + atol (R0: residual at the step's start)
 *    or after max_it iterations; banded Gaussian elimination without
 *    pivoting for the linear systems.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int nx, ny, nn, ne, n, kb;
  const double *X;   /* [nn][3] */
  double E, nu, h, rho;
  const int *fixed;  /* [6 nn] */
  double *Kl;        /* [ne][24][24] local stiffness */
  double *Re0;       /* [ne][3][3] reference frames (columns e1 e2 e3) */
  double *xb0;       /* [ne][4][3] reference local node positions */
  double *m, *Jr;    /* [nn] lumped translational mass / rotational inertia */
} shell_t;

/* ------------------------------------------------------------ rotations */
static void skew(const double *a, double S[3][3]) {
  S[0][0] = 0; S[0][1] = -a[2]; S[0][2] = a[1];
  S[1][0] = a[2]; S[1][1] = 0; S[1][2] = -a[0];
  S[2][0] = -a[1]; S[2][1] = a[0]; S[2][2] = 0;
}

/* exp of the skew matrix of phi (Rodrigues' formula). */
static void rot_exp(const double *phi, double R[3][3]) {
  const double t = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  double S[3][3], S2[3][3];
  skew(phi, S);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S2[i][j] = 0;
      for (int k = 0; k < 3; ++k) S2[i][j] += S[i][k] * S[k][j];
    }
  double a, b;
  if (t < 1e-6) {
    a = 1.0 - t * t / 6.0;
    b = 0.5 - t * t / 24.0;
  } else {
    a = sin(t) / t;
    b = (1.0 - cos(t)) / (t * t);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = (i == j ? 1.0 : 0.0) + a * S[i][j] + b * S2[i][j];
}

/* Axial vector of log(R) for a rotation by less than pi. */
static void rot_log(const double R[3][3], double *phi) {
  const double w[3] = {R[2][1] - R[1][2], R[0][2] - R[2][0], R[1][0] - R[0][1]};
  double c = 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1.0);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  const double t = acos(c);
  const double s = sin(t);
  const double f = (t < 1e-6) ? 0.5 * (1.0 + t * t / 6.0) : 0.5 * t / s;
  for (int i = 0; i < 3; ++i) phi[i] = f * w[i];
}

static void mat_mul(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C[i][j] = 0;
      for (int k = 0; k < 3; ++k) C[i][j] += A[i][k] * B[k][j];
    }
}

static void mat_tmul(const double A[3][3], const double B[3][3], double C[3][3]) { /* A^T B */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C[i][j] = 0;
      for (int k = 0; k < 3; ++k) C[i][j] += A[k][i] * B[k][j];
    }
}

/* Element frame (columns e1, e2, e3) and centre of four points. */
static void quad_frame(const double x[4][3], double R[3][3], double c[3]) {
  double d13[3], d24[3], n[3], a[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.25 * (x[0][k] + x[1][k] + x[2][k] + x[3][k]);
    d13[k] = x[2][k] - x[0][k];
    d24[k] = x[3][k] - x[1][k];
    a[k] = x[1][k] + x[2][k] - x[0][k] - x[3][k];
  }
  n[0] = d13[1] * d24[2] - d13[2] * d24[1];
  n[1] = d13[2] * d24[0] - d13[0] * d24[2];
  n[2] = d13[0] * d24[1] - d13[1] * d24[0];
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double e3[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
  const double ae = a[0] * e3[0] + a[1] * e3[1] + a[2] * e3[2];
  double e1[3] = {a[0] - ae * e3[0], a[1] - ae * e3[1], a[2] - ae * e3[2]};
  const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int k = 0; k < 3; ++k) e1[k] /= l1;
  const double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                        e3[0] * e1[1] - e3[1] * e1[0]};
  for (int k = 0; k < 3; ++k) {
    R[k][0] = e1[k];
    R[k][1] = e2[k];
    R[k][2] = e3[k];
  }
}

static void elem_nodes(const shell_t *S, int e, int id[4]) {
  const int i = e / (S->ny - 1), j = e % (S->ny - 1);
  id[0] = i * S->ny + j;
  id[1] = (i + 1) * S->ny + j;
  id[2] = (i + 1) * S->ny + j + 1;
  id[3] = i * S->ny + j + 1;
}

/* ------------------------------------------------------------ local element */
static const double XI[4] = {-1, 1, 1, -1}, ETA[4] = {-1, -1, 1, 1};

static void shape(double xi, double eta, double N[4], double Nxi[4], double Neta[4]) {
  for (int a = 0; a < 4; ++a) {
    N[a] = 0.25 * (1 + xi * XI[a]) * (1 + eta * ETA[a]);
    Nxi[a] = 0.25 * XI[a] * (1 + eta * ETA[a]);
    Neta[a] = 0.25 * ETA[a] * (1 + xi * XI[a]);
  }
}

/* Row of the covariant transverse shear strain along xi (dir 0) or eta (dir 1)
 * at (xi, eta): w_,dir + beta_x x_,dir + beta_y y_,dir with beta_x = theta_y,
 * beta_y = -theta_x. */
static void shear_row(const double xl[4][2], double xi, double eta, int dir, double row[24]) {
  double N[4], Nxi[4], Neta[4];
  shape(xi, eta, N, Nxi, Neta);
  const double *Nd = dir == 0 ? Nxi : Neta;
  double xd = 0, yd = 0;
  for (int a = 0; a < 4; ++a) {
    xd += Nd[a] * xl[a][0];
    yd += Nd[a] * xl[a][1];
  }
  memset(row, 0, sizeof(double) * 24);
  for (int a = 0; a < 4; ++a) {
    row[6 * a + 2] = Nd[a];
    row[6 * a + 4] = N[a] * xd;
    row[6 * a + 3] = -N[a] * yd;
  }
}

static void add_btdb(double K[24][24], const double *B, int rows, const double *D, double w) {
  /* K += w B^T D B, B [rows][24], D [rows][rows] */
  double DB[3][24];
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < 24; ++c) {
      DB[r][c] = 0;
      for (int k = 0; k < rows; ++k) DB[r][c] += D[r * rows + k] * B[k * 24 + c];
    }
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      double s = 0;
      for (int r = 0; r < rows; ++r) s += B[r * 24 + i] * DB[r][j];
      K[i][j] += w * s;
    }
}

static void local_stiffness(const shell_t *S, const double xl[4][2], double K[24][24]) {
  memset(K, 0, sizeof(double) * 576);
  const double E = S->E, nu = S->nu, h = S->h;
  const double cm = E * h / (1 - nu * nu), cb = E * h * h * h / (12 * (1 - nu * nu));
  const double Dm[9] = {cm, cm * nu, 0, cm * nu, cm, 0, 0, 0, cm * (1 - nu) / 2};
  const double Db[9] = {cb, cb * nu, 0, cb * nu, cb, 0, 0, 0, cb * (1 - nu) / 2};
  const double ks = 5.0 / 6.0 * E / (2 * (1 + nu)) * h;
  const double Ds[4] = {ks, 0, 0, ks};
  const double g = 1.0 / sqrt(3.0);
  double rA[24], rC[24], rD[24], rB[24];
  shear_row(xl, 0, -1, 0, rA);
  shear_row(xl, 0, 1, 0, rC);
  shear_row(xl, -1, 0, 1, rD);
  shear_row(xl, 1, 0, 1, rB);
  for (int gp = 0; gp < 4; ++gp) {
    const double xi = g * XI[gp], eta = g * ETA[gp];
    double N[4], Nxi[4], Neta[4];
    shape(xi, eta, N, Nxi, Neta);
    double J[2][2] = {{0, 0}, {0, 0}};
    for (int a = 0; a < 4; ++a) {
      J[0][0] += Nxi[a] * xl[a][0]; J[0][1] += Nxi[a] * xl[a][1];
      J[1][0] += Neta[a] * xl[a][0]; J[1][1] += Neta[a] * xl[a][1];
    }
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double iJ[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    double Nx[4], Ny[4];
    for (int a = 0; a < 4; ++a) {
      Nx[a] = iJ[0][0] * Nxi[a] + iJ[0][1] * Neta[a];
      Ny[a] = iJ[1][0] * Nxi[a] + iJ[1][1] * Neta[a];
    }
    double Bm[3 * 24], Bb[3 * 24], Bs[2 * 24];
    memset(Bm, 0, sizeof(Bm));
    memset(Bb, 0, sizeof(Bb));
    for (int a = 0; a < 4; ++a) {
      Bm[0 * 24 + 6 * a + 0] = Nx[a];
      Bm[1 * 24 + 6 * a + 1] = Ny[a];
      Bm[2 * 24 + 6 * a + 0] = Ny[a];
      Bm[2 * 24 + 6 * a + 1] = Nx[a];
      Bb[0 * 24 + 6 * a + 4] = Nx[a];
      Bb[1 * 24 + 6 * a + 3] = -Ny[a];
      Bb[2 * 24 + 6 * a + 4] = Ny[a];
      Bb[2 * 24 + 6 * a + 3] = -Nx[a];
    }
    for (int c = 0; c < 24; ++c) {
      const double gxi = 0.5 * (1 - eta) * rA[c] + 0.5 * (1 + eta) * rC[c];
      const double geta = 0.5 * (1 - xi) * rD[c] + 0.5 * (1 + xi) * rB[c];
      Bs[0 * 24 + c] = iJ[0][0] * gxi + iJ[0][1] * geta;
      Bs[1 * 24 + c] = iJ[1][0] * gxi + iJ[1][1] * geta;
    }
    add_btdb(K, Bm, 3, Dm, det);
    add_btdb(K, Bb, 3, Db, det);
    add_btdb(K, Bs, 2, Ds, det);
  }
  for (int a = 0; a < 4; ++a) K[6 * a + 5][6 * a + 5] += 1e-3 * cb;
}

/* ------------------------------------------------------------ set-up */
static int shell_init(shell_t *S, int nx, int ny, const double *X, double E, double nu, double h,
                      double rho, const int *fixed) {
  S->nx = nx; S->ny = ny; S->nn = nx * ny; S->ne = (nx - 1) * (ny - 1); S->n = 6 * S->nn;
  S->kb = 6 * (ny + 1) + 5;
  S->X = X; S->E = E; S->nu = nu; S->h = h; S->rho = rho; S->fixed = fixed;
  S->Kl = (double *)calloc((size_t)S->ne * 576, sizeof(double));
  S->Re0 = (double *)calloc((size_t)S->ne * 9, sizeof(double));
  S->xb0 = (double *)calloc((size_t)S->ne * 12, sizeof(double));
  S->m = (double *)calloc((size_t)S->nn, sizeof(double));
  S->Jr = (double *)calloc((size_t)S->nn, sizeof(double));
  if (!S->Kl || !S->Re0 || !S->xb0 || !S->m || !S->Jr) return -1;
  for (int e = 0; e < S->ne; ++e) {
    int id[4];
    elem_nodes(S, e, id);
    double x[4][3], R[3][3], c[3], xl[4][2];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) x[a][k] = X[3 * id[a] + k];
    quad_frame(x, R, c);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S->Re0[9 * e + 3 * i + j] = R[i][j];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int q = 0; q < 3; ++q) s += R[q][k] * (x[a][q] - c[q]);
        S->xb0[12 * e + 3 * a + k] = s;
      }
    for (int a = 0; a < 4; ++a) {
      xl[a][0] = S->xb0[12 * e + 3 * a];
      xl[a][1] = S->xb0[12 * e + 3 * a + 1];
    }
    local_stiffness(S, xl, (double(*)[24])(S->Kl + 576 * e));
    /* area by the diagonals */
    const double A = 0.5 * fabs((xl[2][0] - xl[0][0]) * (xl[3][1] - xl[1][1]) -
                                (xl[2][1] - xl[0][1]) * (xl[3][0] - xl[1][0]));
    for (int a = 0; a < 4; ++a) {
      S->m[id[a]] += rho * h * A / 4;
      S->Jr[id[a]] += rho * h * h * h / 12 * A / 4;
    }
  }
  return 0;
}

static void shell_free(shell_t *S) {
  free(S->Kl); free(S->Re0); free(S->xb0); free(S->m); free(S->Jr);
}

/* ------------------------------------------------------------ element force */
/* Global force fe[24] of element e at (u, Rn) and (if Ke) the tangent block
 * Ke[24][24] (global DOFs, node order of the element). */
static void elem_force(const shell_t *S, int e, const double *u, const double *Rn, double fe[24],
                       double Ke[24][24]) {
  int id[4];
  elem_nodes(S, e, id);
  double x[4][3], Re[3][3], c[3], xb[4][3], R0e[3][3];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) x[a][k] = S->X[3 * id[a] + k] + u[3 * id[a] + k];
  quad_frame(x, Re, c);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R0e[i][j] = S->Re0[9 * e + 3 * i + j];
  double d[24];
  for (int a = 0; a < 4; ++a) {
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int q = 0; q < 3; ++q) s += Re[q][k] * (x[a][q] - c[q]);
      xb[a][k] = s;
      d[6 * a + k] = s - S->xb0[12 * e + 3 * a + k];
    }
    double Rnode[3][3], T1[3][3], Rd[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Rnode[i][j] = Rn[9 * id[a] + 3 * i + j];
    mat_tmul(Re, Rnode, T1);
    mat_mul(T1, R0e, Rd);
    rot_log(Rd, d + 6 * a + 3);
  }
  const double *Kl = S->Kl + 576 * e;
  double fl[24];
  for (int i = 0; i < 24; ++i) {
    double s = 0;
    for (int j = 0; j < 24; ++j) s += Kl[24 * i + j] * d[j];
    fl[i] = s;
  }
  /* spin of the frame: omega = G dq (local) */
  double G[3][24];
  memset(G, 0, sizeof(G));
  const double a1 = xb[2][0] - xb[0][0], a2 = xb[2][1] - xb[0][1];
  const double b1 = xb[3][0] - xb[1][0], b2 = xb[3][1] - xb[1][1];
  const double Nn = a1 * b2 - a2 * b1;
  G[0][6 * 2 + 2] += -b1 / Nn; G[0][6 * 0 + 2] += b1 / Nn;
  G[0][6 * 3 + 2] += a1 / Nn;  G[0][6 * 1 + 2] += -a1 / Nn;
  G[1][6 * 2 + 2] += -b2 / Nn; G[1][6 * 0 + 2] += b2 / Nn;
  G[1][6 * 3 + 2] += a2 / Nn;  G[1][6 * 1 + 2] += -a2 / Nn;
  const double ap = xb[1][0] + xb[2][0] - xb[0][0] - xb[3][0];
  G[2][6 * 1 + 1] += 1 / ap; G[2][6 * 2 + 1] += 1 / ap;
  G[2][6 * 0 + 1] -= 1 / ap; G[2][6 * 3 + 1] -= 1 / ap;
  /* projector P (24 x 24) */
  double P[24][24];
  memset(P, 0, sizeof(P));
  for (int a = 0; a < 4; ++a) {
    double Sx[3][3];
    skew(xb[a], Sx);
    for (int r = 0; r < 3; ++r) {
      for (int b = 0; b < 4; ++b) P[6 * a + r][6 * b + r] -= 0.25;
      P[6 * a + r][6 * a + r] += 1.0;
      for (int col = 0; col < 24; ++col) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += Sx[r][k] * G[k][col];
        P[6 * a + r][col] += s;
      }
      P[6 * a + 3 + r][6 * a + 3 + r] += 1.0;
      for (int col = 0; col < 24; ++col) P[6 * a + 3 + r][col] -= G[r][col];
    }
  }
  double fp[24];
  for (int j = 0; j < 24; ++j) {
    double s = 0;
    for (int i = 0; i < 24; ++i) s += P[i][j] * fl[i];
    fp[j] = s;
  }
  for (int blk = 0; blk < 8; ++blk)
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int q = 0; q < 3; ++q) s += Re[k][q] * fp[3 * blk + q];
      fe[3 * blk + k] = s;
    }
  if (Ke) {
    double KP[24][24], Kp[24][24];
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j) {
        double s = 0;
        for (int k = 0; k < 24; ++k) s += Kl[24 * i + k] * P[k][j];
        KP[i][j] = s;
      }
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j) {
        double s = 0;
        for (int k = 0; k < 24; ++k) s += P[k][i] * KP[k][j];
        Kp[i][j] = s;
      }
    for (int bi = 0; bi < 8; ++bi)
      for (int bj = 0; bj < 8; ++bj)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) s += Re[i][p] * Kp[3 * bi + p][3 * bj + q] * Re[j][q];
            Ke[3 * bi + i][3 * bj + j] = s;
          }
  }
}

/* Global internal force f[6 nn] and (if Kb) band tangent Kb[n][2 kb + 1]. */
static void shell_internal(const shell_t *S, const double *u, const double *Rn, double *f,
                           double *Kb) {
  const int W = 2 * S->kb + 1;
  memset(f, 0, sizeof(double) * S->n);
  if (Kb) memset(Kb, 0, sizeof(double) * (size_t)S->n * W);
  double fe[24], Ke[24][24];
  for (int e = 0; e < S->ne; ++e) {
    int id[4];
    elem_nodes(S, e, id);
    elem_force(S, e, u, Rn, fe, Kb ? Ke : NULL);
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 6; ++k) {
        f[6 * id[a] + k] += fe[6 * a + k];
        if (!Kb) continue;
        const int gi = 6 * id[a] + k;
        for (int b = 0; b < 4; ++b)
          for (int l = 0; l < 6; ++l) {
            const int gj = 6 * id[b] + l;
            Kb[(size_t)gi * W + (gj - gi + S->kb)] += Ke[6 * a + k][6 * b + l];
          }
      }
  }
}

/* Solve the band system A x = r in place (r <- x); no pivoting. */
static int band_solve(double *A, double *r, int n, int kb) {
  const int W = 2 * kb + 1;
  for (int k = 0; k < n; ++k) {
    const double piv = A[(size_t)k * W + kb];
    if (piv == 0.0) return -1;
    const int iend = k + kb < n - 1 ? k + kb : n - 1;
    for (int i = k + 1; i <= iend; ++i) {
      const double m = A[(size_t)i * W + (k - i + kb)] / piv;
      if (m == 0.0) continue;
      for (int j = k + 1; j <= iend; ++j) A[(size_t)i * W + (j - i + kb)] -= m * A[(size_t)k * W + (j - k + kb)];
      r[i] -= m * r[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = r[k];
    const int jend = k + kb < n - 1 ? k + kb : n - 1;
    for (int j = k + 1; j <= jend; ++j) s -= A[(size_t)k * W + (j - k + kb)] * r[j];
    r[k] = s / A[(size_t)k * W + kb];
  }
  return 0;
}

/* ------------------------------------------------------------ API */
int or_shell_internal(int nx, int ny, const double *X, double E, double nu, double h, double rho,
                      const int *fixed, const double *u, const double *Rn, double *f) {
  shell_t S;
  if (shell_init(&S, nx, ny, X, E, nu, h, rho, fixed)) return -1;
  shell_internal(&S, u, Rn, f, NULL);
  shell_free(&S);
  return 0;
}

/* Lumped mass: m[nn] translational, Jr[nn] rotational. */
int or_shell_mass(int nx, int ny, const double *X, double E, double nu, double h, double rho,
                  double *m, double *Jr) {
  shell_t S;
  if (shell_init(&S, nx, ny, X, E, nu, h, rho, NULL)) return -1;
  memcpy(m, S.m, sizeof(double) * S.nn);
  memcpy(Jr, S.Jr, sizeof(double) * S.nn);
  shell_free(&S);
  return 0;
}

/* One theta-scheme step.  u[nn][3], Rn[nn][9], v[nn][6] (translational then
 * angular velocity) in/out; F0, F1 [nn][6] nodal forces and moments (global).
 * Returns the Newton iterations (negative when max_it was reached). */
int or_shell_step(int nx, int ny, const double *X, double E, double nu, double h, double rho,
                  const int *fixed, double dt, double theta, double lam, double rtol, double atol,
                  int max_it, const double *F0, const double *F1, double *u, double *Rn,
                  double *v) {
  shell_t S;
  if (shell_init(&S, nx, ny, X, E, nu, h, rho, fixed)) return -100000;
  const int n = S.n, nn = S.nn, W = 2 * S.kb + 1;
  double *u0 = malloc(sizeof(double) * 3 * nn), *R0 = malloc(sizeof(double) * 9 * nn);
  double *v0 = malloc(sizeof(double) * n), *dq = calloc(n, sizeof(double));
  double *f0 = malloc(sizeof(double) * n), *f1 = malloc(sizeof(double) * n);
  double *res = malloc(sizeof(double) * n), *Kb = malloc(sizeof(double) * (size_t)n * W);
  double *u1 = malloc(sizeof(double) * 3 * nn), *R1 = malloc(sizeof(double) * 9 * nn);
  double *v1 = malloc(sizeof(double) * n);
  memcpy(u0, u, sizeof(double) * 3 * nn);
  memcpy(R0, Rn, sizeof(double) * 9 * nn);
  memcpy(v0, v, sizeof(double) * n);
  shell_internal(&S, u0, R0, f0, NULL);
  double r0 = -1.0;
  int it, conv = 0;
  for (it = 0; it <= max_it; ++it) {
    for (int a = 0; a < nn; ++a) {
      for (int k = 0; k < 3; ++k) u1[3 * a + k] = u0[3 * a + k] + dq[6 * a + k];
      double E1[3][3], Ra[3][3], Rb[3][3];
      rot_exp(dq + 6 * a + 3, E1);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ra[i][j] = R0[9 * a + 3 * i + j];
      mat_mul(E1, Ra, Rb);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R1[9 * a + 3 * i + j] = Rb[i][j];
    }
    shell_internal(&S, u1, R1, f1, Kb);
    double rn = 0.0;
    for (int i = 0; i < n; ++i) {
      const int a = i / 6;
      const double mi = (i % 6) < 3 ? S.m[a] : S.Jr[a];
      v1[i] = (dq[i] / dt - (1.0 - theta) * v0[i]) / theta;
      double R = mi * (v1[i] - v0[i]) / dt - theta * (F1[i] - f1[i]) - (1.0 - theta) * (F0[i] - f0[i]);
      if (fixed[i]) R = 0.0;
      res[i] = -R;
      rn += R * R;
    }
    rn = sqrt(rn);
    if (r0 < 0) r0 = rn;
    if (rn <= rtol * r0 + atol) {
      conv = 1;
      break;
    }
    if (it == max_it) break;
    for (int i = 0; i < n; ++i) {
      const int a = i / 6;
      const double mi = (i % 6) < 3 ? S.m[a] : S.Jr[a];
      for (int o = 0; o < W; ++o) {
        const int j = i + o - S.kb;
        double val = Kb[(size_t)i * W + o] * theta;
        if (j == i) val += mi / (theta * dt * dt);
        if (j >= 0 && j < n && (fixed[i] || fixed[j])) val = (i == j) ? 1.0 : 0.0;
        Kb[(size_t)i * W + o] = val;
      }
    }
    if (band_solve(Kb, res, n, S.kb)) break;
    for (int i = 0; i < n; ++i) dq[i] += lam * res[i];
  }
  memcpy(u, u1, sizeof(double) * 3 * nn);
  memcpy(Rn, R1, sizeof(double) * 9 * nn);
  for (int i = 0; i < n; ++i) v[i] = fixed[i] ? 0.0 : v1[i];
  free(u0); free(R0); free(v0); free(dq); free(f0); free(f1); free(res); free(Kb);
  free(u1); free(R1); free(v1);
  shell_free(&S);
  return conv ? it : -it - 1;
}

/* Static equilibrium f(u, R) = F by Newton with relaxation lam from the
 * reference state (or the given u, Rn). */
int or_shell_static(int nx, int ny, const double *X, double E, double nu, double h,
                    const int *fixed, const double *F, double lam, double rtol, double atol,
                    int max_it, double *u, double *Rn) {
  shell_t S;
  if (shell_init(&S, nx, ny, X, E, nu, h, 1.0, fixed)) return -100000;
  const int n = S.n, nn = S.nn, W = 2 * S.kb + 1;
  double *f = malloc(sizeof(double) * n), *res = malloc(sizeof(double) * n);
  double *Kb = malloc(sizeof(double) * (size_t)n * W);
  double r0 = -1.0;
  int it, conv = 0;
  for (it = 0; it <= max_it; ++it) {
    shell_internal(&S, u, Rn, f, Kb);
    double rn = 0.0;
    for (int i = 0; i < n; ++i) {
      double R = f[i] - F[i];
      if (fixed[i]) R = 0.0;
      res[i] = -R;
      rn += R * R;
    }
    rn = sqrt(rn);
    if (r0 < 0) r0 = rn;
    if (rn <= rtol * r0 + atol) {
      conv = 1;
      break;
    }
    if (it == max_it) break;
    for (int i = 0; i < n; ++i)
      for (int o = 0; o < W; ++o) {
        const int j = i + o - S.kb;
        if (j >= 0 && j < n && (fixed[i] || fixed[j])) Kb[(size_t)i * W + o] = (i == j) ? 1.0 : 0.0;
      }
    if (band_solve(Kb, res, n, S.kb)) break;
    for (int a = 0; a < nn; ++a) {
      for (int k = 0; k < 3; ++k) u[3 * a + k] += lam * res[6 * a + k];
      double phi[3] = {lam * res[6 * a + 3], lam * res[6 * a + 4], lam * res[6 * a + 5]};
      double E1[3][3], Ra[3][3], Rb[3][3];
      rot_exp(phi, E1);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ra[i][j] = Rn[9 * a + 3 * i + j];
      mat_mul(E1, Ra, Rb);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rn[9 * a + 3 * i + j] = Rb[i][j];
    }
  }
  free(f); free(res); free(Kb);
  shell_free(&S);
  return conv ? it : -it - 1;
}
