// fem_shell.cu -- GPU co-rotational flat shell for the 3-D plate (FP64).
//
// Structural model (replacing the paper's Q2 continuum elements of section
// "Structural modeling" for the plate cases): 4-node quadrilaterals on a
// structured nx x ny node grid (node i*ny + j, element (i, j) with nodes
// (i,j), (i+1,j), (i+1,j+1), (i,j+1)), six DOFs per node (translations and a
// rotation, carried as a rotation matrix).  Local element: linear and
// constant -- plane-stress membrane and Mindlin plate bending at 2x2 Gauss
// points, MITC4 transverse shear (covariant strains tied at the edge
// midpoints, shear factor 5/6), drilling stiffness 1e-3 D on the rotation
// about the element normal.  Co-rotation: element frame from the diagonals
// (normal) and the mean of the two x-running sides (e1); local deformations
// d = (R_e^T (x - c) - x_ref, log(R_e^T R_node R_e0)); internal force
// T^T P^T K_l d with P the projector that removes the frame's rigid motion
// (written as I - U V, rank 6); tangent T^T P^T K_l P T.  Lumped mass.
//
// Time step: theta-scheme in the two-field form (Eq. timeInt), Newton with
// the paper's constant relaxation lambda on the step increments (rotation
// vectors for the rotations); every linearised system is solved by
// Jacobi-preconditioned conjugate gradients on the element tangents (no
// assembled matrix).  One cooperative launch runs the whole step: one CTA per
// element (grid-stride), grid-wide barriers between the phases, reductions
// by FP64 atomics into three rotating slots.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/kbc_lbm.h"
#include "lbm_internal.h"

namespace cg = cooperative_groups;

namespace kbc {

constexpr int kShellThreads = 128;
constexpr int kShellMaxNodes = 4096;

struct ShellParams {
  int nx, ny, nn, ne, n;
  double E, nu, h, rho;
  double theta, lambda, rtol, atol, dt;
  int max_it, max_cg;
  double cg_rtol;
};

struct ShellDev {
  const double *X;           // [nn][3]
  const int32_t *fixed;      // [6 nn]
  double *Kl;                // [ne][576] local stiffness
  double *Re0;               // [ne][9] reference frames (row-major, columns e1 e2 e3)
  double *xb0;               // [ne][12] reference local node positions
  double *mt, *mr;           // [nn] lumped translational / rotational mass
  double *u, *R, *v, *F0;    // state: [nn][3], [nn][9], [6 nn], previous loads [6 nn]
  double *u0, *R0, *v0;      // state at the start of the step
  double *u1, *R1;           // current Newton iterate
  double *dq;                // [6 nn] step increments (translations, rotation vectors)
  double *f0, *f, *kd;       // internal force at start / current, diagonal of K
  double *eg;                // [ne][kEG] frame data of the current iterate
  double *rhs, *x, *r, *z, *p, *Ap, *Ap2;
  double *red;               // [3][2] reduction slots
  const double *F1;          // [6 nn] loads of the step
  int *iters;                // [2]: Newton iterations of the last step, CG iterations
  double *Fm2;               // [6 nn] loads two steps back (surrogate input)
  const double *dqg;         // [6 nn] Newton start (surrogate guess), nullptr: zero
  double accept_tol;         // > 0: accept the guess when |R| <= accept_tol |F_ext|
  int *stats;                // [4]: guesses accepted, rejected, Newton solves, steps
};

__device__ __forceinline__ void elem_ids(const ShellParams &P, int e, int id[4]) {
  const int i = e / (P.ny - 1), j = e % (P.ny - 1);
  id[0] = i * P.ny + j;
  id[1] = (i + 1) * P.ny + j;
  id[2] = (i + 1) * P.ny + j + 1;
  id[3] = i * P.ny + j + 1;
}

// Frame (row-major, columns e1 e2 e3) and centre of four points xs[4][3].
__device__ void quad_frame_dev(const double *xs, double *Re, double *c) {
  double d13[3], d24[3], a[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.25 * (xs[k] + xs[3 + k] + xs[6 + k] + xs[9 + k]);
    d13[k] = xs[6 + k] - xs[k];
    d24[k] = xs[9 + k] - xs[3 + k];
    a[k] = xs[3 + k] + xs[6 + k] - xs[k] - xs[9 + k];
  }
  double e3[3] = {d13[1] * d24[2] - d13[2] * d24[1], d13[2] * d24[0] - d13[0] * d24[2],
                  d13[0] * d24[1] - d13[1] * d24[0]};
  const double in3 = rsqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
  for (int k = 0; k < 3; ++k) e3[k] *= in3;
  const double ad = a[0] * e3[0] + a[1] * e3[1] + a[2] * e3[2];
  double e1[3] = {a[0] - ad * e3[0], a[1] - ad * e3[1], a[2] - ad * e3[2]};
  const double in1 = rsqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int k = 0; k < 3; ++k) e1[k] *= in1;
  const double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                        e3[0] * e1[1] - e3[1] * e1[0]};
  for (int k = 0; k < 3; ++k) {
    Re[3 * k] = e1[k];
    Re[3 * k + 1] = e2[k];
    Re[3 * k + 2] = e3[k];
  }
}

// exp of the skew matrix of phi (Rodrigues), row-major.
__device__ void rodrigues(const double *phi, double *Rm) {
  const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  const double t = sqrt(t2);
  double s1, s2;
  if (t < 1e-6) {
    s1 = 1.0 - t2 / 6.0;
    s2 = 0.5 - t2 / 24.0;
  } else {
    // sin and cos from one call; 1 - cos t = sin^2 t / (1 + cos t) (t < pi)
    double st, ct;
    sincos(t, &st, &ct);
    s1 = st / t;
    s2 = s1 * s1 / (1.0 + ct);
  }
  const double x = phi[0], y = phi[1], z = phi[2];
  // I + s1 S + s2 S^2 with S^2 = phi phi^T - t2 I
  Rm[0] = 1.0 + s2 * (x * x - t2); Rm[1] = -s1 * z + s2 * x * y;      Rm[2] = s1 * y + s2 * x * z;
  Rm[3] = s1 * z + s2 * x * y;      Rm[4] = 1.0 + s2 * (y * y - t2); Rm[5] = -s1 * x + s2 * y * z;
  Rm[6] = -s1 * y + s2 * x * z;     Rm[7] = s1 * x + s2 * y * z;      Rm[8] = 1.0 + s2 * (z * z - t2);
}

// Rotation vector of Rm (angle below pi).
// w = (R32 - R23, R13 - R31, R21 - R12) = 2 sin(t) n and cos(t) = (tr R - 1) / 2,
// so t = atan2(|w| / 2, cos t) and phi = t w / |w| (one atan2 instead of an
// acos and a sin; accurate at small angles, where acos is not).
__device__ void rotvec(const double *Rm, double *phi) {
  const double ct = 0.5 * (Rm[0] + Rm[4] + Rm[8] - 1.0);
  const double w[3] = {Rm[7] - Rm[5], Rm[2] - Rm[6], Rm[3] - Rm[1]};
  const double sw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  const double t = atan2(0.5 * sw, ct);
  const double g = (sw < 1e-12) ? 0.5 + t * t / 12.0 : t / sw;
  phi[0] = g * w[0];
  phi[1] = g * w[1];
  phi[2] = g * w[2];
}

// ---------------------------------------------------------------- set-up
// Reference frame, local positions, local stiffness and lumped masses of
// element blockIdx.x (one CTA per element).
__global__ void __launch_bounds__(kShellThreads) k_shell_setup(ShellParams P, ShellDev D) {
  const int e = blockIdx.x, t = threadIdx.x;
  __shared__ double xs[12], Re[9], c[3], xl[4][2];
  __shared__ double Bm[4][3][24], Bb[4][3][24], Bs[4][2][24], dj[4];
  __shared__ double tie[4][24];  // covariant shear rows at A(0,-1), C(0,1), D(-1,0), B(1,0)
  int id[4];
  elem_ids(P, e, id);
  if (t < 12) xs[t] = D.X[3 * id[t / 3] + t % 3];
  __syncthreads();
  if (t == 0) quad_frame_dev(xs, Re, c);
  __syncthreads();
  if (t < 12) {
    const int a = t / 3, k = t % 3;
    double s = 0.0;
    for (int q = 0; q < 3; ++q) s += Re[3 * q + k] * (xs[3 * a + q] - c[q]);
    D.xb0[12 * e + t] = s;
    if (k < 2) xl[a][k] = s;
  }
  if (t < 9) D.Re0[9 * e + t] = Re[t];
  __syncthreads();
  const double sgn_xi[4] = {-1, 1, 1, -1}, sgn_eta[4] = {-1, -1, 1, 1};
  // tying rows (threads 0..3) and Gauss-point rows (threads 4..7)
  if (t < 8) {
    const bool tying = t < 4;
    const double gp = 0.57735026918962576;
    double xi, eta;
    if (tying) {
      const double txi[4] = {0, 0, -1, 1}, teta[4] = {-1, 1, 0, 0};
      xi = txi[t];
      eta = teta[t];
    } else {
      xi = gp * sgn_xi[t - 4];
      eta = gp * sgn_eta[t - 4];
    }
    double N[4], Nx[4], Ne[4];
    for (int a = 0; a < 4; ++a) {
      N[a] = 0.25 * (1 + xi * sgn_xi[a]) * (1 + eta * sgn_eta[a]);
      Nx[a] = 0.25 * sgn_xi[a] * (1 + eta * sgn_eta[a]);
      Ne[a] = 0.25 * sgn_eta[a] * (1 + xi * sgn_xi[a]);
    }
    double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
    for (int a = 0; a < 4; ++a) {
      j00 += Nx[a] * xl[a][0]; j01 += Nx[a] * xl[a][1];
      j10 += Ne[a] * xl[a][0]; j11 += Ne[a] * xl[a][1];
    }
    if (tying) {
      // covariant shear along xi (A, C) or eta (D, B): w_,s + beta_x x_,s + beta_y y_,s,
      // beta_x = theta_y, beta_y = -theta_x
      const bool along_xi = t < 2;
      const double xd = along_xi ? j00 : j10, yd = along_xi ? j01 : j11;
      for (int a = 0; a < 4; ++a) {
        tie[t][6 * a + 0] = 0; tie[t][6 * a + 1] = 0; tie[t][6 * a + 5] = 0;
        tie[t][6 * a + 2] = along_xi ? Nx[a] : Ne[a];
        tie[t][6 * a + 3] = -N[a] * yd;
        tie[t][6 * a + 4] = N[a] * xd;
      }
    } else {
      const int g = t - 4;
      const double det = j00 * j11 - j01 * j10;
      dj[g] = det;
      const double i00 = j11 / det, i01 = -j01 / det, i10 = -j10 / det, i11 = j00 / det;
      for (int col = 0; col < 24; ++col) {
        Bm[g][0][col] = Bm[g][1][col] = Bm[g][2][col] = 0.0;
        Bb[g][0][col] = Bb[g][1][col] = Bb[g][2][col] = 0.0;
      }
      for (int a = 0; a < 4; ++a) {
        const double dx = i00 * Nx[a] + i01 * Ne[a], dy = i10 * Nx[a] + i11 * Ne[a];
        Bm[g][0][6 * a] = dx;
        Bm[g][1][6 * a + 1] = dy;
        Bm[g][2][6 * a] = dy;
        Bm[g][2][6 * a + 1] = dx;
        Bb[g][0][6 * a + 4] = dx;
        Bb[g][1][6 * a + 3] = -dy;
        Bb[g][2][6 * a + 4] = dy;
        Bb[g][2][6 * a + 3] = -dx;
      }
    }
  }
  __syncthreads();
  // Cartesian shear rows at the Gauss points from the tied covariant strains
  for (int w = t; w < 4 * 24; w += blockDim.x) {
    const int g = w / 24, col = w % 24;
    const double gp = 0.57735026918962576;
    const double xi = gp * sgn_xi[g], eta = gp * sgn_eta[g];
    const double sxi = 0.5 * (1 - eta) * tie[0][col] + 0.5 * (1 + eta) * tie[1][col];
    const double seta = 0.5 * (1 - xi) * tie[2][col] + 0.5 * (1 + xi) * tie[3][col];
    // inverse Jacobian at the point
    double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
    for (int a = 0; a < 4; ++a) {
      const double nx = 0.25 * sgn_xi[a] * (1 + eta * sgn_eta[a]);
      const double ne = 0.25 * sgn_eta[a] * (1 + xi * sgn_xi[a]);
      j00 += nx * xl[a][0]; j01 += nx * xl[a][1];
      j10 += ne * xl[a][0]; j11 += ne * xl[a][1];
    }
    const double det = j00 * j11 - j01 * j10;
    Bs[g][0][col] = (j11 * sxi - j01 * seta) / det;
    Bs[g][1][col] = (-j10 * sxi + j00 * seta) / det;
  }
  __syncthreads();
  const double cm = P.E * P.h / (1 - P.nu * P.nu);
  const double cb = P.E * P.h * P.h * P.h / (12 * (1 - P.nu * P.nu));
  const double ks = 5.0 / 6.0 * P.E / (2 * (1 + P.nu)) * P.h;
  for (int w = t; w < 576; w += blockDim.x) {
    const int i = w / 24, j = w % 24;
    double s = 0.0;
    for (int g = 0; g < 4; ++g) {
      const double m0 = Bm[g][0][i], m1 = Bm[g][1][i], m2 = Bm[g][2][i];
      const double n0 = Bm[g][0][j], n1 = Bm[g][1][j], n2 = Bm[g][2][j];
      const double mem = cm * (m0 * (n0 + P.nu * n1) + m1 * (P.nu * n0 + n1) + 0.5 * (1 - P.nu) * m2 * n2);
      const double b0 = Bb[g][0][i], b1 = Bb[g][1][i], b2 = Bb[g][2][i];
      const double c0 = Bb[g][0][j], c1 = Bb[g][1][j], c2 = Bb[g][2][j];
      const double ben = cb * (b0 * (c0 + P.nu * c1) + b1 * (P.nu * c0 + c1) + 0.5 * (1 - P.nu) * b2 * c2);
      const double she = ks * (Bs[g][0][i] * Bs[g][0][j] + Bs[g][1][i] * Bs[g][1][j]);
      s += (mem + ben + she) * dj[g];
    }
    if (i == j && i % 6 == 5) s += 1e-3 * cb;
    D.Kl[576 * (long long)e + w] = s;
  }
  if (t == 0) {
    const double A = 0.5 * fabs((xl[2][0] - xl[0][0]) * (xl[3][1] - xl[1][1]) -
                                (xl[2][1] - xl[0][1]) * (xl[3][0] - xl[1][0]));
    for (int a = 0; a < 4; ++a) {
      atomicAdd(D.mt + id[a], P.rho * P.h * A * 0.25);
      atomicAdd(D.mr + id[a], P.rho * P.h * P.h * P.h / 12.0 * A * 0.25);
    }
  }
}

// ---------------------------------------------------------------- element work
// One warp per element: lanes over the 24 element DOFs, per-warp scratch in
// shared memory, warp-synchronous.  The tangent is never formed: its product
// with a vector is T^T P^T K_l P T p, P = I - U V (rank 6), and the frame
// data it needs (R_e, local positions, frame-spin coefficients) is kept per
// element from the force evaluation of the current iterate.
constexpr int kEG = 28;  // per-element geometry: R_e (9), xb (12), spin coefficients (6), pad

struct ShellWarp {
  double xs[12], Rs[36], Re[9], c[3], xb[12], d[24], fl[24], w6[6], gc[6];
  double U[24][6], V[6][24];
  int id[4];
};

// U and V of the projector from the local positions xb and the spin
// coefficients gc = (a1, a2, b1, b2, N, ap).
__device__ __forceinline__ void warp_projector(ShellWarp &W, int lane) {
  for (int w = lane; w < 144; w += 32) {
    const int i = w / 6, k = w % 6, a = i / 6, s = i % 6;
    double val = 0.0;
    if (s < 3) {
      if (k < 3) {
        val = (k == s) ? 1.0 : 0.0;
      } else {
        // -(xb_a x e_m)_s, m = k - 3
        const double *xa = W.xb + 3 * a;
        const int m = k - 3;
        const double em[3] = {m == 0 ? 1.0 : 0.0, m == 1 ? 1.0 : 0.0, m == 2 ? 1.0 : 0.0};
        const double cr[3] = {xa[1] * em[2] - xa[2] * em[1], xa[2] * em[0] - xa[0] * em[2],
                              xa[0] * em[1] - xa[1] * em[0]};
        val = -cr[s];
      }
    } else {
      val = (k >= 3 && k - 3 == s - 3) ? 1.0 : 0.0;
    }
    W.U[i][k] = val;
  }
  // one reciprocal of N and of ap per warp instead of a division per entry
  const double iN = 1.0 / W.gc[4], iap = 1.0 / W.gc[5];
  for (int w = lane; w < 144; w += 32) {
    const int k = w / 24, j = w % 24, b = j / 6, s = j % 6;
    const double a1 = W.gc[0], a2 = W.gc[1], b1 = W.gc[2], b2 = W.gc[3];
    double val = 0.0;
    if (k < 3) {
      val = (s == k) ? 0.25 : 0.0;
    } else {
      // frame spin: x and y tilts from the diagonals, z from the sides
      if (k == 3 && s == 2) val = (b == 2 ? -b1 : b == 0 ? b1 : b == 3 ? a1 : -a1) * iN;
      if (k == 4 && s == 2) val = (b == 2 ? -b2 : b == 0 ? b2 : b == 3 ? a2 : -a2) * iN;
      if (k == 5 && s == 1) val = (b == 1 || b == 2 ? iap : -iap);
    }
    W.V[k][j] = val;
  }
  __syncwarp();
}

// Internal force of element e at (u, R) scattered into fout; with eg, the
// element's frame data is stored, with kd the diagonal of T^T K_l T added.
// The state is (u + dq_t, exp(dq_r) R) per node when dq is given, else (u, R).
__device__ void warp_element_force(const ShellParams &P, const ShellDev &D, int e, const double *u,
                                   const double *R, const double *dq, double *fout, double *eg,
                                   double *kd, ShellWarp &W, int lane) {
  if (lane < 4) {
    int id[4];
    elem_ids(P, e, id);
    W.id[lane] = id[lane];
  }
  __syncwarp();
  if (lane < 12) {
    const int a = W.id[lane / 3], k = lane % 3;
    W.xs[lane] = D.X[3 * a + k] + u[3 * a + k] + (dq ? dq[6 * a + k] : 0.0);
  }
  if (dq) {
    if (lane < 4) {
      const int a = W.id[lane];
      double Ex[9];
      rodrigues(dq + 6 * a + 3, Ex);
      const double *Ra = R + 9 * a;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          W.Rs[9 * lane + 3 * i + j] = Ex[3 * i] * Ra[j] + Ex[3 * i + 1] * Ra[3 + j] + Ex[3 * i + 2] * Ra[6 + j];
    }
  } else {
    for (int w = lane; w < 36; w += 32) W.Rs[w] = R[9 * W.id[w / 9] + w % 9];
  }
  __syncwarp();
  if (lane == 0) quad_frame_dev(W.xs, W.Re, W.c);
  __syncwarp();
  if (lane < 12) {
    const int a = lane / 3, k = lane % 3;
    double s = 0.0;
    for (int q = 0; q < 3; ++q) s += W.Re[3 * q + k] * (W.xs[3 * a + q] - W.c[q]);
    W.xb[lane] = s;
    W.d[6 * a + k] = s - D.xb0[12 * e + lane];
  } else if (lane < 16) {
    // deformational rotation R_e^T R_a R_e0 of node a
    const int a = lane - 12;
    const double *R0 = D.Re0 + 9 * e;
    double T1[9], Rd[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) s += W.Re[3 * q + i] * W.Rs[9 * a + 3 * q + j];
        T1[3 * i + j] = s;
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) s += T1[3 * i + q] * R0[3 * q + j];
        Rd[3 * i + j] = s;
      }
    rotvec(Rd, W.d + 6 * a + 3);
  }
  __syncwarp();
  if (lane == 0) {
    W.gc[0] = W.xb[6] - W.xb[0];
    W.gc[1] = W.xb[7] - W.xb[1];
    W.gc[2] = W.xb[9] - W.xb[3];
    W.gc[3] = W.xb[10] - W.xb[4];
    W.gc[4] = W.gc[0] * W.gc[3] - W.gc[1] * W.gc[2];
    W.gc[5] = W.xb[3] + W.xb[6] - W.xb[0] - W.xb[9];
  }
  __syncwarp();
  warp_projector(W, lane);
  const double *Kl = D.Kl + 576 * (long long)e;
  if (lane < 24) {
    double s = 0.0;
    for (int j = 0; j < 24; ++j) s += Kl[24 * lane + j] * W.d[j];
    W.fl[lane] = s;
  }
  __syncwarp();
  if (lane < 6) {
    double s = 0.0;
    for (int i = 0; i < 24; ++i) s += W.U[i][lane] * W.fl[i];
    W.w6[lane] = s;
  }
  __syncwarp();
  double fp = 0.0;
  if (lane < 24) {
    fp = W.fl[lane];
    for (int k = 0; k < 6; ++k) fp -= W.V[k][lane] * W.w6[k];
  }
  __syncwarp();
  if (lane < 24) W.d[lane] = fp;  // reuse as the projected local force
  __syncwarp();
  if (lane < 24) {
    const int blk = lane / 3, k = lane % 3, a = blk / 2, kind = blk % 2;
    double s = 0.0;
    for (int q = 0; q < 3; ++q) s += W.Re[3 * k + q] * W.d[3 * blk + q];
    atomicAdd(fout + 6 * W.id[a] + 3 * kind + k, s);
    if (kd) {
      // (T^T K_l T)_{ii} for the global DOF (block blk, axis k)
      double t = 0.0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
          t += W.Re[3 * k + p] * Kl[24 * (3 * blk + p) + 3 * blk + q] * W.Re[3 * k + q];
      atomicAdd(kd + 6 * W.id[a] + 3 * kind + k, t);
    }
  }
  if (eg && lane < kEG) {
    double v = 0.0;
    if (lane < 9) v = W.Re[lane];
    else if (lane < 21) v = W.xb[lane - 9];
    else if (lane < 27) v = W.gc[lane - 21];
    eg[kEG * (long long)e + lane] = v;
  }
  __syncwarp();
}

// y += theta T^T P^T K_l P T p for element e.  With own, the warp's scratch
// still holds e's frame and projector from the force evaluation; otherwise
// they are rebuilt from the frame data in eg.
__device__ void warp_element_matvec(const ShellParams &P, const ShellDev &D, int e, const double *eg,
                                    const double *z, const double *p, double beta, double *y,
                                    ShellWarp &W, int lane, bool own) {
  if (!own) {
    if (lane < 4) {
      int id[4];
      elem_ids(P, e, id);
      W.id[lane] = id[lane];
    }
    if (lane < kEG) {
      const double v = eg[kEG * (long long)e + lane];
      if (lane < 9) W.Re[lane] = v;
      else if (lane < 21) W.xb[lane - 9] = v;
      else if (lane < 27) W.gc[lane - 21] = v;
    }
    __syncwarp();
    warp_projector(W, lane);
  }
  if (lane < 24) {
    // q = T p: block of three rotated into the element frame
    const int blk = lane / 3, k = lane % 3, a = blk / 2, kind = blk % 2;
    const long long g0 = 6 * W.id[a] + 3 * kind;
    const double q0 = z[g0] + beta * p[g0], q1 = z[g0 + 1] + beta * p[g0 + 1],
                 q2 = z[g0 + 2] + beta * p[g0 + 2];
    W.fl[lane] = W.Re[k] * q0 + W.Re[3 + k] * q1 + W.Re[6 + k] * q2;
  }
  __syncwarp();
  if (lane < 6) {
    double s = 0.0;
    for (int j = 0; j < 24; ++j) s += W.V[lane][j] * W.fl[j];
    W.w6[lane] = s;
  }
  __syncwarp();
  if (lane < 24) {
    double s = W.fl[lane];
    for (int k = 0; k < 6; ++k) s -= W.U[lane][k] * W.w6[k];
    W.d[lane] = s;  // P T p
  }
  __syncwarp();
  const double *Kl = D.Kl + 576 * (long long)e;
  double kz = 0.0;
  if (lane < 24)
    for (int j = 0; j < 24; ++j) kz += Kl[24 * lane + j] * W.d[j];
  __syncwarp();
  if (lane < 24) W.fl[lane] = kz;
  __syncwarp();
  if (lane < 6) {
    double s = 0.0;
    for (int i = 0; i < 24; ++i) s += W.U[i][lane] * W.fl[i];
    W.w6[lane] = s;
  }
  __syncwarp();
  if (lane < 24) {
    double s = W.fl[lane];
    for (int k = 0; k < 6; ++k) s -= W.V[k][lane] * W.w6[k];
    W.d[lane] = s;  // P^T K_l P T p
  }
  __syncwarp();
  if (lane < 24) {
    const int blk = lane / 3, k = lane % 3, a = blk / 2, kind = blk % 2;
    double s = 0.0;
    for (int q = 0; q < 3; ++q) s += W.Re[3 * k + q] * W.d[3 * blk + q];
    atomicAdd(y + 6 * W.id[a] + 3 * kind + k, P.theta * s);
  }
  __syncwarp();
}

// Barrier over all CTAs of the step: the cooperative grid, or the single
// thread-block cluster (with a device-scope fence for the global updates).
template <bool CLUSTER>
__device__ __forceinline__ void step_sync() {
  if constexpr (CLUSTER) {
    __threadfence();
    cg::this_cluster().sync();
  } else {
    cg::this_grid().sync();
  }
}

// Sums of two values over all CTAs: block reduction, one atomic per block
// into slot s, barrier, read; the slot two ahead is cleared for later use.
template <bool CLUSTER>
__device__ __forceinline__ void step_sum2(double *red, int &slot, double a, double b, double &ra,
                                          double &rb) {
  __shared__ double part[2][kShellThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    part[0][w] = a;
    part[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sa += part[0][k];
      sb += part[1][k];
    }
    atomicAdd(red + 2 * slot, sa);
    atomicAdd(red + 2 * slot + 1, sb);
  }
  step_sync<CLUSTER>();
  ra = *(volatile double *)(red + 2 * slot);
  rb = *(volatile double *)(red + 2 * slot + 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int clr = (slot + 2) % 3;
    red[2 * clr] = 0.0;
    red[2 * clr + 1] = 0.0;
  }
  slot = (slot + 1) % 3;
  __syncthreads();
}

// Barriers per Newton iteration: element forces (1), residual with the CG
// start (1), three per CG iteration (element products, two reductions; the
// search direction z + beta p is formed where it is used), increment
// update (1).
template <bool CLUSTER>
__global__ void __launch_bounds__(kShellThreads) k_shell_step(ShellParams P, ShellDev D) {
  __shared__ ShellWarp Wsh[kShellThreads / 32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  ShellWarp &W = Wsh[wl];
  const int wg = blockIdx.x * (kShellThreads / 32) + wl, nwg = gridDim.x * (kShellThreads / 32);
  const bool own = nwg >= P.ne;  // one element per warp for the whole step
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const int n = P.n, nn = P.nn;
  int slot = 0;
  double ra, rb;
  for (long long i = gt; i < n; i += gs) {
    D.v0[i] = D.v[i];
    D.dq[i] = D.dqg ? D.dqg[i] : 0.0;
    D.f0[i] = 0.0;
    D.f[i] = 0.0;
    D.kd[i] = 0.0;
  }
  for (long long i = gt; i < 3 * nn; i += gs) D.u0[i] = D.u[i];
  for (long long i = gt; i < 9 * nn; i += gs) D.R0[i] = D.R[i];
  if (gt < 6) D.red[gt] = 0.0;
  step_sync<CLUSTER>();
  for (int e = wg; e < P.ne; e += nwg)
    warp_element_force(P, D, e, D.u0, D.R0, nullptr, D.f0, nullptr, nullptr, W, lane);
  const double ith = 1.0 / P.theta, idt = 1.0 / P.dt, cM = 1.0 / (P.theta * P.dt * P.dt);
  double r0 = -1.0;
  int it = 0, conv = 0, cg_total = 0;
  for (it = 0;; ++it) {
    // forces and frames of the iterate (u0 + dq, exp(dq_r) R0); f and kd
    // were zeroed before the last barrier
    step_sync<CLUSTER>();
    for (int e = wg; e < P.ne; e += nwg)
      warp_element_force(P, D, e, D.u0, D.R0, D.dq, D.f, D.eg, D.kd, W, lane);
    step_sync<CLUSTER>();
    // residual, and the start of the conjugate gradients on J x = -R
    double part = 0.0, rz0 = 0.0;
    for (long long i = gt; i < n; i += gs) {
      const long long a = i / 6;
      const double m = (i % 6) < 3 ? D.mt[a] : D.mr[a];
      const double v1 = (D.dq[i] * idt - (1.0 - P.theta) * D.v0[i]) * ith;
      double Rv = m * (v1 - D.v0[i]) * idt - P.theta * (D.F1[i] - D.f[i]) -
                  (1.0 - P.theta) * (D.F0[i] - D.f0[i]);
      if (D.fixed[i]) Rv = 0.0;
      const double dJ = D.fixed[i] ? 1.0 : m * cM + P.theta * D.kd[i];
      D.rhs[i] = -Rv;
      D.x[i] = 0.0;
      D.r[i] = -Rv;
      D.z[i] = -Rv / dJ;
      D.p[i] = 0.0;
      D.Ap[i] = 0.0;
      part += Rv * Rv;
      rz0 += Rv * Rv / dJ;
    }
    step_sum2<CLUSTER>(D.red, slot, part, rz0, ra, rb);
    const double rn = sqrt(ra);
    if (it == 0 && D.dqg) {
      // started from a guess: the stopping test stays relative to the
      // residual at the step's start (dq = 0), and the guess is accepted
      // outright when its residual is small against the loads
      double p0 = 0.0, pf = 0.0;
      for (long long i = gt; i < n; i += gs) {
        if (D.fixed[i]) continue;
        const long long a = i / 6;
        const double m = (i % 6) < 3 ? D.mt[a] : D.mr[a];
        const double v1 = -(1.0 - P.theta) * D.v0[i] * ith;
        const double R0 = m * (v1 - D.v0[i]) * idt - P.theta * (D.F1[i] - D.f0[i]) -
                          (1.0 - P.theta) * (D.F0[i] - D.f0[i]);
        const double fe = P.theta * D.F1[i] + (1.0 - P.theta) * D.F0[i];
        p0 += R0 * R0;
        pf += fe * fe;
      }
      double r0sq, fe2;
      step_sum2<CLUSTER>(D.red, slot, p0, pf, r0sq, fe2);
      r0 = sqrt(r0sq);
      if (D.accept_tol > 0.0) {
        const bool accept = rn <= D.accept_tol * sqrt(fe2);
        if (gt == 0 && D.stats) atomicAdd(&D.stats[accept ? 0 : 1], 1);
        if (accept) {
          conv = 1;
          break;
        }
      }
    }
    if (r0 < 0.0) r0 = rn;
    if (rn <= P.rtol * r0 + P.atol) {
      conv = 1;
      break;
    }
    if (it >= P.max_it) break;
    double rz = rb, beta = 0.0;
    const double stop2 = P.cg_rtol * P.cg_rtol * ra;
    double *Ap[2] = {D.Ap, D.Ap2};
    for (int k = 0; k < P.max_cg && ra > 0.0; ++k) {
      double *Ac = Ap[k & 1], *An = Ap[(k + 1) & 1];
      // element products with the direction z + beta p
      for (int e = wg; e < P.ne; e += nwg)
        warp_element_matvec(P, D, e, D.eg, D.z, D.p, beta, Ac, W, lane, own);
      step_sync<CLUSTER>();
      double pap = 0.0;
      for (long long i = gt; i < n; i += gs) {
        const long long a = i / 6;
        const double m = (i % 6) < 3 ? D.mt[a] : D.mr[a];
        const double pn = D.z[i] + beta * D.p[i];
        const double y = D.fixed[i] ? pn : Ac[i] + m * cM * pn;
        D.p[i] = pn;
        Ac[i] = y;
        An[i] = 0.0;
        pap += pn * y;
      }
      double pAp;
      step_sum2<CLUSTER>(D.red, slot, pap, 0.0, pAp, rb);
      const double alpha = rz / pAp;
      double rzp = 0.0, rrp = 0.0;
      for (long long i = gt; i < n; i += gs) {
        const long long a = i / 6;
        const double m = (i % 6) < 3 ? D.mt[a] : D.mr[a];
        const double dJ = D.fixed[i] ? 1.0 : m * cM + P.theta * D.kd[i];
        D.x[i] += alpha * D.p[i];
        const double ri = D.r[i] - alpha * Ac[i];
        D.r[i] = ri;
        D.z[i] = ri / dJ;
        rzp += ri * ri / dJ;
        rrp += ri * ri;
      }
      double rzn, rr;
      step_sum2<CLUSTER>(D.red, slot, rzp, rrp, rzn, rr);
      ++cg_total;
      if (rr <= stop2) break;
      beta = rzn / rz;
      rz = rzn;
    }
    for (long long i = gt; i < n; i += gs) {
      D.dq[i] += P.lambda * D.x[i];
      D.f[i] = 0.0;
      D.kd[i] = 0.0;
    }
  }
  // final state from the increments
  for (long long i = gt; i < n; i += gs) {
    const double v1 = (D.dq[i] * idt - (1.0 - P.theta) * D.v0[i]) * ith;
    D.v[i] = D.fixed[i] ? 0.0 : v1;
    D.Fm2[i] = D.F0[i];
    D.F0[i] = D.F1[i];
  }
  for (long long a = gt; a < nn; a += gs) {
    for (int k = 0; k < 3; ++k) D.u[3 * a + k] = D.u0[3 * a + k] + D.dq[6 * a + k];
    double Ex[9];
    rodrigues(D.dq + 6 * a + 3, Ex);
    const double *Ra = D.R0 + 9 * a;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        D.R[9 * a + 3 * i + j] = Ex[3 * i] * Ra[j] + Ex[3 * i + 1] * Ra[3 + j] + Ex[3 * i + 2] * Ra[6 + j];
  }
  if (gt == 0) {
    D.iters[0] = conv ? it : -it - 1;
    D.iters[1] = cg_total;
    if (D.stats) {
      atomicAdd(&D.stats[2], it);  // Newton solves of this step
      atomicAdd(&D.stats[3], 1);
    }
  }
}

// Internal force of the current state (one warp per element).
__global__ void __launch_bounds__(kShellThreads) k_shell_force_now(ShellParams P, ShellDev D,
                                                                   double *fout) {
  __shared__ ShellWarp Wsh[kShellThreads / 32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int wg = blockIdx.x * (kShellThreads / 32) + wl, nwg = gridDim.x * (kShellThreads / 32);
  for (int e = wg; e < P.ne; e += nwg)
    warp_element_force(P, D, e, D.u, D.R, nullptr, fout, nullptr, nullptr, Wsh[wl], lane);
}

// Surrogate input of the coming step (normalised, FP32): out-of-balance loads
// F1 - f, F0 - f, Fm2 - f, then the state (translations, rotation vectors)
// and the velocities, each block over the free DOFs in freemap order.
__global__ void k_shell_surr_input(ShellParams P, ShellDev D, const double *fcur,
                                   const int *freemap, int nf, const float *xm, const float *xs,
                                   float *xin) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 5 * nf) return;
  const int blk = j / nf, i = freemap[j % nf], a = i / 6, c = i % 6;
  double val;
  if (blk == 0) val = D.F1[i] - fcur[i];
  else if (blk == 1) val = D.F0[i] - fcur[i];
  else if (blk == 2) val = D.Fm2[i] - fcur[i];
  else if (blk == 3) {
    if (c < 3) {
      val = D.u[3 * a + c];
    } else {
      double phi[3];
      rotvec(D.R + 9 * a, phi);
      val = phi[c - 3];
    }
  } else {
    val = D.v[i];
  }
  xin[j] = (float)((val - (double)xm[j]) / (double)xs[j]);
}

// Newton start of the step: dt v plus the network's correction on the free
// DOFs (the held DOFs stay zero: dqg is cleared when the surrogate is set).
__global__ void k_shell_surr_guess(ShellParams P, ShellDev D, const float *yhat, const int *freemap,
                                   int nf, const float *ym, const float *ys, double *dqg) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nf) return;
  const int i = freemap[j];
  dqg[i] = P.dt * D.v[i] + (double)(yhat[j] * ys[j] + ym[j]);
}

// Nodal loads of a coupled plate: each node takes the momentum-exchange
// forces of its two surface vertices (above and below), no moments.
__global__ void k_shell_loads(ShellParams P, double *F1, const double *vforce, int v0) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= P.nn) return;
  const int vt = v0 + a, vb = v0 + P.nn + a;
  for (int k = 0; k < 3; ++k) {
    F1[6 * a + k] = vforce[3 * vt + k] + vforce[3 * vb + k];
    F1[6 * a + 3 + k] = 0.0;
  }
}

// Surface vertices and velocities of the plate from the shell state: node
// position plus / minus h/2 times the rotated reference normal (third column
// of the nodal rotation), velocities v +- omega x (h/2 d).
__global__ void k_shell_surface(ShellParams P, ShellDev D, double *surf_x, double *surf_v, int v0) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= P.nn) return;
  const double *Ra = D.R + 9 * a;
  const double hd[3] = {0.5 * P.h * Ra[2], 0.5 * P.h * Ra[5], 0.5 * P.h * Ra[8]};
  const double *w = D.v + 6 * a + 3;
  const double wx[3] = {w[1] * hd[2] - w[2] * hd[1], w[2] * hd[0] - w[0] * hd[2],
                        w[0] * hd[1] - w[1] * hd[0]};
  const int vt = v0 + a, vb = v0 + P.nn + a;
  for (int k = 0; k < 3; ++k) {
    const double x = D.X[3 * a + k] + D.u[3 * a + k];
    surf_x[3 * vt + k] = x + hd[k];
    surf_x[3 * vb + k] = x - hd[k];
    surf_v[3 * vt + k] = D.v[6 * a + k] + wx[k];
    surf_v[3 * vb + k] = D.v[6 * a + k] - wx[k];
  }
}

}  // namespace kbc

using namespace kbc;

struct fem_shell_ctx {
  ShellParams p;
  ShellDev d;
  double *F1 = nullptr;
  char *ws = nullptr;
  bool own_ws = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double *dqg = nullptr, *fcur = nullptr;  // surrogate guess, internal force at the state
  int *freemap = nullptr;                  // free DOF indices (surrogate feature order)
  int nfree = 0;
  float *xm = nullptr, *xs = nullptr, *ym = nullptr, *ys = nullptr;
  int grid = 0;      // CTAs of the cooperative launch
  int cluster = 0;   // CTAs of the single-cluster launch (0: not available)
  bool poisoned = false;
  char msg[256] = {0};
  std::vector<int32_t> fixed_h;  // Dirichlet mask (host copy)
};

// One structural step: a single cluster when available, else the cooperative grid.
static cudaError_t launch_shell_step(fem_shell_ctx *s, cudaStream_t st) {
  if (s->cluster > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(s->cluster);
    cfg.blockDim = dim3(kShellThreads);
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_shell_step<true>, s->p, s->d);
  }
  void *args[] = {(void *)&s->p, (void *)&s->d};
  return cudaLaunchCooperativeKernel((const void *)k_shell_step<false>, dim3(s->grid),
                                     dim3(kShellThreads), args, 0, st);
}

namespace {

thread_local char g_shell_msg[256];

size_t al(size_t b) { return (b + 255) / 256 * 256; }

size_t shell_layout(int nx, int ny, fem_shell_ctx *s) {
  const size_t nn = (size_t)nx * ny, ne = (size_t)(nx - 1) * (ny - 1), n = 6 * nn;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al(bytes);
    return o;
  };
  const size_t oX = take(sizeof(double) * 3 * nn), ofx = take(sizeof(int32_t) * n);
  const size_t oKl = take(sizeof(double) * 576 * ne), oRe0 = take(sizeof(double) * 9 * ne);
  const size_t oxb0 = take(sizeof(double) * 12 * ne), omt = take(sizeof(double) * nn),
               omr = take(sizeof(double) * nn);
  const size_t ou = take(sizeof(double) * 3 * nn), oR = take(sizeof(double) * 9 * nn),
               ov = take(sizeof(double) * n), oF0 = take(sizeof(double) * n);
  const size_t ou0 = take(sizeof(double) * 3 * nn), oR0 = take(sizeof(double) * 9 * nn),
               ov0 = take(sizeof(double) * n);
  const size_t ou1 = take(sizeof(double) * 3 * nn), oR1 = take(sizeof(double) * 9 * nn);
  const size_t odq = take(sizeof(double) * n), of0 = take(sizeof(double) * n),
               of = take(sizeof(double) * n), okd = take(sizeof(double) * n);
  const size_t oeg = take(sizeof(double) * kEG * ne);
  size_t ovec[7];
  for (int k = 0; k < 7; ++k) ovec[k] = take(sizeof(double) * n);
  const size_t ored = take(sizeof(double) * 6), oF1 = take(sizeof(double) * n),
               oit = take(sizeof(int) * 2);
  const size_t oFm2 = take(sizeof(double) * n), ostats = take(sizeof(int) * 4);
  // surrogate: guess, current internal force, free-DOF map, normalisation
  const size_t odqg = take(sizeof(double) * n), ofc = take(sizeof(double) * n),
               ofree = take(sizeof(int) * n), oxm = take(sizeof(float) * 5 * n),
               oxs = take(sizeof(float) * 5 * n), oym = take(sizeof(float) * n),
               oys = take(sizeof(float) * n);
  if (s) {
    char *w = s->ws;
    ShellDev &d = s->d;
    d.X = (const double *)(w + oX);
    d.fixed = (const int32_t *)(w + ofx);
    d.Kl = (double *)(w + oKl); d.Re0 = (double *)(w + oRe0); d.xb0 = (double *)(w + oxb0);
    d.mt = (double *)(w + omt); d.mr = (double *)(w + omr);
    d.u = (double *)(w + ou); d.R = (double *)(w + oR); d.v = (double *)(w + ov);
    d.F0 = (double *)(w + oF0);
    d.u0 = (double *)(w + ou0); d.R0 = (double *)(w + oR0); d.v0 = (double *)(w + ov0);
    d.u1 = (double *)(w + ou1); d.R1 = (double *)(w + oR1);
    d.dq = (double *)(w + odq); d.f0 = (double *)(w + of0); d.f = (double *)(w + of);
    d.kd = (double *)(w + okd);
    d.eg = (double *)(w + oeg);
    d.rhs = (double *)(w + ovec[0]); d.x = (double *)(w + ovec[1]); d.r = (double *)(w + ovec[2]);
    d.z = (double *)(w + ovec[3]); d.p = (double *)(w + ovec[4]); d.Ap = (double *)(w + ovec[5]);
    d.Ap2 = (double *)(w + ovec[6]);
    d.red = (double *)(w + ored);
    s->F1 = (double *)(w + oF1);
    d.F1 = s->F1;
    d.iters = (int *)(w + oit);
    d.Fm2 = (double *)(w + oFm2);
    d.stats = (int *)(w + ostats);
    d.dqg = nullptr;
    d.accept_tol = 0.0;
    s->dqg = (double *)(w + odqg);
    s->fcur = (double *)(w + ofc);
    s->freemap = (int *)(w + ofree);
    s->xm = (float *)(w + oxm); s->xs = (float *)(w + oxs);
    s->ym = (float *)(w + oym); s->ys = (float *)(w + oys);
  }
  return off;
}

const char *shell_validate(const fem_shell_config *c) {
  if (!c) return "config is NULL";
  if (c->nx < 2 || c->ny < 2 || (long long)c->nx * c->ny > kShellMaxNodes)
    return "nx, ny >= 2 and nx * ny <= 4096";
  if (!c->X || !c->fixed) return "X and fixed are required";
  if (!(c->E > 0 && c->h > 0 && c->rho > 0 && c->nu >= 0 && c->nu < 0.5))
    return "E, h, rho > 0 and 0 <= nu < 0.5";
  if (!(c->theta > 0 && c->theta <= 1) || !(c->lambda > 0 && c->lambda <= 1) || c->max_it < 1 ||
      !(c->dt > 0))
    return "bad time-integration parameters";
  return nullptr;
}

}  // namespace

#define SHELL_CK(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      s->poisoned = true;                                                           \
      snprintf(s->msg, sizeof(s->msg), "%s: %s", #call, cudaGetErrorString(e_));    \
      return LBM_ECUDA;                                                             \
    }                                                                               \
  } while (0)

extern "C" {

lbm_status fem_shell_workspace_size(const fem_shell_config *c, size_t *bytes) {
  if (!bytes || shell_validate(c)) return LBM_EINVAL;
  *bytes = shell_layout(c->nx, c->ny, nullptr);
  return LBM_OK;
}

lbm_status fem_shell_create(const fem_shell_config *c, void *workspace, size_t bytes,
                            fem_shell_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (const char *why = shell_validate(c)) {
    snprintf(g_shell_msg, sizeof(g_shell_msg), "fem_shell_create: %s", why);
    return LBM_EINVAL;
  }
  fem_shell_ctx *s = new (std::nothrow) fem_shell_ctx();
  if (!s) return LBM_ENOMEM;
  const size_t need = shell_layout(c->nx, c->ny, nullptr);
  if (workspace) {
    if (bytes < need || ((uintptr_t)workspace % 256)) {
      delete s;
      snprintf(g_shell_msg, sizeof(g_shell_msg), "fem_shell_create: workspace needs %zu bytes", need);
      return LBM_ENOMEM;
    }
    s->ws = (char *)workspace;
  } else {
    if (cudaMalloc((void **)&s->ws, need) != cudaSuccess) {
      delete s;
      return LBM_ENOMEM;
    }
    s->own_ws = true;
  }
  if (c->stream) {
    s->stream = (cudaStream_t)c->stream;
  } else {
    cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    s->own_stream = true;
  }
  shell_layout(c->nx, c->ny, s);
  ShellParams &p = s->p;
  p.nx = c->nx; p.ny = c->ny; p.nn = c->nx * c->ny; p.ne = (c->nx - 1) * (c->ny - 1);
  p.n = 6 * p.nn;
  p.E = c->E; p.nu = c->nu; p.h = c->h; p.rho = c->rho;
  p.theta = c->theta; p.lambda = c->lambda; p.rtol = c->rtol; p.atol = c->atol; p.dt = c->dt;
  p.max_it = c->max_it;
  p.max_cg = c->max_cg > 0 ? c->max_cg : 4 * p.n;
  p.cg_rtol = c->cg_rtol > 0 ? c->cg_rtol : 1e-3;
  cudaError_t e = cudaMemsetAsync(s->ws, 0, need, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)s->d.X, c->X, sizeof(double) * 3 * p.nn, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)s->d.fixed, c->fixed, sizeof(int32_t) * p.n, cudaMemcpyDefault,
                        s->stream);
  if (e == cudaSuccess) {
    s->fixed_h.resize(p.n);
    e = cudaMemcpy(s->fixed_h.data(), c->fixed, sizeof(int32_t) * p.n, cudaMemcpyDefault);
  }
  if (e == cudaSuccess) {
    std::vector<double> Rid(9 * (size_t)p.nn, 0.0);
    for (int a = 0; a < p.nn; ++a) Rid[9 * a] = Rid[9 * a + 4] = Rid[9 * a + 8] = 1.0;
    e = cudaMemcpyAsync(s->d.R, Rid.data(), sizeof(double) * 9 * p.nn, cudaMemcpyHostToDevice,
                        s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  if (e == cudaSuccess) {
    k_shell_setup<<<p.ne, kShellThreads, 0, s->stream>>>(p, s->d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shell_step<false>, kShellThreads, 0);
  if (e != cudaSuccess || !coop || per_sm < 1) {
    snprintf(g_shell_msg, sizeof(g_shell_msg), "fem_shell_create: %s",
             e != cudaSuccess ? cudaGetErrorString(e) : "cooperative launch unavailable");
    if (s->own_ws) cudaFree(s->ws);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return LBM_ECUDA;
  }
  const int warps = kShellThreads / 32;
  s->grid = (p.ne + warps - 1) / warps;
  if (s->grid > sms * per_sm) s->grid = sms * per_sm;
  // One thread-block cluster of up to 16 CTAs would replace the grid-wide
  // barriers by cluster barriers, but on the 16 x 8 plate it measured slower
  // (2.48 ms against 1.58 ms per step: the per-element FP64 chains then share
  // 16 SMs), so the cooperative grid with one element per warp is used.
  const bool try_cluster = false;
  int want = (p.ne + warps - 1) / warps;
  if (want > 16) want = 16;
  if (want > 8 &&
      cudaFuncSetAttribute(k_shell_step<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    want = 8;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(want);
  cfg.blockDim = dim3(kShellThreads);
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = want;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (try_cluster && cudaOccupancyMaxActiveClusters(&nclusters, k_shell_step<true>, &cfg) == cudaSuccess &&
      nclusters >= 1)
    s->cluster = want;
  cudaGetLastError();
  *out = s;
  return LBM_OK;
}

lbm_status fem_shell_step(fem_shell_ctx *s, const double *F1) {
  if (!s || !F1) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  SHELL_CK(cudaMemcpyAsync(s->F1, F1, sizeof(double) * s->p.n, cudaMemcpyDefault, s->stream));
  SHELL_CK(launch_shell_step(s, s->stream));
  return LBM_OK;
}

lbm_status fem_shell_get_state(fem_shell_ctx *s, double *u, double *R, double *v, int *iters) {
  if (!s) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  const size_t nn = s->p.nn;
  if (u) SHELL_CK(cudaMemcpyAsync(u, s->d.u, sizeof(double) * 3 * nn, cudaMemcpyDefault, s->stream));
  if (R) SHELL_CK(cudaMemcpyAsync(R, s->d.R, sizeof(double) * 9 * nn, cudaMemcpyDefault, s->stream));
  if (v) SHELL_CK(cudaMemcpyAsync(v, s->d.v, sizeof(double) * 6 * nn, cudaMemcpyDefault, s->stream));
  if (iters) SHELL_CK(cudaMemcpyAsync(iters, s->d.iters, sizeof(int) * 2, cudaMemcpyDefault, s->stream));
  SHELL_CK(cudaStreamSynchronize(s->stream));
  return LBM_OK;
}

lbm_status fem_shell_set_state(fem_shell_ctx *s, const double *u, const double *R, const double *v,
                               const double *F0) {
  if (!s) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  const size_t nn = s->p.nn;
  if (u) SHELL_CK(cudaMemcpyAsync(s->d.u, u, sizeof(double) * 3 * nn, cudaMemcpyDefault, s->stream));
  if (R) SHELL_CK(cudaMemcpyAsync(s->d.R, R, sizeof(double) * 9 * nn, cudaMemcpyDefault, s->stream));
  if (v) SHELL_CK(cudaMemcpyAsync(s->d.v, v, sizeof(double) * 6 * nn, cudaMemcpyDefault, s->stream));
  if (F0) SHELL_CK(cudaMemcpyAsync(s->d.F0, F0, sizeof(double) * 6 * nn, cudaMemcpyDefault, s->stream));
  SHELL_CK(cudaStreamSynchronize(s->stream));
  return LBM_OK;
}

const char *fem_shell_last_error(const fem_shell_ctx *s) { return s ? s->msg : g_shell_msg; }

void fem_shell_destroy(fem_shell_ctx *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  if (s->own_ws) cudaFree(s->ws);
  delete s;
}

}  // extern "C"

namespace kbc {

int shell_nodes(const fem_shell_ctx *s) { return s->p.nn; }

cudaError_t launch_shell_surface(fem_shell_ctx *s, double *surf_x, double *surf_v, int v0,
                                 cudaStream_t st) {
  k_shell_surface<<<(s->p.nn + 127) / 128, 128, 0, st>>>(s->p, s->d, surf_x, surf_v, v0);
  return cudaGetLastError();
}

// Coupled structural step on the lattice stream: nodal loads from the
// surface forces, the cooperative shell step, the new plate surface.
cudaError_t launch_shell_coupled(fem_shell_ctx *s, const double *vforce, double *surf_x,
                                 double *surf_v, int v0, cudaStream_t st) {
  k_shell_loads<<<(s->p.nn + 127) / 128, 128, 0, st>>>(s->p, s->F1, vforce, v0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_shell_step(s, st);
  if (e != cudaSuccess) return e;
  return launch_shell_surface(s, surf_x, surf_v, v0, st);
}

}  // namespace kbc

namespace kbc {

int shell_free_dofs(const fem_shell_ctx *s) {
  int nf = 0;
  for (int32_t f : s->fixed_h) nf += f ? 0 : 1;
  return nf;
}

// Normalisation of the surrogate network (5 nf inputs, nf outputs) and the
// free-DOF map; clears the guess and the counters.
lbm_status shell_set_surrogate(fem_shell_ctx *s, const float *in_mean, const float *in_std,
                               const float *out_mean, const float *out_std) {
  std::vector<int> map;
  for (int i = 0; i < s->p.n; ++i)
    if (!s->fixed_h[i]) map.push_back(i);
  const size_t nf = map.size();
  s->nfree = (int)nf;
  cudaError_t e = cudaMemcpyAsync(s->freemap, map.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->xm, in_mean, sizeof(float) * 5 * nf, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->xs, in_std, sizeof(float) * 5 * nf, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->ym, out_mean, sizeof(float) * nf, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->ys, out_std, sizeof(float) * nf, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->dqg, 0, sizeof(double) * s->p.n, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.stats, 0, sizeof(int) * 4, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

lbm_status shell_get_stats(fem_shell_ctx *s, int *stats, int reset) {
  cudaError_t e = cudaMemcpyAsync(stats, s->d.stats, sizeof(int) * 4, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(s->d.stats, 0, sizeof(int) * 4, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// Coupled step with the surrogate: loads, internal force of the state,
// network input, forward pass, guess, shell step started from the guess
// (accepted by its residual or refined by Newton), surface.
cudaError_t launch_shell_coupled_guess(fem_shell_ctx *s, const double *vforce, double *surf_x,
                                       double *surf_v, int v0, double accept_tol, mlp_ctx *mlp,
                                       cudaStream_t st) {
  k_shell_loads<<<(s->p.nn + 127) / 128, 128, 0, st>>>(s->p, s->F1, vforce, v0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(s->fcur, 0, sizeof(double) * s->p.n, st);
  if (e != cudaSuccess) return e;
  k_shell_force_now<<<(s->p.ne + 3) / 4, kShellThreads, 0, st>>>(s->p, s->d, s->fcur);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nf = s->nfree;
  k_shell_surr_input<<<(5 * nf + 127) / 128, 128, 0, st>>>(s->p, s->d, s->fcur, s->freemap, nf, s->xm,
                                                          s->xs, mlp_input_buffer(mlp));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float *yhat = nullptr, *xin = nullptr;
  if (mlp_forward_device(mlp, 1, st, &yhat, &xin) != LBM_OK) return cudaErrorLaunchFailure;
  k_shell_surr_guess<<<(nf + 127) / 128, 128, 0, st>>>(s->p, s->d, yhat, s->freemap, nf, s->ym, s->ys,
                                                      s->dqg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ShellDev saved = s->d;
  s->d.dqg = s->dqg;
  s->d.accept_tol = accept_tol;
  e = launch_shell_step(s, st);
  s->d = saved;
  if (e != cudaSuccess) return e;
  return launch_shell_surface(s, surf_x, surf_v, v0, st);
}

}  // namespace kbc
