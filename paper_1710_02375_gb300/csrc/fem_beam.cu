// fem_beam.cu -- FP64 structural step on the GPU: 2-D co-rotational
// Euler-Bernoulli beam, one-step-theta time integration in the two-field
// (v, u) form and Newton-Raphson with a constant line-search relaxation
// (arXiv 1710.02375, section "Structural modeling": Eqs. (timeInt),
// (timeDiscrete_solid_velocity), (timeDiscrete_solid_displacement), Newton
// update with lambda; section "Fluid-structure coupling" for the loads).
//
// Element a-b (reference length L0, chord angle b0; current length L, angle
// b): ul = L - L0, t1 = th_a - (b - b0), t2 = th_b - (b - b0);
// N = EA ul/L0, M1 = 2EI/L0 (2 t1 + t2), M2 = 2EI/L0 (t1 + 2 t2);
// f = B^T (N, M1, M2); K = B^T D B + N/L z z^T + (M1 + M2)/L^2 (r z^T + z r^T).
// Mass: consistent Hermite mass of the linear element (constant).
// Step: R(u1) = M (v1 - v0)/dt - th (F1 - f(u1)) - (1 - th)(F0 - f(u0)),
// v1 = ((u1 - u0)/dt - (1 - th) v0)/th, J = M/(th dt^2) + th K(u1),
// u1 += lambda du until |R| <= rtol |R0| + atol.
//
// One CTA per beam.  Matrices are banded (node-major DOFs: half bandwidth 5)
// in shared memory; element loops run in two colour passes (even, odd
// elements) so no two threads add into the same entries; the Newton system
// (block tridiagonal in the 3 x 3 node blocks; no pivoting: the mass term
// keeps J diagonally dominant at these steps) is solved by block elimination
// from both ends at once on two threads in FP32 registers (an inexact Newton
// step: residual, stopping test and state stay FP64).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <type_traits>

#include "../../include/kbc_lbm.h"
#include "fem_beam.cuh"
#include "lbm_internal.h"

namespace kbc {

constexpr int KB = 5;            // half bandwidth
constexpr int BW = 2 * KB + 1;   // band width
constexpr int kMaxN = 3 * kMaxBeamNodes, kMaxE = kMaxBeamNodes - 1;


__device__ __forceinline__ double &band(double *A, int i, int j) { return A[i * BW + (j - i + KB)]; }
template <typename T>
__device__ __forceinline__ T &bandf(T *A, int i, int j) { return A[i * BW + (j - i + KB)]; }
template <typename T>
__device__ __forceinline__ T bandf(const T *__restrict__ A, int i, int j) {
  return A[i * BW + (j - i + KB)];
}

__device__ void element_geom(const BeamParams &p, const double *X, const double *u, int a,
                             double &L0, double &L, double &c, double &s, double &rot) {
  const int b = a + 1;
  const double X0x = X[2 * b] - X[2 * a], X0y = X[2 * b + 1] - X[2 * a + 1];
  L0 = sqrt(X0x * X0x + X0y * X0y);
  const double b0 = atan2(X0y, X0x);
  const double dx = X0x + u[3 * b] - u[3 * a], dy = X0y + u[3 * b + 1] - u[3 * a + 1];
  L = sqrt(dx * dx + dy * dy);
  const double bb = atan2(dy, dx);
  c = dx / L;
  s = dy / L;
  rot = bb - b0;
  const double PI = 3.14159265358979323846;
  while (rot > PI) rot -= 2 * PI;
  while (rot <= -PI) rot += 2 * PI;
}

// Add element e's internal force (and tangent if K != nullptr) at state u.
__device__ void element_internal(const BeamParams &p, const double *X, const double *u, int e,
                                 double *f, double *K) {
  double L0, L, c, s, rot;
  element_geom(p, X, u, e, L0, L, c, s, rot);
  const int a = e, b = e + 1;
  const double ul = L - L0, t1 = u[3 * a + 2] - rot, t2 = u[3 * b + 2] - rot;
  const double N = p.EA * ul / L0;
  const double k2 = 2.0 * p.EI / L0;
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
  const int d0 = 3 * a;
  for (int k = 0; k < 6; ++k) f[d0 + k] += Bm[0][k] * q[0] + Bm[1][k] * q[1] + Bm[2][k] * q[2];
  if (K) {
    const double D[3][3] = {{p.EA / L0, 0, 0}, {0, 2 * k2, k2}, {0, k2, 2 * k2}};
    for (int k = 0; k < 6; ++k)
      for (int l = 0; l < 6; ++l) {
        double v = 0.0;
        for (int m = 0; m < 3; ++m)
          for (int q2 = 0; q2 < 3; ++q2) v += Bm[m][k] * D[m][q2] * Bm[q2][l];
        v += N / L * z[k] * z[l] + (M1 + M2) / (L * L) * (r[k] * z[l] + z[k] * r[l]);
        band(K, d0 + k, d0 + l) += v;
      }
  }
}

__device__ void element_mass(const BeamParams &p, const double *X, int e, double *M) {
  const int a = e, b = e + 1;
  const double X0x = X[2 * b] - X[2 * a], X0y = X[2 * b + 1] - X[2 * a + 1];
  const double L = sqrt(X0x * X0x + X0y * X0y);
  const double c = X0x / L, s = X0y / L;
  double Ml[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Ml[i][j] = 0.0;
  const double ma = p.rhoA * L / 6.0, mb = p.rhoA * L / 420.0;
  Ml[0][0] = 2 * ma; Ml[0][3] = ma; Ml[3][0] = ma; Ml[3][3] = 2 * ma;
  const int bi[4] = {1, 2, 4, 5};
  const double Mb[4][4] = {{156, 22 * L, 54, -13 * L},
                           {22 * L, 4 * L * L, 13 * L, -3 * L * L},
                           {54, 13 * L, 156, -22 * L},
                           {-13 * L, -3 * L * L, -22 * L, 4 * L * L}};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ml[bi[i]][bi[j]] = mb * Mb[i][j];
  double T[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) T[i][j] = 0.0;
  for (int k = 0; k < 2; ++k) {
    T[3 * k][3 * k] = c; T[3 * k][3 * k + 1] = s;
    T[3 * k + 1][3 * k] = -s; T[3 * k + 1][3 * k + 1] = c;
    T[3 * k + 2][3 * k + 2] = 1;
  }
  const int d0 = 3 * a;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
      for (int k = 0; k < 6; ++k)
        for (int l = 0; l < 6; ++l) v += T[k][i] * Ml[k][l] * T[l][j];
      band(M, d0 + i, d0 + j) += v;
    }
}

// Consistent mass matrix (band storage), constant: the reference orientation.
__global__ void k_beam_mass(BeamParams p, const double *X, double *M) {
  const int n = 3 * p.nn, ne = p.nn - 1;
  for (int i = threadIdx.x; i < n * BW; i += blockDim.x) M[i] = 0.0;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = 2 * threadIdx.x + pass; e < ne; e += 2 * blockDim.x) element_mass(p, X, e, M);
    __syncthreads();
  }
}

// Surface of the flag around the beam: bottom vertices 0..nn-1 (node order),
// top vertices nn..2nn-1 (reverse node order), offset h/2 along the normal of
// each cross-section.
__device__ void flag_vertex(const BeamParams &p, const double *X, const double *u, const double *v,
                            int j, double *xb, double *vb, double *xt, double *vt) {
  const double th = u[3 * j + 2], om = v[3 * j + 2];
  const double nx = -sin(th), ny = cos(th);
  const double dnx = -cos(th) * om, dny = -sin(th) * om;
  const double cx = X[2 * j] + u[3 * j], cy = X[2 * j + 1] + u[3 * j + 1];
  xb[0] = cx - 0.5 * p.h * nx; xb[1] = cy - 0.5 * p.h * ny;
  xt[0] = cx + 0.5 * p.h * nx; xt[1] = cy + 0.5 * p.h * ny;
  vb[0] = v[3 * j] - 0.5 * p.h * dnx; vb[1] = v[3 * j + 1] - 0.5 * p.h * dny;
  vt[0] = v[3 * j] + 0.5 * p.h * dnx; vt[1] = v[3 * j + 1] + 0.5 * p.h * dny;
}

// The two surface vertices of beam node j (bottom edge vertex v0 + j, top
// edge vertex v0 + 2 nn - 1 - j): 2-D positions and velocities, or, for the
// spanwise extrusion, 3-D vertices at z0 (from v0) and at z1 (from p.v1)
// moving in the plane.
__device__ void store_flag_vertices(const BeamParams &p, const double *X, const double *u,
                                    const double *v, int j, int v0, double *surf_x,
                                    double *surf_v) {
  double xb[2], vb[2], xt[2], vt[2];
  flag_vertex(p, X, u, v, j, xb, vb, xt, vt);
  const int nn = p.nn;
  if (!p.span) {
    const int ib = v0 + j, it = v0 + 2 * nn - 1 - j;
    surf_x[2 * ib] = xb[0]; surf_x[2 * ib + 1] = xb[1];
    surf_v[2 * ib] = vb[0]; surf_v[2 * ib + 1] = vb[1];
    surf_x[2 * it] = xt[0]; surf_x[2 * it + 1] = xt[1];
    surf_v[2 * it] = vt[0]; surf_v[2 * it + 1] = vt[1];
    return;
  }
  for (int end = 0; end < 2; ++end) {
    const int base = end == 0 ? v0 : p.v1;
    const double z = end == 0 ? p.z0 : p.z1;
    const int ib = base + j, it = base + 2 * nn - 1 - j;
    surf_x[3 * ib] = xb[0]; surf_x[3 * ib + 1] = xb[1]; surf_x[3 * ib + 2] = z;
    surf_v[3 * ib] = vb[0]; surf_v[3 * ib + 1] = vb[1]; surf_v[3 * ib + 2] = 0.0;
    surf_x[3 * it] = xt[0]; surf_x[3 * it + 1] = xt[1]; surf_x[3 * it + 2] = z;
    surf_v[3 * it] = vt[0]; surf_v[3 * it + 1] = vt[1]; surf_v[3 * it + 2] = 0.0;
  }
}

// ---- per-step work split for GB300's FP64 rate: each FP64 warp instruction
// occupies the FP64 pipe for many cycles, so the step is organised to keep
// FP64 instruction counts per warp low -- element scalars once per element,
// internal forces and tangent entries spread over the CTA, the tangent and
// the block-tridiagonal solve in FP32.

// Upper-triangle index pairs (k <= l) of a 6 x 6 element matrix.
__constant__ unsigned char c_pk[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__constant__ unsigned char c_pl[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

// r and z vectors of the co-rotational element (local DOF k of nodes a, b).
__device__ __forceinline__ double elem_r(int k, double c, double s) {
  const double v = (k % 3 == 0) ? c : ((k % 3 == 1) ? s : 0.0);
  return k < 3 ? -v : v;
}
__device__ __forceinline__ double elem_z(int k, double c, double s) {
  const double v = (k % 3 == 0) ? s : ((k % 3 == 1) ? -c : 0.0);
  return k < 3 ? v : -v;
}

template <typename T>
__device__ __forceinline__ T elem_rf(int k, T c, T s) {
  const T v = (k % 3 == 0) ? c : ((k % 3 == 1) ? s : (T)0);
  return k < 3 ? -v : v;
}
template <typename T>
__device__ __forceinline__ T elem_zf(int k, T c, T s) {
  const T v = (k % 3 == 0) ? s : ((k % 3 == 1) ? -c : (T)0);
  return k < 3 ? v : -v;
}

__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return 1.0 / x; }

// 3 x 3 helpers (row-major, registers of the solve precision T).
template <typename T>
__device__ __forceinline__ void inv3(const T (&S)[9], T (&A)[9]) {
  A[0] = S[4] * S[8] - S[5] * S[7];
  A[1] = S[2] * S[7] - S[1] * S[8];
  A[2] = S[1] * S[5] - S[2] * S[4];
  A[3] = S[5] * S[6] - S[3] * S[8];
  A[4] = S[0] * S[8] - S[2] * S[6];
  A[5] = S[2] * S[3] - S[0] * S[5];
  A[6] = S[3] * S[7] - S[4] * S[6];
  A[7] = S[1] * S[6] - S[0] * S[7];
  A[8] = S[0] * S[4] - S[1] * S[3];
  const T idet = recip_rn(S[0] * A[0] + S[1] * A[3] + S[2] * A[6]);
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] *= idet;
}
template <typename T>
__device__ __forceinline__ void load_block(const T *__restrict__ J, int r0, int c0, T (&B)[9]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) B[3 * a + c] = bandf(J, r0 + a, c0 + c);
}

// One elimination step of the block-tridiagonal system from either end
// (Thomas' algorithm with 3 x 3 blocks): node i with diagonal block D_i, the
// coupling C to the node eliminated before (L_i going down, U_i going up) and
// the coupling E to the node after (U_i going down, L_i going up):
//   S = D_i - C W_prev,  g = S^-1 (b_i - C g_prev),  W = S^-1 E
// g overwrites rhs_i, W goes to Wsc[i].  last: no E (end of the sweep).
template <typename T>
__device__ __forceinline__ void thomas_step(const T *__restrict__ J, T *__restrict__ rhs,
                                            T *__restrict__ Wsc, int i, int prev, int next,
                                            T (&Wp)[9], T (&gp)[3], bool first) {
  const int r0 = 3 * i;
  T S[9], b[3];
  load_block(J, r0, r0, S);
  b[0] = rhs[r0];
  b[1] = rhs[r0 + 1];
  b[2] = rhs[r0 + 2];
  if (!first) {
    T C[9];
    load_block(J, r0, 3 * prev, C);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        S[3 * a + c] -= C[3 * a] * Wp[c] + C[3 * a + 1] * Wp[3 + c] + C[3 * a + 2] * Wp[6 + c];
      b[a] -= C[3 * a] * gp[0] + C[3 * a + 1] * gp[1] + C[3 * a + 2] * gp[2];
    }
  }
  T A[9];
  inv3(S, A);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gp[a] = A[3 * a] * b[0] + A[3 * a + 1] * b[1] + A[3 * a + 2] * b[2];
    rhs[r0 + a] = gp[a];
  }
  if (next >= 0) {
    T E[9];
    load_block(J, r0, 3 * next, E);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Wp[3 * a + c] = A[3 * a] * E[c] + A[3 * a + 1] * E[3 + c] + A[3 * a + 2] * E[6 + c];
        Wsc[9 * i + 3 * a + c] = Wp[3 * a + c];
      }
  }
}

// J x = rhs for the block-tridiagonal J of the node-major beam DOFs (3 x 3
// node blocks read from band storage; no pivoting: the mass term keeps the
// diagonal blocks well conditioned), eliminated from both ends at once
// (twisted block factorisation): thread 0 (warp 0) sweeps nodes 0 .. m-1
// downwards, thread 32 (warp 1) nodes nn-1 .. m+1 upwards, thread 0 then
// solves node m from both sides, and each thread substitutes back along its
// half.  Registers of the solve precision T; x overwrites rhs.  Called by
// every thread of the CTA (it contains barriers).
template <typename T>
__device__ __forceinline__ void block_twisted(const T *__restrict__ J, T *__restrict__ rhs,
                                              T *__restrict__ Wsc, T *__restrict__ gm, int nn) {
  const int tid = threadIdx.x, m = nn / 2;
  if (tid == 0 || tid == 32) {
    T Wp[9], gp[3];
    if (tid == 0) {
      for (int i = 0; i < m; ++i) thomas_step(J, rhs, Wsc, i, i - 1, i + 1, Wp, gp, i == 0);
    } else {
      for (int i = nn - 1; i > m; --i) thomas_step(J, rhs, Wsc, i, i + 1, i - 1, Wp, gp, i == nn - 1);
    }
  }
  __syncthreads();
  if (tid == 0) {
    // node m: (D_m - L_m W_{m-1} - U_m W_{m+1}) x_m = b_m - L_m g_{m-1} - U_m g_{m+1}
    const int r0 = 3 * m;
    T S[9], b[3];
    load_block(J, r0, r0, S);
    b[0] = rhs[r0];
    b[1] = rhs[r0 + 1];
    b[2] = rhs[r0 + 2];
    for (int side = 0; side < 2; ++side) {
      const int o = side == 0 ? m - 1 : m + 1;
      if (o < 0 || o >= nn) continue;
      T C[9];
      load_block(J, r0, 3 * o, C);
      const T *W = Wsc + 9 * o, *g = rhs + 3 * o;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          S[3 * a + c] -= C[3 * a] * W[c] + C[3 * a + 1] * W[3 + c] + C[3 * a + 2] * W[6 + c];
        b[a] -= C[3 * a] * g[0] + C[3 * a + 1] * g[1] + C[3 * a + 2] * g[2];
      }
    }
    T A[9];
    inv3(S, A);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gm[a] = A[3 * a] * b[0] + A[3 * a + 1] * b[1] + A[3 * a + 2] * b[2];
      rhs[r0 + a] = gm[a];
    }
  }
  __syncthreads();
  if (tid == 0 || tid == 32) {
    T xn[3] = {gm[0], gm[1], gm[2]};
    const int step = tid == 0 ? -1 : 1;
    for (int i = m + step; i >= 0 && i < nn; i += step) {
      T x[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T *w = Wsc + 9 * i + 3 * a;
        x[a] = rhs[3 * i + a] - (w[0] * xn[0] + w[1] * xn[1] + w[2] * xn[2]);
        rhs[3 * i + a] = x[a];
      }
      xn[0] = x[0];
      xn[1] = x[1];
      xn[2] = x[2];
    }
  }
}

// T: precision of the Newton matrix and its solve (float: the default inexact
// Newton step; double: the FP64 mode).  FP32 keeps the matrix's mass part
// in MJ; FP64 forms it from M each iteration (the shared memory of the
// FP64 matrix takes the place of both FP32 arrays).
template <typename T>
struct BeamMat {
  float J[kMaxN * BW], MJ[kMaxN * BW];
};
template <>
struct BeamMat<double> {
  double J[kMaxN * BW];
};
template <typename T>
struct BeamShared {
  BeamMat<T> mat;  // Newton matrix (band storage)
  double M[kMaxN * BW];
  double u[kMaxN], u0[kMaxN], v0[kMaxN], f0[kMaxN], F1[kMaxN], R[kMaxN], D[kMaxN];
  double Rc[kMaxN];         // load part of the residual, theta F1 + (1 - theta)(F0 - f(u0))
  unsigned char fx[kMaxN];  // Dirichlet mask
  T rhs[kMaxN], W[kMaxBeamNodes * 9], gm[3];
  double X[2 * kMaxBeamNodes];
  // element scalars: constants of the step, then the current state's
  double L0[kMaxE], b0[kMaxE], EAL0[kMaxE], k2[kMaxE];
  double c[kMaxE], s[kMaxE], iL[kMaxE], N[kMaxE], M1[kMaxE], M2[kMaxE];
  double rot0[kMaxE], c0[kMaxE], s0[kMaxE];  // chord rotation and direction at the step's start
  // copies in the solve precision for the tangent: c, s, 1/L, N/L,
  // (M1 + M2)/L^2, EA/L0, k2
  T tc[kMaxE], ts[kMaxE], tiL[kMaxE], tNL[kMaxE], tML[kMaxE], tEA[kMaxE], tk2[kMaxE];
  double red[4];
};

// Element state scalars at the displacement u (thread per element).  base:
// the step's start state, whose chord rotation comes from a full atan2 and is
// kept with the chord direction; otherwise the rotation is that start value
// plus the angle from the start chord to the current one, by the arctangent
// series when it is small (|tan| < 0.1: terms to t^15, truncation below
// 1e-17 relative) and by atan2 otherwise.
template <typename T>
__device__ __forceinline__ void elem_state(const BeamParams &p, BeamShared<T> &S, const double *u,
                                           int ne, bool base) {
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int a = e, b = e + 1;
    const double dx = S.X[2 * b] - S.X[2 * a] + u[3 * b] - u[3 * a];
    const double dy = S.X[2 * b + 1] - S.X[2 * a + 1] + u[3 * b + 1] - u[3 * a + 1];
    const double L = sqrt(dx * dx + dy * dy);
    const double iL = 1.0 / L;
    const double PI = 3.14159265358979323846;
    double rot;
    if (base) {
      rot = atan2(dy, dx) - S.b0[e];
      if (rot > PI) rot -= 2 * PI;
      if (rot <= -PI) rot += 2 * PI;
      S.rot0[e] = rot;
      S.c0[e] = dx * iL;
      S.s0[e] = dy * iL;
    } else {
      const double y = S.c0[e] * dy - S.s0[e] * dx, x = S.c0[e] * dx + S.s0[e] * dy;
      double dr;
      if (x > 0.0 && fabs(y) < 0.1 * x) {
        const double t = y / x, t2 = t * t;
        double q = -1.0 / 15.0;
        q = q * t2 + 1.0 / 13.0;
        q = q * t2 - 1.0 / 11.0;
        q = q * t2 + 1.0 / 9.0;
        q = q * t2 - 1.0 / 7.0;
        q = q * t2 + 1.0 / 5.0;
        q = q * t2 - 1.0 / 3.0;
        q = q * t2 + 1.0;
        dr = t * q;
      } else {
        dr = atan2(y, x);
      }
      rot = S.rot0[e] + dr;
      if (rot > PI) rot -= 2 * PI;
      if (rot <= -PI) rot += 2 * PI;
    }
    const double t1 = u[3 * a + 2] - rot, t2 = u[3 * b + 2] - rot;
    S.c[e] = dx * iL;
    S.s[e] = dy * iL;
    S.iL[e] = iL;
    S.N[e] = S.EAL0[e] * (L - S.L0[e]);
    S.M1[e] = S.k2[e] * (2 * t1 + t2);
    S.M2[e] = S.k2[e] * (t1 + 2 * t2);
    S.tc[e] = (T)S.c[e];
    S.ts[e] = (T)S.s[e];
    S.tiL[e] = (T)iL;
    S.tNL[e] = (T)(S.N[e] * iL);
    S.tML[e] = (T)((S.M1[e] + S.M2[e]) * iL * iL);
  }
}

// Internal force of DOF i from its (at most two) elements.
template <typename T>
__device__ __forceinline__ double dof_internal(const BeamShared<T> &S, int i, int ne) {
  const int j = i / 3, q = i % 3;
  double f = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int e = side == 0 ? j - 1 : j;  // element with node j as its b / a node
    if (e < 0 || e >= ne) continue;
    const int k = side == 0 ? 3 + q : q;
    const double c = S.c[e], s = S.s[e];
    f += elem_r(k, c, s) * S.N[e] - elem_z(k, c, s) * S.iL[e] * (S.M1[e] + S.M2[e]) +
         (k == 2 ? S.M1[e] : 0.0) + (k == 5 ? S.M2[e] : 0.0);
  }
  return f;
}

// Block sum of one value per thread (all threads call; result to all).
template <typename T>
__device__ __forceinline__ double block_sum(BeamShared<T> &S, double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) S.red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += S.red[k];
  return t;
}

// One structural step.  Loads F1 come from F1_in (standalone) or from the
// momentum-exchange forces of the flag's surface vertices (coupled: vforce,
// surf_x / surf_v of the whole surface, the flag's vertices start at v0).
// Launch: one CTA of 128 threads per beam.
template <bool COUPLED, typename T>
__device__ __forceinline__ void beam_step_body(const BeamParams &p, const BeamDev &d,
                                               const double *__restrict__ F1_in,
                                               const double *__restrict__ vforce, double *surf_x,
                                               double *surf_v, int v0) {
  __shared__ BeamShared<T> S;
  constexpr bool FP64 = std::is_same<T, double>::value;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = p.nn, n = 3 * nn, ne = nn - 1;
  const double a_v = 1.0 / (p.theta * p.dt), i_th = 1.0 / p.theta, i_dt = 1.0 / p.dt;
  const double cM = 1.0 / (p.theta * p.dt * p.dt);
  for (int i = tid; i < n; i += nt) {
    S.u0[i] = d.u[i];
    S.u[i] = (d.u_guess && !d.fixed[i]) ? d.u_guess[i] : d.u[i];
    S.v0[i] = d.v[i];
  }
  for (int i = tid; i < n * BW; i += nt) {
    S.M[i] = d.M[i];
    if constexpr (!FP64) S.mat.MJ[i] = (float)(d.M[i] * cM);
  }
  for (int i = tid; i < 2 * nn; i += nt) S.X[i] = d.X[i];
  __syncthreads();
  for (int e = tid; e < ne; e += nt) {
    const double X0x = S.X[2 * e + 2] - S.X[2 * e], X0y = S.X[2 * e + 3] - S.X[2 * e + 1];
    const double L0 = sqrt(X0x * X0x + X0y * X0y);
    S.L0[e] = L0;
    S.b0[e] = atan2(X0y, X0x);
    S.EAL0[e] = p.EA / L0;
    S.k2[e] = 2.0 * p.EI / L0;
    S.tEA[e] = (T)S.EAL0[e];
    S.tk2[e] = (T)S.k2[e];
  }
  // ---- loads F1
  if (COUPLED) {
    // nodal loads: the forces of the node's two surface vertices (their
    // moments about the centre line are not transferred: the flag-tip
    // rotation is a stiff mode that the staggered one-step lag destabilises)
    for (int j = tid; j < nn; j += nt) {
      const int vb = v0 + j, vt = v0 + 2 * nn - 1 - j;
      double fx = vforce[3 * vb] + vforce[3 * vt], fy = vforce[3 * vb + 1] + vforce[3 * vt + 1];
      if (p.span) {
        // quasi-2-D: the same polygon vertices at the far end of the span,
        // the summed force per unit span
        const int wb = p.v1 + j, wt = p.v1 + 2 * nn - 1 - j;
        fx = (fx + (vforce[3 * wb] + vforce[3 * wt])) * p.inv_depth;
        fy = (fy + (vforce[3 * wb + 1] + vforce[3 * wt + 1])) * p.inv_depth;
      }
      S.F1[3 * j] = fx;
      S.F1[3 * j + 1] = fy;
      S.F1[3 * j + 2] = 0.0;
    }
  } else {
    for (int i = tid; i < n; i += nt) S.F1[i] = F1_in[i];
  }
  __syncthreads();
  // ---- f(u0)
  elem_state(p, S, S.u0, ne, true);
  __syncthreads();
  double fe2 = 0.0;
  for (int i = tid; i < n; i += nt) {
    const double f0 = dof_internal(S, i, ne), F0 = d.F0[i];
    const bool fixed = d.fixed[i] != 0;
    S.f0[i] = f0;
    S.fx[i] = fixed;
    S.Rc[i] = p.theta * S.F1[i] + (1.0 - p.theta) * (F0 - f0);
    const double fe = fixed ? 0.0 : p.theta * S.F1[i] + (1.0 - p.theta) * F0;
    fe2 += fe * fe;
  }
  __syncthreads();
  const double fext = sqrt(block_sum(S, fe2));
  // ---- Newton iterations with the constant relaxation lambda.  The
  // convergence test is relative to the residual at the start u0, also when
  // the iteration starts from a surrogate guess, so that a guess changes
  // where Newton starts but not where it stops.
  double r0 = -1.0;
  if (d.u_guess) {
    double part = 0.0;
    for (int i = tid; i < n; i += nt) {
      double mv = 0.0;
      for (int j = (i - KB > 0 ? i - KB : 0); j <= (i + KB < n - 1 ? i + KB : n - 1); ++j)
        mv += band(S.M, i, j) * (-S.v0[j] * i_th);
      const double R = mv * i_dt - p.theta * (S.F1[i] - S.f0[i]) - (1.0 - p.theta) * (d.F0[i] - S.f0[i]);
      if (!d.fixed[i]) part += R * R;
    }
    r0 = sqrt(block_sum(S, part));
  }
  int it = 0, conv = 0;
  for (it = 0; it < p.max_it; ++it) {
    elem_state(p, S, S.u, ne, false);
    for (int i = tid; i < n; i += nt) S.D[i] = (S.u[i] - S.u0[i]) * a_v - S.v0[i] * i_th;
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < n; i += nt) {
      double mv = 0.0;
      for (int j = (i - KB > 0 ? i - KB : 0); j <= (i + KB < n - 1 ? i + KB : n - 1); ++j)
        mv += band(S.M, i, j) * S.D[j];
      const double f = dof_internal(S, i, ne);
      double R = mv * i_dt + p.theta * f - S.Rc[i];
      if (S.fx[i]) R = 0.0;
      S.rhs[i] = (T)-R;  // right-hand side of J du = -R
      part += R * R;
    }
    const double rn = sqrt(block_sum(S, part));
    if (it == 0 && d.u_guess && p.accept_tol > 0.0) {
      // surrogate guess: accept it when the residual is small against the loads
      const bool accept = rn <= p.accept_tol * fext;
      if (tid == 0 && d.stats) atomicAdd(&d.stats[accept ? 0 : 1], 1);
      if (accept) {
        conv = 1;
        break;
      }
    }
    if (r0 < 0) r0 = rn;
    if (rn <= p.rtol * r0 + p.atol) {
      conv = 1;
      break;
    }
    // ---- Newton matrix J = M / (theta dt^2) + theta K (band), Dirichlet
    // rows / columns, and the solve of J du = -R in precision T.  FP32 (the
    // default): an inexact Newton step (relative error ~1e-6 on this
    // diagonally dominant J) while the residual and its stopping test stay
    // FP64, so the converged state meets the same FP64 test, and the serial
    // elimination chain stays off GB300's scarce FP64 pipe.  FP64: the exact
    // Newton step of the oracle.
    for (int i = tid; i < n * BW; i += nt) {
      if constexpr (FP64) S.mat.J[i] = S.M[i] * cM;
      else S.mat.J[i] = S.mat.MJ[i];
    }
    __syncthreads();
    const T thf = (T)p.theta;
    for (int colour = 0; colour < 2; ++colour) {
      const int nel = (ne - colour + 1) / 2;  // elements colour, colour + 2, ...
      for (int w = tid; w < nel * 21; w += nt) {
        const int e = colour + 2 * (w / 21), pk = c_pk[w % 21], pl = c_pl[w % 21];
        const T c = S.tc[e], s = S.ts[e], iL = S.tiL[e], k2 = S.tk2[e];
        const T rk = elem_rf(pk, c, s), rl = elem_rf(pl, c, s);
        const T zk = elem_zf(pk, c, s), zl = elem_zf(pl, c, s);
        const T b1k = -zk * iL + (pk == 2 ? (T)1 : (T)0), b2k = -zk * iL + (pk == 5 ? (T)1 : (T)0);
        const T b1l = -zl * iL + (pl == 2 ? (T)1 : (T)0), b2l = -zl * iL + (pl == 5 ? (T)1 : (T)0);
        T v = S.tEA[e] * rk * rl + b1k * ((T)2 * k2 * b1l + k2 * b2l) +
              b2k * (k2 * b1l + (T)2 * k2 * b2l) + S.tNL[e] * zk * zl +
              S.tML[e] * (rk * zl + zk * rl);
        v *= thf;
        const int gi = 3 * e + pk, gj = 3 * e + pl;
        bandf(S.mat.J, gi, gj) += v;
        if (pk != pl) bandf(S.mat.J, gj, gi) += v;
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n * BW; idx += nt) {
      const int i = idx / BW, j = i + idx % BW - KB;
      if (j >= 0 && j < n && (S.fx[i] || S.fx[j])) S.mat.J[idx] = (i == j) ? (T)1 : (T)0;
    }
    __syncthreads();
    block_twisted(S.mat.J, S.rhs, S.W, S.gm, nn);
    __syncthreads();
    for (int i = tid; i < n; i += nt) S.u[i] += p.lambda * (double)S.rhs[i];
    __syncthreads();
  }
  // ---- final velocities, state, loads
  for (int i = tid; i < n; i += nt) {
    double ui = S.u[i], vi = (S.u[i] - S.u0[i]) * a_v - (1.0 - p.theta) * i_th * S.v0[i];
    if (d.fixed[i]) { ui = 0.0; vi = 0.0; }
    d.u[i] = ui;
    d.v[i] = vi;
    d.F0[i] = S.F1[i];
    S.u[i] = ui;
    S.R[i] = vi;
  }
  if (tid == 0) {
    *d.iters = conv ? it : -it - 1;
    if (d.stats) {
      atomicAdd(&d.stats[2], it);  // Newton solves of this step
      atomicAdd(&d.stats[3], 1);
    }
  }
  __syncthreads();
  if (COUPLED) {
    // transfer displacement and velocity to the surface mesh
    for (int j = tid; j < nn; j += nt) store_flag_vertices(p, S.X, S.u, S.R, j, v0, surf_x, surf_v);
  }
}

template <bool COUPLED, typename T>
__global__ void __launch_bounds__(128)
    k_beam_step(BeamParams p, BeamDev d, const double *__restrict__ F1_in,
                const double *__restrict__ vforce, double *surf_x, double *surf_v, int v0) {
  beam_step_body<COUPLED, T>(p, d, F1_in, vforce, surf_x, surf_v, v0);
}

// Launch of one beam step in the solve precision the beam's parameters ask for.
template <bool COUPLED>
static cudaError_t launch_beam_step(const BeamParams &p, const BeamDev &d, const double *F1_in,
                                    const double *vforce, double *surf_x, double *surf_v, int v0,
                                    cudaStream_t s) {
  if (p.solve64)
    k_beam_step<COUPLED, double><<<1, 128, 0, s>>>(p, d, F1_in, vforce, surf_x, surf_v, v0);
  else
    k_beam_step<COUPLED, float><<<1, 128, 0, s>>>(p, d, F1_in, vforce, surf_x, surf_v, v0);
  return cudaGetLastError();
}

// One CTA per coupled beam of a batch; each launch takes the beams of its
// solve precision.
template <typename T>
__global__ void __launch_bounds__(128) k_beam_step_batch(const BeamBatchDesc *__restrict__ d) {
  const BeamBatchDesc &b = d[blockIdx.x];
  if ((b.p.solve64 != 0) != std::is_same<T, double>::value) return;
  beam_step_body<true, T>(b.p, b.d, nullptr, b.vforce, b.surf_x, b.surf_v, b.v0);
}

cudaError_t launch_beam_batch(const BeamBatchDesc *d, int n, int any_fp64, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_beam_step_batch<float><<<n, 128, 0, s>>>(d);
  if (any_fp64) k_beam_step_batch<double><<<n, 128, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace kbc

using namespace kbc;

struct fem_ctx {
  BeamParams p;
  BeamDev d;
  // surrogate coupling: nodal load history ring [3][nn][2] (FP64), guess,
  // statistics (accepted, rejected, Newton solves, steps), normalisation of
  // the network input / output
  double *hist = nullptr;
  double *u_guess = nullptr;
  int *stats = nullptr;
  float *in_mean = nullptr, *in_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
  char *ws = nullptr;
  bool own_ws = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double *F1 = nullptr;   // staging of standalone loads
  bool poisoned = false;
  char msg[256] = {0};
};

static size_t fem_bytes(int nn) {
  const size_t n = 3 * (size_t)nn;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t nin = surrogate_inputs(nn), nout = 3 * (size_t)nn - 3;
  return al(sizeof(double) * 2 * nn) + al(sizeof(int32_t) * n) + 4 * al(sizeof(double) * n) +
         al(sizeof(double) * n * BW) +
         al(sizeof(int)) + al(sizeof(double) * 6 * nn) + al(sizeof(double) * n) +
         al(kFemStats * sizeof(int)) + 2 * al(sizeof(float) * nin) + 2 * al(sizeof(float) * nout);
}

static thread_local char g_fem_msg[256];

extern "C" {

lbm_status fem_beam_workspace_size(const fem_beam_config *c, size_t *bytes) {
  if (!c || !bytes || c->nn < 2 || c->nn > kMaxBeamNodes) return LBM_EINVAL;
  *bytes = fem_bytes(c->nn);
  return LBM_OK;
}

lbm_status fem_beam_create(const fem_beam_config *c, void *workspace, size_t bytes, fem_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!c || c->nn < 2 || c->nn > kMaxBeamNodes || !c->X || !c->fixed ||
      !(c->EA > 0 && c->EI > 0 && c->rhoA > 0 && c->thickness >= 0) ||
      !(c->theta > 0 && c->theta <= 1) || !(c->lambda > 0 && c->lambda <= 1) || c->max_it < 1 ||
      !(c->dt > 0)) {
    snprintf(g_fem_msg, sizeof(g_fem_msg), "fem_beam_create: bad configuration (nn in [2, %d])",
             kMaxBeamNodes);
    return LBM_EINVAL;
  }
  fem_ctx *f = new (std::nothrow) fem_ctx();
  if (!f) return LBM_ENOMEM;
  const size_t need = fem_bytes(c->nn);
  if (workspace) {
    if (bytes < need || ((uintptr_t)workspace % 256) != 0) {
      delete f;
      snprintf(g_fem_msg, sizeof(g_fem_msg), "fem_beam_create: workspace needs %zu bytes", need);
      return LBM_ENOMEM;
    }
    f->ws = (char *)workspace;
  } else {
    if (cudaMalloc((void **)&f->ws, need) != cudaSuccess) {
      delete f;
      return LBM_ENOMEM;
    }
    f->own_ws = true;
  }
  if (c->stream) {
    f->stream = (cudaStream_t)c->stream;
  } else {
    cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
    f->own_stream = true;
  }
  const int nn = c->nn;
  const size_t n = 3 * (size_t)nn;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char *p = f->ws;
  double *X = (double *)p; p += al(sizeof(double) * 2 * nn);
  int32_t *fx = (int32_t *)p; p += al(sizeof(int32_t) * n);
  double *u = (double *)p; p += al(sizeof(double) * n);
  double *v = (double *)p; p += al(sizeof(double) * n);
  double *F0 = (double *)p; p += al(sizeof(double) * n);
  double *F1 = (double *)p; p += al(sizeof(double) * n);
  int *iters = (int *)p; p += al(sizeof(int));
  double *Mb = (double *)p; p += al(sizeof(double) * n * BW);
  const size_t nin = surrogate_inputs(nn), nout = 3 * (size_t)nn - 3;
  f->hist = (double *)p; p += al(sizeof(double) * 6 * nn);
  f->u_guess = (double *)p; p += al(sizeof(double) * n);
  f->stats = (int *)p; p += al(kFemStats * sizeof(int));
  f->in_mean = (float *)p; p += al(sizeof(float) * nin);
  f->in_std = (float *)p; p += al(sizeof(float) * nin);
  f->out_mean = (float *)p; p += al(sizeof(float) * nout);
  f->out_std = (float *)p;
  f->p = BeamParams{nn, c->EA, c->EI, c->rhoA, c->thickness, c->theta, c->lambda, c->rtol,
                    c->atol, c->dt, c->max_it, 0.0, c->solve_fp64 != 0};
  f->d = BeamDev{X, fx, u, v, F0, iters, nullptr, f->stats, Mb};
  f->F1 = F1;
  cudaError_t e = cudaMemcpyAsync(X, c->X, sizeof(double) * 2 * nn, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fx, c->fixed, sizeof(int32_t) * n, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, sizeof(double) * n, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(double) * n, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(F0, 0, sizeof(double) * n, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(iters, 0, sizeof(int), f->stream);
  if (e == cudaSuccess) {
    k_beam_mass<<<1, 128, 0, f->stream>>>(f->p, X, Mb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(f->hist, 0, sizeof(double) * 6 * nn, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->stats, 0, kFemStats * sizeof(int), f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) {
    snprintf(g_fem_msg, sizeof(g_fem_msg), "fem_beam_create: %s", cudaGetErrorString(e));
    if (f->own_ws) cudaFree(f->ws);
    delete f;
    return LBM_ECUDA;
  }
  *out = f;
  return LBM_OK;
}

#define FEM_CK(call)                                                             \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      f->poisoned = true;                                                        \
      snprintf(f->msg, sizeof(f->msg), "%s: %s", #call, cudaGetErrorString(e_)); \
      return LBM_ECUDA;                                                          \
    }                                                                            \
  } while (0)

lbm_status fem_beam_step(fem_ctx *f, const double *F1) {
  if (!f || !F1) return LBM_EINVAL;
  if (f->poisoned) return LBM_ESTATE;
  FEM_CK(cudaMemcpyAsync(f->F1, F1, sizeof(double) * 3 * f->p.nn, cudaMemcpyDefault, f->stream));
  FEM_CK(launch_beam_step<false>(f->p, f->d, f->F1, nullptr, nullptr, nullptr, 0, f->stream));
  return LBM_OK;
}

lbm_status fem_beam_get_state(fem_ctx *f, double *u, double *v, int *iterations) {
  if (!f) return LBM_EINVAL;
  if (f->poisoned) return LBM_ESTATE;
  const size_t n = 3 * (size_t)f->p.nn;
  if (u) FEM_CK(cudaMemcpyAsync(u, f->d.u, sizeof(double) * n, cudaMemcpyDefault, f->stream));
  if (v) FEM_CK(cudaMemcpyAsync(v, f->d.v, sizeof(double) * n, cudaMemcpyDefault, f->stream));
  if (iterations)
    FEM_CK(cudaMemcpyAsync(iterations, f->d.iters, sizeof(int), cudaMemcpyDefault, f->stream));
  FEM_CK(cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

lbm_status fem_beam_set_state(fem_ctx *f, const double *u, const double *v, const double *F0) {
  if (!f) return LBM_EINVAL;
  if (f->poisoned) return LBM_ESTATE;
  const size_t n = 3 * (size_t)f->p.nn;
  if (u) FEM_CK(cudaMemcpyAsync(f->d.u, u, sizeof(double) * n, cudaMemcpyDefault, f->stream));
  if (v) FEM_CK(cudaMemcpyAsync(f->d.v, v, sizeof(double) * n, cudaMemcpyDefault, f->stream));
  if (F0) FEM_CK(cudaMemcpyAsync(f->d.F0, F0, sizeof(double) * n, cudaMemcpyDefault, f->stream));
  FEM_CK(cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

const char *fem_last_error(const fem_ctx *f) { return f ? f->msg : g_fem_msg; }

void fem_destroy(fem_ctx *f) {
  if (!f) return;
  if (f->stream) cudaStreamSynchronize(f->stream);
  if (f->own_stream) cudaStreamDestroy(f->stream);
  if (f->own_ws) cudaFree(f->ws);
  delete f;
}

}  // extern "C"

namespace kbc {

int fem_nodes(const fem_ctx *f) { return f->p.nn; }

void fem_describe(const fem_ctx *f, BeamParams *p, BeamDev *d) {
  *p = f->p;
  *d = f->d;
}

// Coupled structural step on the lattice stream: loads from the surface
// forces of vertices [v0, v0 + 2 nn), then the new flag surface.
cudaError_t launch_beam_coupled(fem_ctx *f, const double *vforce, double *surf_x, double *surf_v,
                                int v0, cudaStream_t s) {
  return launch_beam_step<true>(f->p, f->d, nullptr, vforce, surf_x, surf_v, v0, s);
}

// Flag surface of the current beam state (used when coupling starts).
__global__ void k_flag_surface(BeamParams p, BeamDev d, double *surf_x, double *surf_v, int v0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.nn) return;
  store_flag_vertices(p, d.X, d.u, d.v, j, v0, surf_x, surf_v);
}

// Network input of the surrogate for step t: the out-of-balance loads
// F(t-k) - f(u) for k = 0, 1, 2 (F: nodal loads, the sums of each node's two
// surface-vertex forces; f: internal force at the state u before the step),
// then u and v, all on the free DOFs (the root node's three excluded);
// normalised with the training statistics.  One CTA.
__global__ void __launch_bounds__(128)
    k_surrogate_input(BeamParams p, BeamDev d, double *hist, const double *vforce, int v0,
                      const float *mean, const float *stdv, float *xin) {
  __shared__ double sX[2 * kMaxBeamNodes], su[3 * kMaxBeamNodes], sf[3 * kMaxBeamNodes];
  const int nn = p.nn, n = 3 * nn, ne = nn - 1, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) {
    su[i] = d.u[i];
    sf[i] = 0.0;
  }
  for (int i = tid; i < 2 * nn; i += nt) sX[i] = d.X[i];
  // ring slots 0 (t), 1 (t-1), 2 (t-2), each [nn][2]: shift, then store step t
  for (int k = tid; k < 2 * nn; k += nt) {
    const double h1 = hist[2 * nn + k], h0 = hist[k];
    hist[4 * nn + k] = h1;
    hist[2 * nn + k] = h0;
  }
  __syncthreads();
  for (int j = tid; j < nn; j += nt) {
    const int vb = v0 + j, vt = v0 + 2 * nn - 1 - j;
    hist[2 * j] = vforce[3 * vb] + vforce[3 * vt];
    hist[2 * j + 1] = vforce[3 * vb + 1] + vforce[3 * vt + 1];
  }
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = 2 * tid + pass; e < ne; e += 2 * nt) element_internal(p, sX, su, e, sf, nullptr);
    __syncthreads();
  }
  const int nf = n - 3, nin = 5 * nf;
  for (int k = tid; k < nin; k += nt) {
    const int blk = k / nf, i = 3 + k % nf;  // DOF index
    double val;
    if (blk < 3) {
      const int comp = i % 3;
      const double F = comp < 2 ? hist[2 * nn * blk + 2 * (i / 3) + comp] : 0.0;
      val = F - sf[i];
    } else if (blk == 3) {
      val = su[i];
    } else {
      val = d.v[i];
    }
    xin[k] = (float)((val - (double)mean[k]) / (double)stdv[k]);
  }
}

// Newton initial guess: the constant-velocity predictor u + dt v plus the
// network's correction to it (de-normalised), root node held.
__global__ void k_surrogate_guess(BeamParams p, BeamDev d, const float *yhat, const float *mean,
                                  const float *stdv, double *u_guess) {
  const int n = 3 * p.nn;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double g = d.u[i] + p.dt * d.v[i];
    if (i >= 3) g += (double)(yhat[i - 3] * stdv[i - 3] + mean[i - 3]);
    u_guess[i] = d.fixed[i] ? 0.0 : g;
  }
}

cudaError_t launch_surrogate_input(fem_ctx *f, const double *vforce, int v0, float *xin,
                                   cudaStream_t s) {
  k_surrogate_input<<<1, 128, 0, s>>>(f->p, f->d, f->hist, vforce, v0, f->in_mean, f->in_std, xin);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_guess(fem_ctx *f, const float *yhat, cudaStream_t s) {
  k_surrogate_guess<<<1, 128, 0, s>>>(f->p, f->d, yhat, f->out_mean, f->out_std, f->u_guess);
  return cudaGetLastError();
}

// Coupled step with the surrogate guess: the beam kernel first checks it.
cudaError_t launch_beam_coupled_guess(fem_ctx *f, const double *vforce, double *surf_x,
                                      double *surf_v, int v0, double accept_tol, cudaStream_t s) {
  BeamParams p = f->p;
  p.accept_tol = accept_tol;
  BeamDev d = f->d;
  d.u_guess = f->u_guess;
  return launch_beam_step<true>(p, d, nullptr, vforce, surf_x, surf_v, v0, s);
}

lbm_status fem_set_normalisation(fem_ctx *f, const float *in_mean, const float *in_std,
                                 const float *out_mean, const float *out_std) {
  const size_t nin = surrogate_inputs(f->p.nn), nout = 3 * (size_t)f->p.nn - 3;
  cudaError_t e = cudaMemcpyAsync(f->in_mean, in_mean, sizeof(float) * nin, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->in_std, in_std, sizeof(float) * nin, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->out_mean, out_mean, sizeof(float) * nout, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->out_std, out_std, sizeof(float) * nout, cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->stats, 0, kFemStats * sizeof(int), f->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->hist, 0, sizeof(double) * 6 * f->p.nn, f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

lbm_status fem_reset_stats(fem_ctx *f) {
  cudaError_t e = cudaMemsetAsync(f->stats, 0, kFemStats * sizeof(int), f->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

lbm_status fem_get_stats(fem_ctx *f, int *stats) {
  cudaError_t e = cudaMemcpyAsync(stats, f->stats, kFemStats * sizeof(int), cudaMemcpyDefault, f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

void fem_set_span(fem_ctx *f, int span, int v1, double z0, double z1, double inv_depth) {
  f->p.span = span;
  f->p.v1 = v1;
  f->p.z0 = z0;
  f->p.z1 = z1;
  f->p.inv_depth = inv_depth;
}

int fem_span(const fem_ctx *f) { return f->p.span; }

cudaError_t launch_flag_surface(fem_ctx *f, double *surf_x, double *surf_v, int v0,
                                cudaStream_t s) {
  k_flag_surface<<<1, 64, 0, s>>>(f->p, f->d, surf_x, surf_v, v0);
  return cudaGetLastError();
}

}  // namespace kbc
