// fem_svk.cu -- the paper's structural model on the GPU (FP64): the
// total-Lagrangian St Venant-Kirchhoff continuum of section "Structural
// modeling" with Q2 Lagrange elements (9-node quadrilaterals in plane
// strain, 27-node hexahedra), the element geometry mapped from its corner
// nodes by the bilinear (trilinear) map, 3 Gauss points per axis.
//   S = lambda tr(E) I + 2 mu E, E = (F^T F - I) / 2, P = F S;
//   consistent mass (rho psi, psi);
//   the two-field theta scheme (Eq. timeInt) with the displacement equation
//   solved exactly (u1 - u0 = dt (theta v1 + (1 - theta) v0)), so Newton runs
//   on u1: G(u) = M (u - u0 - dt v0) / (theta dt^2) + theta R(u) - theta F1 -
//   (1 - theta) (F0 - R(u0)), tangent M / (theta dt^2) + theta A'(u) with the
//   analytic Gateaux derivative printed after Eq. (matrixForm2), steps
//   relaxed by lambda; stop at |G| <= rtol |G_0| + atol.
// Every linearised system is solved by Jacobi-preconditioned conjugate
// gradients on element products (no assembled matrix).  One cooperative
// launch runs the whole step: one warp per element (grid-stride), lanes on
// Gauss points for the stresses, then on element nodes for the nodal sums,
// FP64 atomics into the global vectors, grid-wide barriers between phases.
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

// CTA size of the cooperative grid (one warp per element).  (One CTA of 512
// threads running the CSM3 flag alone, with block barriers, measured 254 ms
// per step against 97 ms on the grid: latency-bound on one SM.)
constexpr int kSvkThreads = 128;

struct SvkParams {
  int dim, nn, ne, n;
  double mu, lmb, rho;
  double theta, lambda, rtol, atol, dt;
  int max_it, max_cg;
  double cg_rtol;
};

struct SvkDev {
  const int32_t *conn;   // [ne][nen]
  const int32_t *fixed;  // [n]
  const double *wdet;    // [ne][ng] Gauss weight x det J
  const double *dNX;     // [ne][ng][nen][dim] reference-frame gradients
  const double *Ntab;    // [ng][nen] shape-function values
  double *u, *v, *F0, *F1;
  double *u0, *v0, *rhs0, *f, *Mq, *diag;
  double *x, *r, *z, *p, *Ap;
  double *Fg, *Sg;       // [ne][ng][dim^2] F and S of the current iterate
  // FP32 copies for the FP32 element products inside CG
  const float *dNXf, *wdetf, *Ntabf;
  float *Fgf, *Sgf;
  double *red;           // 6 reduction slots
  int *iters;            // [2] Newton iterations (negative: not converged), CG total
};

template <int D>
struct SvkEl {
  static constexpr int nen = D == 2 ? 9 : 27;
  static constexpr int ng = nen;
  static constexpr int DD = D * D;
};

// per-warp scratch
template <int D>
struct SvkWarp {
  double gp[SvkEl<D>::ng][SvkEl<D>::DD];  // w P (or the tangent's Q) per Gauss point
  double gm[SvkEl<D>::ng][D];             // mass term per Gauss point
  double a[SvkEl<D>::nen][D];             // element nodal vector
  double b[SvkEl<D>::nen][D];             // second element nodal vector
  int node[SvkEl<D>::nen];
  // FP32 scratch of the FP32 tangent products (no conversions in the loops)
  float gpf[SvkEl<D>::ng][SvkEl<D>::DD];
  float gmf[SvkEl<D>::ng][D];
  float af[SvkEl<D>::nen][D];
};

// The warp scratch in precision T
template <int D, typename T>
struct SvkScr;
template <int D>
struct SvkScr<D, double> {
  double (*gp)[SvkEl<D>::DD];
  double (*gm)[D];
  double (*a)[D];
  __device__ SvkScr(SvkWarp<D> &W) : gp(W.gp), gm(W.gm), a(W.a) {}
};
template <int D>
struct SvkScr<D, float> {
  float (*gp)[SvkEl<D>::DD];
  float (*gm)[D];
  float (*a)[D];
  __device__ SvkScr(SvkWarp<D> &W) : gp(W.gpf), gm(W.gmf), a(W.af) {}
};

// S of a deformation gradient (row-major D x D)
template <int D>
__device__ __forceinline__ void svk_S(const SvkParams &P, const double (&F)[D][D], double (&S)[D][D]) {
  double E[D][D];
  double tr = 0.0;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
      for (int k = 0; k < D; ++k) s += F[k][i] * F[k][j];
      E[i][j] = 0.5 * (s - (i == j ? 1.0 : 0.0));
    }
  for (int i = 0; i < D; ++i) tr += E[i][i];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) S[i][j] = 2.0 * P.mu * E[i][j] + (i == j ? P.lmb * tr : 0.0);
}

// Element e, force (+ mass) pass: f += R_e(u), and with q != null Mq +=
// M_e (u - u0 - dt v0); F and S of each Gauss point stored for the tangent.
template <int D>
__device__ void svk_force(const SvkParams &P, const SvkDev &V, int e, const double *u,
                          double *f, bool with_mass, SvkWarp<D> &W, int lane) {
  constexpr int nen = SvkEl<D>::nen, ng = SvkEl<D>::ng, DD = SvkEl<D>::DD;
  if (lane < nen) {
    const int nd = V.conn[(long long)e * nen + lane];
    W.node[lane] = nd;
    for (int d = 0; d < D; ++d) {
      W.a[lane][d] = u[(long long)nd * D + d];
      if (with_mass)
        W.b[lane][d] = u[(long long)nd * D + d] - V.u0[(long long)nd * D + d] -
                       P.dt * V.v0[(long long)nd * D + d];
    }
  }
  __syncwarp();
  if (lane < ng) {
    const double *dN = V.dNX + ((long long)e * ng + lane) * nen * D;
    double F[D][D];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) F[i][j] = (i == j) ? 1.0 : 0.0;
    for (int a = 0; a < nen; ++a)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F[i][j] += W.a[a][i] * dN[a * D + j];
    double S[D][D];
    svk_S<D>(P, F, S);
    const double w = V.wdet[(long long)e * ng + lane];
    const long long go = ((long long)e * ng + lane) * DD;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        V.Fg[go + i * D + j] = F[i][j];
        V.Sg[go + i * D + j] = S[i][j];
        V.Fgf[go + i * D + j] = (float)F[i][j];
        V.Sgf[go + i * D + j] = (float)S[i][j];
        double pij = 0.0;
        for (int k = 0; k < D; ++k) pij += F[i][k] * S[k][j];
        W.gp[lane][i * D + j] = w * pij;
      }
    if (with_mass) {
      const double *N = V.Ntab + (long long)lane * nen;
      for (int i = 0; i < D; ++i) {
        double s = 0.0;
        for (int b = 0; b < nen; ++b) s += N[b] * W.b[b][i];
        W.gm[lane][i] = P.rho * w * s;
      }
    }
  }
  __syncwarp();
  if (lane < nen) {
    for (int i = 0; i < D; ++i) {
      double s = 0.0, m = 0.0;
      for (int g = 0; g < ng; ++g) {
        const double *dN = V.dNX + (((long long)e * ng + g) * nen + lane) * D;
        for (int j = 0; j < D; ++j) s += W.gp[g][i * D + j] * dN[j];
        if (with_mass) m += V.Ntab[(long long)g * nen + lane] * W.gm[g][i];
      }
      atomicAdd(f + (long long)W.node[lane] * D + i, s);
      if (with_mass) atomicAdd(V.Mq + (long long)W.node[lane] * D + i, m);
    }
  }
  __syncwarp();
}

// Tables of the element products in precision T
template <typename T>
struct SvkTab;
template <>
struct SvkTab<double> {
  const double *dN, *w, *N, *F, *S;
  __device__ SvkTab(const SvkDev &V) : dN(V.dNX), w(V.wdet), N(V.Ntab), F(V.Fg), S(V.Sg) {}
};
template <>
struct SvkTab<float> {
  const float *dN, *w, *N, *F, *S;
  __device__ SvkTab(const SvkDev &V) : dN(V.dNXf), w(V.wdetf), N(V.Ntabf), F(V.Fgf), S(V.Sgf) {}
};

// Element e, tangent product: y += (cM M_e + theta A'_e(u)) p, p = z + beta
// p_prev formed here (the CG search direction before it is stored), with the
// stored F, S: the printed Gateaux form (grad p S + F (mu (grad p^T F + F^T
// grad p) + lambda tr(F^T grad p) I), grad psi).
template <int D, typename T>
__device__ void svk_tangent(const SvkParams &P, const SvkDev &V, int e, const double *z,
                            const double *p, double beta, double *y, double cM, SvkWarp<D> &W,
                            int lane) {
  const SvkTab<T> tb(V);
  const SvkScr<D, T> sc(W);
  constexpr int nen = SvkEl<D>::nen, ng = SvkEl<D>::ng, DD = SvkEl<D>::DD;
  if (lane < nen) {
    const int nd = V.conn[(long long)e * nen + lane];
    W.node[lane] = nd;
    for (int d = 0; d < D; ++d) {
      const long long k = (long long)nd * D + d;
      sc.a[lane][d] = (T)__fma_rn(beta, p[k], z[k]);
    }
  }
  __syncwarp();
  if (lane < ng) {
    const T *dN = tb.dN + ((long long)e * ng + lane) * nen * D;
    const T *Fi = tb.F + ((long long)e * ng + lane) * DD, *Si = tb.S + ((long long)e * ng + lane) * DD;
    T dH[D][D], F[D][D], S[D][D];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        dH[i][j] = (T)0;
        F[i][j] = Fi[i * D + j];
        S[i][j] = Si[i * D + j];
      }
    for (int a = 0; a < nen; ++a)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) dH[i][j] += sc.a[a][i] * dN[a * D + j];
    T FtdH[D][D], tr = (T)0;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        T s = (T)0;
        for (int k = 0; k < D; ++k) s += F[k][i] * dH[k][j];
        FtdH[i][j] = s;
      }
    for (int i = 0; i < D; ++i) tr += FtdH[i][i];
    T inner[D][D];
    const T mu = (T)P.mu, lmb = (T)P.lmb;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        inner[i][j] = mu * (FtdH[j][i] + FtdH[i][j]) + (i == j ? lmb * tr : (T)0);
    const T w = tb.w[(long long)e * ng + lane];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        T q = (T)0;
        for (int k = 0; k < D; ++k) q += dH[i][k] * S[k][j] + F[i][k] * inner[k][j];
        sc.gp[lane][i * D + j] = (T)P.theta * w * q;
      }
    const T *N = tb.N + (long long)lane * nen;
    for (int i = 0; i < D; ++i) {
      T s = (T)0;
      for (int b = 0; b < nen; ++b) s += N[b] * sc.a[b][i];
      sc.gm[lane][i] = (T)(cM * P.rho) * w * s;
    }
  }
  __syncwarp();
  if (lane < nen) {
    for (int i = 0; i < D; ++i) {
      T s = (T)0;
      for (int g = 0; g < ng; ++g) {
        const T *dN = tb.dN + (((long long)e * ng + g) * nen + lane) * D;
        for (int j = 0; j < D; ++j) s += sc.gp[g][i * D + j] * dN[j];
        s += tb.N[(long long)g * nen + lane] * sc.gm[g][i];
      }
      atomicAdd(y + (long long)W.node[lane] * D + i, (double)s);
    }
  }
  __syncwarp();
}

// Element e, Jacobi diagonal: diag += the diagonal of cM M_e + theta A'_e(u)
// (the Gateaux form for p = psi = e_i N_a: grad N_a . S grad N_a + mu ((F
// grad N_a)_i^2 + (F F^T)_ii |grad N_a|^2) + lambda (F grad N_a)_i^2).
template <int D, typename T>
__device__ void svk_diag(const SvkParams &P, const SvkDev &V, int e, double cM, int lane) {
  constexpr int nen = SvkEl<D>::nen, ng = SvkEl<D>::ng, DD = SvkEl<D>::DD;
  if (lane >= nen) return;
  const SvkTab<T> tb(V);
  const T th = (T)P.theta, mu = (T)P.mu, lmb = (T)P.lmb, cMr = (T)(cM * P.rho);
  const int nd = V.conn[(long long)e * nen + lane];
  T acc[D];
  for (int i = 0; i < D; ++i) acc[i] = (T)0;
  for (int g = 0; g < ng; ++g) {
    const T *dN = tb.dN + (((long long)e * ng + g) * nen + lane) * D;
    const T *F = tb.F + ((long long)e * ng + g) * DD, *S = tb.S + ((long long)e * ng + g) * DD;
    const T w = tb.w[(long long)e * ng + g], Na = tb.N[(long long)g * nen + lane];
    T gv[D], nSn = (T)0, nn = (T)0;
    for (int i = 0; i < D; ++i) {
      T s = (T)0, t = (T)0;
      for (int j = 0; j < D; ++j) {
        s += F[i * D + j] * dN[j];
        t += S[i * D + j] * dN[j];
      }
      gv[i] = s;
      nSn += dN[i] * t;
      nn += dN[i] * dN[i];
    }
    for (int i = 0; i < D; ++i) {
      T ffii = (T)0;
      for (int k = 0; k < D; ++k) ffii += F[i * D + k] * F[i * D + k];
      acc[i] += w * (th * (nSn + mu * (gv[i] * gv[i] + ffii * nn) + lmb * gv[i] * gv[i]) +
                     cMr * Na * Na);
    }
  }
  for (int i = 0; i < D; ++i) atomicAdd(V.diag + (long long)nd * D + i, (double)acc[i]);
}

__device__ __forceinline__ void svk_sync() { cg::this_grid().sync(); }

// Sums of two values over the grid: block reduction, one atomic per block
// into slot s, barrier, read; the slot two ahead is cleared for later use.
template <int THREADS>
__device__ __forceinline__ void svk_sum2(double *red, int &slot, double a, double b, double &ra,
                                         double &rb) {
  constexpr int kSvkWarps = THREADS / 32;
  __shared__ double part[2][kSvkWarps];
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
    for (int k = 0; k < kSvkWarps; ++k) {
      sa += part[0][k];
      sb += part[1][k];
    }
    atomicAdd(red + 2 * slot, sa);
    atomicAdd(red + 2 * slot + 1, sb);
  }
  svk_sync();
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

// One theta step.  Barriers per Newton iteration: element forces and mass
// (1), the residual norm (1), the Jacobi diagonal (1), per CG iteration the
// tangent products and two reductions (3; the search direction p = z + beta
// p_prev is formed where it is read, the same FMA at every site, and stored
// by the update), the relaxed update (1).
template <int D, typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_svk_step(SvkParams P, SvkDev V) {
  constexpr int kSvkWarps = THREADS / 32;
  __shared__ SvkWarp<D> Wsh[kSvkWarps];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  SvkWarp<D> &W = Wsh[wl];
  const int wg = blockIdx.x * kSvkWarps + wl, nwg = gridDim.x * kSvkWarps;
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const int n = P.n;
  const double th = P.theta, cM = 1.0 / (th * P.dt * P.dt);
  int slot = 0;
  double ra, rb;
  for (long long i = gt; i < n; i += gs) {
    V.u0[i] = V.u[i];
    V.v0[i] = V.v[i];
    V.f[i] = 0.0;
  }
  if (gt < 6) V.red[gt] = 0.0;
  svk_sync();
  for (int e = wg; e < P.ne; e += nwg) svk_force<D>(P, V, e, V.u0, V.f, false, W, lane);
  svk_sync();
  for (long long i = gt; i < n; i += gs) {
    V.rhs0[i] = th * V.F1[i] + (1.0 - th) * (V.F0[i] - V.f[i]);
    V.u[i] = V.fixed[i] ? V.u0[i] : V.u0[i] + P.dt * V.v0[i];
    V.f[i] = 0.0;
    V.Mq[i] = 0.0;
    V.diag[i] = 0.0;
  }
  svk_sync();
  double g0 = -1.0;
  int it = 0, cg_total = 0;
  bool conv = false;
  for (it = 0;; ++it) {
    for (int e = wg; e < P.ne; e += nwg) svk_force<D>(P, V, e, V.u, V.f, true, W, lane);
    svk_sync();
    double gg = 0.0;
    for (long long i = gt; i < n; i += gs) {
      const double G = V.fixed[i] ? 0.0 : cM * V.Mq[i] + th * V.f[i] - V.rhs0[i];
      V.r[i] = -G;
      V.x[i] = 0.0;
      gg += G * G;
    }
    svk_sum2<THREADS>(V.red, slot, gg, 0.0, ra, rb);
    const double gn = sqrt(ra);
    if (g0 < 0.0) g0 = gn;
    if (gn <= P.rtol * g0 + P.atol) {
      conv = true;
      break;
    }
    if (it >= P.max_it) break;
    for (int e = wg; e < P.ne; e += nwg) svk_diag<D, T>(P, V, e, cM, lane);
    svk_sync();
    double rz = 0.0;
    for (long long i = gt; i < n; i += gs) {
      const double z = V.fixed[i] ? 0.0 : V.r[i] / V.diag[i];
      V.z[i] = z;
      V.p[i] = 0.0;
      V.Ap[i] = 0.0;
      rz += V.r[i] * z;
    }
    svk_sum2<THREADS>(V.red, slot, rz, 0.0, ra, rb);
    rz = ra;
    double beta = 0.0;
    int k = 0;
    while (k < P.max_cg) {
      for (int e = wg; e < P.ne; e += nwg)
        svk_tangent<D, T>(P, V, e, V.z, V.p, beta, V.Ap, cM, W, lane);
      svk_sync();
      double pAp = 0.0;
      for (long long i = gt; i < n; i += gs)
        if (!V.fixed[i]) pAp += __fma_rn(beta, V.p[i], V.z[i]) * V.Ap[i];
      svk_sum2<THREADS>(V.red, slot, pAp, 0.0, ra, rb);
      ++k;
      if (!(ra > 0.0)) break;
      const double alpha = rz / ra;
      double rzn = 0.0, rr = 0.0;
      for (long long i = gt; i < n; i += gs) {
        if (V.fixed[i]) continue;
        const double pk = __fma_rn(beta, V.p[i], V.z[i]);
        V.p[i] = pk;
        V.x[i] += alpha * pk;
        const double r = V.r[i] - alpha * V.Ap[i];
        const double z = r / V.diag[i];
        V.Ap[i] = 0.0;
        V.r[i] = r;
        V.z[i] = z;
        rzn += r * z;
        rr += r * r;
      }
      svk_sum2<THREADS>(V.red, slot, rzn, rr, ra, rb);
      if (sqrt(rb) <= P.cg_rtol * gn) break;
      beta = ra / rz;
      rz = ra;
    }
    cg_total += k;
    for (long long i = gt; i < n; i += gs) {
      if (!V.fixed[i]) V.u[i] += P.lambda * V.x[i];
      V.f[i] = 0.0;
      V.Mq[i] = 0.0;
      V.diag[i] = 0.0;
    }
    svk_sync();
  }
  for (long long i = gt; i < n; i += gs) {
    V.v[i] = V.fixed[i] ? 0.0 : (V.u[i] - V.u0[i]) / (th * P.dt) - (1.0 - th) / th * V.v0[i];
    V.F0[i] = V.F1[i];
  }
  if (gt == 0) {
    V.iters[0] = conv ? it : -(it + 1);
    V.iters[1] = cg_total;
  }
}

// Consistent loads of a uniform body force b per unit mass: F += (rho b, psi_a).
template <int D>
__global__ void k_svk_body(SvkParams P, SvkDev V, double b0, double b1, double b2, double *F) {
  constexpr int nen = SvkEl<D>::nen, ng = SvkEl<D>::ng;
  const int lane = threadIdx.x & 31;
  const int e = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (e >= P.ne || lane >= nen) return;
  const double b[3] = {b0, b1, b2};
  double s = 0.0;
  for (int g = 0; g < ng; ++g) s += V.wdet[(long long)e * ng + g] * V.Ntab[(long long)g * nen + lane];
  const int nd = V.conn[(long long)e * nen + lane];
  for (int i = 0; i < D; ++i) atomicAdd(F + (long long)nd * D + i, P.rho * s * b[i]);
}

}  // namespace kbc

using namespace kbc;

struct fem_svk_ctx {
  SvkParams p;
  SvkDev d;
  char *ws = nullptr;
  bool own_ws = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int grid = 0;
  const void *fn = nullptr;  // the step kernel (dimension, precision of the CG products, CTA size)
  int threads = 0;
  bool poisoned = false;
  char msg[256] = {0};
};

namespace {

thread_local char g_svk_msg[256];

size_t svk_al(size_t b) { return (b + 255) / 256 * 256; }

int svk_nen(int dim) { return dim == 2 ? 9 : 27; }

size_t svk_layout(int dim, int nn, int ne, fem_svk_ctx *s) {
  const size_t nen = svk_nen(dim), ng = nen, n = (size_t)nn * dim, dd = (size_t)dim * dim;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += svk_al(bytes);
    return o;
  };
  const size_t oconn = take(sizeof(int32_t) * nen * ne), ofix = take(sizeof(int32_t) * n);
  const size_t ow = take(sizeof(double) * ng * ne), odN = take(sizeof(double) * ng * nen * dim * ne);
  const size_t oN = take(sizeof(double) * ng * nen);
  size_t ovec[16];
  for (int k = 0; k < 16; ++k) ovec[k] = take(sizeof(double) * n);
  const size_t oFg = take(sizeof(double) * dd * ng * ne), oSg = take(sizeof(double) * dd * ng * ne);
  const size_t ored = take(sizeof(double) * 6), oit = take(sizeof(int) * 2);
  const size_t odNf = take(sizeof(float) * ng * nen * dim * ne), owf = take(sizeof(float) * ng * ne);
  const size_t oNf = take(sizeof(float) * ng * nen);
  const size_t oFgf = take(sizeof(float) * dd * ng * ne), oSgf = take(sizeof(float) * dd * ng * ne);
  if (s) {
    char *w = s->ws;
    SvkDev &d = s->d;
    d.conn = (const int32_t *)(w + oconn);
    d.fixed = (const int32_t *)(w + ofix);
    d.wdet = (const double *)(w + ow);
    d.dNX = (const double *)(w + odN);
    d.Ntab = (const double *)(w + oN);
    double **v[16] = {&d.u, &d.v, &d.F0, &d.F1, &d.u0, &d.v0, &d.rhs0, &d.f,
                      &d.Mq, &d.diag, &d.x, &d.r, &d.z, &d.p, &d.Ap, nullptr};
    for (int k = 0; k < 15; ++k) *v[k] = (double *)(w + ovec[k]);
    d.Fg = (double *)(w + oFg);
    d.Sg = (double *)(w + oSg);
    d.red = (double *)(w + ored);
    d.iters = (int *)(w + oit);
    d.dNXf = (const float *)(w + odNf);
    d.wdetf = (const float *)(w + owf);
    d.Ntabf = (const float *)(w + oNf);
    d.Fgf = (float *)(w + oFgf);
    d.Sgf = (float *)(w + oSgf);
  }
  return off;
}

const char *svk_validate(const fem_svk_config *c) {
  if (!c) return "config is NULL";
  if (c->dim != 2 && c->dim != 3) return "dim must be 2 or 3";
  if (c->nn < 1 || c->ne < 1) return "nn and ne must be >= 1";
  if ((long long)c->nn * c->dim > (1LL << 30)) return "too many DOFs";
  if (!c->X || !c->conn || !c->fixed) return "X, conn and fixed are required";
  if (!(c->E > 0 && c->rho > 0 && c->nu >= 0 && c->nu < 0.5)) return "E, rho > 0 and 0 <= nu < 0.5";
  if (!(c->theta > 0 && c->theta <= 1) || !(c->lambda > 0 && c->lambda <= 1) || c->max_it < 1 ||
      !(c->dt > 0) || !(c->rtol >= 0) || !(c->atol >= 0))
    return "bad time-integration parameters";
  return nullptr;
}

// Reference element: Gauss points and nodes in x-fastest order (index i + 3
// j + 9 k), corners c = i + 2 j + 4 k.  w[g], N[g][a], dN[g][a][d] (Q2),
// dL[g][c][d] (the corner map), corner[c] = local node of corner c.
struct SvkRef {
  std::vector<double> w, N, dN, dL;
  int corner[8];
};
SvkRef svk_reference(int dim) {
  const int nen = svk_nen(dim), nc = 1 << dim;
  const double gx[3] = {-sqrt(0.6), 0.0, sqrt(0.6)}, gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  SvkRef R;
  R.w.assign(nen, 1.0);
  R.N.assign((size_t)nen * nen, 1.0);
  R.dN.assign((size_t)nen * nen * dim, 1.0);
  R.dL.assign((size_t)nen * nc * dim, 1.0);
  auto digit = [](int idx, int d, int base) {
    for (int k = 0; k < d; ++k) idx /= base;
    return idx % base;
  };
  for (int g = 0; g < nen; ++g) {
    double xi[3];
    for (int d = 0; d < dim; ++d) {
      xi[d] = gx[digit(g, d, 3)];
      R.w[g] *= gw[digit(g, d, 3)];
    }
    for (int a = 0; a < nen; ++a) {
      double q[3], dq[3];
      for (int d = 0; d < dim; ++d) {
        const double x = xi[d];
        const int m = digit(a, d, 3);
        q[d] = m == 0 ? 0.5 * x * (x - 1.0) : (m == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
        dq[d] = m == 0 ? x - 0.5 : (m == 1 ? -2.0 * x : x + 0.5);
      }
      double prod = 1.0;
      for (int d = 0; d < dim; ++d) prod *= q[d];
      R.N[(size_t)g * nen + a] = prod;
      for (int d = 0; d < dim; ++d) {
        double t = 1.0;
        for (int e = 0; e < dim; ++e) t *= (e == d) ? dq[e] : q[e];
        R.dN[((size_t)g * nen + a) * dim + d] = t;
      }
    }
    for (int c = 0; c < nc; ++c) {
      double l[3], dl[3];
      for (int d = 0; d < dim; ++d) {
        const int m = (c >> d) & 1;
        l[d] = m ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d]);
        dl[d] = m ? 0.5 : -0.5;
      }
      for (int d = 0; d < dim; ++d) {
        double t = 1.0;
        for (int e = 0; e < dim; ++e) t *= (e == d) ? dl[e] : l[e];
        R.dL[((size_t)g * nc + c) * dim + d] = t;
      }
    }
  }
  for (int c = 0; c < nc; ++c) {
    int a = 0, s = 1;
    for (int d = 0; d < dim; ++d, s *= 3) a += 2 * ((c >> d) & 1) * s;
    R.corner[c] = a;
  }
  return R;
}

// Per element and Gauss point: w det J and the reference-frame gradients of
// the shape functions (J from the corner map).  False for det J <= 0.
bool svk_geometry(int dim, int ne, const std::vector<double> &X, const std::vector<int32_t> &conn,
                  const SvkRef &R, std::vector<double> &wdet, std::vector<double> &dNX) {
  const int nen = svk_nen(dim), ng = nen, nc = 1 << dim;
  wdet.assign((size_t)ne * ng, 0.0);
  dNX.assign((size_t)ne * ng * nen * dim, 0.0);
  for (int e = 0; e < ne; ++e) {
    for (int g = 0; g < ng; ++g) {
      double J[3][3] = {{0}}, Ji[3][3] = {{0}};
      for (int c = 0; c < nc; ++c) {
        const int nd = conn[(size_t)e * nen + R.corner[c]];
        for (int d = 0; d < dim; ++d)
          for (int f = 0; f < dim; ++f)
            J[d][f] += X[(size_t)nd * dim + d] * R.dL[((size_t)g * nc + c) * dim + f];
      }
      double det;
      if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
      } else {
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        Ji[0][0] = c00 / det;
        Ji[1][0] = c01 / det;
        Ji[2][0] = c02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      }
      if (!(det > 0)) return false;
      wdet[(size_t)e * ng + g] = R.w[g] * det;
      for (int a = 0; a < nen; ++a)
        for (int d = 0; d < dim; ++d) {
          double s = 0.0;
          for (int f = 0; f < dim; ++f) s += R.dN[((size_t)g * nen + a) * dim + f] * Ji[f][d];
          dNX[(((size_t)e * ng + g) * nen + a) * dim + d] = s;
        }
    }
  }
  return true;
}

}  // namespace

#define SVK_CK(call)                                                                \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      s->poisoned = true;                                                           \
      snprintf(s->msg, sizeof(s->msg), "%s: %s", #call, cudaGetErrorString(e_));    \
      return LBM_ECUDA;                                                             \
    }                                                                               \
  } while (0)

static cudaError_t svk_launch(fem_svk_ctx *s) {
  void *args[] = {(void *)&s->p, (void *)&s->d};
  return cudaLaunchCooperativeKernel(s->fn, dim3(s->grid), dim3(s->threads), args, 0, s->stream);
}

// The step kernel for a dimension and CG-product precision.
static const void *svk_kernel(int dim, bool fp64) {
  if (dim == 2)
    return fp64 ? (const void *)k_svk_step<2, double, kSvkThreads>
                : (const void *)k_svk_step<2, float, kSvkThreads>;
  return fp64 ? (const void *)k_svk_step<3, double, kSvkThreads>
              : (const void *)k_svk_step<3, float, kSvkThreads>;
}

extern "C" {

lbm_status fem_svk_workspace_size(const fem_svk_config *c, size_t *bytes) {
  if (!bytes || svk_validate(c)) return LBM_EINVAL;
  *bytes = svk_layout(c->dim, c->nn, c->ne, nullptr);
  return LBM_OK;
}

lbm_status fem_svk_create(const fem_svk_config *c, void *workspace, size_t bytes,
                          fem_svk_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (const char *why = svk_validate(c)) {
    snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: %s", why);
    return LBM_EINVAL;
  }
  const int dim = c->dim, nen = svk_nen(dim), nn = c->nn, ne = c->ne, n = nn * dim;
  // host copies of the mesh (the inputs may be device memory)
  std::vector<double> X((size_t)nn * dim);
  std::vector<int32_t> conn((size_t)ne * nen), fixed(n);
  if (cudaMemcpy(X.data(), c->X, sizeof(double) * X.size(), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(conn.data(), c->conn, sizeof(int32_t) * conn.size(), cudaMemcpyDefault) !=
          cudaSuccess ||
      cudaMemcpy(fixed.data(), c->fixed, sizeof(int32_t) * n, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: cannot read X, conn or fixed");
    return LBM_EINVAL;
  }
  for (int32_t k : conn)
    if (k < 0 || k >= nn) {
      snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: element node out of range");
      return LBM_EINVAL;
    }
  const SvkRef R = svk_reference(dim);
  std::vector<double> wdet, dNX;
  if (!svk_geometry(dim, ne, X, conn, R, wdet, dNX)) {
    snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: an element has det J <= 0");
    return LBM_EINVAL;
  }
  fem_svk_ctx *s = new (std::nothrow) fem_svk_ctx();
  if (!s) return LBM_ENOMEM;
  const size_t need = svk_layout(dim, nn, ne, nullptr);
  if (workspace) {
    if (bytes < need || ((uintptr_t)workspace % 256)) {
      delete s;
      snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: workspace needs %zu bytes", need);
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
  svk_layout(dim, nn, ne, s);
  SvkParams &p = s->p;
  p.dim = dim; p.nn = nn; p.ne = ne; p.n = n;
  p.mu = c->E / (2.0 * (1.0 + c->nu));
  p.lmb = c->E * c->nu / ((1.0 + c->nu) * (1.0 - 2.0 * c->nu));
  p.rho = c->rho;
  p.theta = c->theta; p.lambda = c->lambda; p.rtol = c->rtol; p.atol = c->atol; p.dt = c->dt;
  p.max_it = c->max_it;
  p.max_cg = c->max_cg > 0 ? c->max_cg : n;
  p.cg_rtol = c->cg_rtol > 0 ? c->cg_rtol : 1e-3;
  cudaError_t e = cudaMemsetAsync(s->ws, 0, need, s->stream);
  auto up = [&](const void *dst, const void *src, size_t b) {
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)dst, src, b, cudaMemcpyHostToDevice, s->stream);
  };
  up(s->d.conn, conn.data(), sizeof(int32_t) * conn.size());
  up(s->d.fixed, fixed.data(), sizeof(int32_t) * n);
  up(s->d.wdet, wdet.data(), sizeof(double) * wdet.size());
  up(s->d.dNX, dNX.data(), sizeof(double) * dNX.size());
  up(s->d.Ntab, R.N.data(), sizeof(double) * R.N.size());
  const std::vector<float> dNf(dNX.begin(), dNX.end()), wf(wdet.begin(), wdet.end()),
      Nf(R.N.begin(), R.N.end());
  up(s->d.dNXf, dNf.data(), sizeof(float) * dNf.size());
  up(s->d.wdetf, wf.data(), sizeof(float) * wf.size());
  up(s->d.Ntabf, Nf.data(), sizeof(float) * Nf.size());
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  s->fn = svk_kernel(dim, c->solve_fp64 != 0);
  s->threads = kSvkThreads;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->fn, s->threads, 0);
  if (e != cudaSuccess || !coop || per_sm < 1) {
    snprintf(g_svk_msg, sizeof(g_svk_msg), "fem_svk_create: %s",
             e != cudaSuccess ? cudaGetErrorString(e) : "cooperative launch unavailable");
    if (s->own_ws) cudaFree(s->ws);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return LBM_ECUDA;
  }
  s->grid = (ne + kSvkThreads / 32 - 1) / (kSvkThreads / 32);
  if (s->grid > sms * per_sm) s->grid = sms * per_sm;
  *out = s;
  return LBM_OK;
}

lbm_status fem_svk_step(fem_svk_ctx *s, const double *F1) {
  if (!s || !F1) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  SVK_CK(cudaMemcpyAsync(s->d.F1, F1, sizeof(double) * s->p.n, cudaMemcpyDefault, s->stream));
  SVK_CK(svk_launch(s));
  return LBM_OK;
}

lbm_status fem_svk_body_load(fem_svk_ctx *s, const double *b, double *F) {
  if (!s || !b || !F) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  double bh[3] = {0.0, 0.0, 0.0};
  SVK_CK(cudaMemcpy(bh, b, sizeof(double) * s->p.dim, cudaMemcpyDefault));
  // accumulate in the CG scratch x (unused between steps), then copy out
  SVK_CK(cudaMemsetAsync(s->d.x, 0, sizeof(double) * s->p.n, s->stream));
  const unsigned blocks = (unsigned)(((long long)s->p.ne * 32 + 127) / 128);
  if (s->p.dim == 2)
    k_svk_body<2><<<blocks, 128, 0, s->stream>>>(s->p, s->d, bh[0], bh[1], bh[2], s->d.x);
  else
    k_svk_body<3><<<blocks, 128, 0, s->stream>>>(s->p, s->d, bh[0], bh[1], bh[2], s->d.x);
  SVK_CK(cudaGetLastError());
  SVK_CK(cudaMemcpyAsync(F, s->d.x, sizeof(double) * s->p.n, cudaMemcpyDefault, s->stream));
  SVK_CK(cudaStreamSynchronize(s->stream));
  return LBM_OK;
}

lbm_status fem_svk_get_state(fem_svk_ctx *s, double *u, double *v, int *iters) {
  if (!s) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  const size_t n = s->p.n;
  if (u) SVK_CK(cudaMemcpyAsync(u, s->d.u, sizeof(double) * n, cudaMemcpyDefault, s->stream));
  if (v) SVK_CK(cudaMemcpyAsync(v, s->d.v, sizeof(double) * n, cudaMemcpyDefault, s->stream));
  if (iters) SVK_CK(cudaMemcpyAsync(iters, s->d.iters, sizeof(int) * 2, cudaMemcpyDefault, s->stream));
  SVK_CK(cudaStreamSynchronize(s->stream));
  return LBM_OK;
}

lbm_status fem_svk_set_state(fem_svk_ctx *s, const double *u, const double *v, const double *F0) {
  if (!s) return LBM_EINVAL;
  if (s->poisoned) return LBM_ESTATE;
  const size_t n = s->p.n;
  if (u) SVK_CK(cudaMemcpyAsync(s->d.u, u, sizeof(double) * n, cudaMemcpyDefault, s->stream));
  if (v) SVK_CK(cudaMemcpyAsync(s->d.v, v, sizeof(double) * n, cudaMemcpyDefault, s->stream));
  if (F0) SVK_CK(cudaMemcpyAsync(s->d.F0, F0, sizeof(double) * n, cudaMemcpyDefault, s->stream));
  SVK_CK(cudaStreamSynchronize(s->stream));
  return LBM_OK;
}

const char *fem_svk_last_error(const fem_svk_ctx *s) { return s ? s->msg : g_svk_msg; }

void fem_svk_destroy(fem_svk_ctx *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  if (s->own_ws) cudaFree(s->ws);
  delete s;
}

}  // extern "C"
