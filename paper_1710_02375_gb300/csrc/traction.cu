// traction.cu -- fluid stress at the immersed boundary nodes and the surface
// traction it gives (the paper's force path of section "Fluid-structure
// coupling": the Cauchy stress of the fluid, sigma_f = -p I - (1 - beta) Pi^(1),
// evaluated at the surface; secondary to the momentum-exchange force).
//
// Readings: pressure relative to the rest state, p = (rho - 1) c_s^2, as for
// the momentum-exchange force; Pi^(1) = Pi - Pi_eq from the pre-collision
// populations of the step (after the Grad fill); each surface element takes
// the stress of the nearest immersed boundary node to its centroid (ties: the
// lower node index) and carries t = sigma n over its length (2-D, per unit
// depth) or area (3-D), n the outward unit normal of its body in the current
// configuration; the element force is shared equally by its vertices.
#include "boundary.cuh"
#include "lbm_internal.h"

namespace kbc {

// Stress (xx, yy, zz, xy, xz, yz) of immersed boundary node t from the
// pulled populations of the source buffer (FP64 arithmetic).
template <int Q, int S>
__global__ void k_stress_nodes(Grid g, const typename Store<S>::T *__restrict__ f,
                               const BNode *__restrict__ bn, const int *__restrict__ nbn, int cap,
                               double beta, double *__restrict__ sigma) {
  using L = Lat<Q>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *nbn < cap ? *nbn : cap;
  if (t >= n) return;
  const long long k = bn[t].k;
  int X, Y, Z;
  decompose(g, k, X, Y, Z);
  double dr = 0.0, j[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    const long long ks = sidx(g, nbr(X, -cx, g.NX), nbr(Y, -cy, g.NY),
                              L::D == 3 ? nbr(Z, -cz, g.NZ) : Z);
    const double gi = (double)Store<S>::load(f + (long long)i * g.N + ks, (float)weight<L>(i));
    dr += gi;
    j[0] += cx * gi; j[1] += cy * gi; j[2] += cz * gi;
    P[0] += cx * cx * gi; P[1] += cy * cy * gi; P[2] += cz * cz * gi;
    P[3] += cx * cy * gi; P[4] += cx * cz * gi; P[5] += cy * cz * gi;
  }
  // raw second moments of f = W + g: sum W c_a c_b = delta_ab / 3
  const double rho = 1.0 + dr;
  const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  // equilibrium second moments of the product-form equilibrium, relative to
  // delta_ab / 3: rho (2 S_a - 1) / 3 - 1/3 on the diagonal, rho u_a u_b off it
  double E[6];
  for (int a = 0; a < 3; ++a) {
    if (a >= L::D) { E[a] = dr / 3.0; continue; }  // no velocity along a missing axis
    const double Sa = sqrt(1.0 + 3.0 * u[a] * u[a]);
    E[a] = (rho * (2.0 * Sa - 1.0) - 1.0) / 3.0;
  }
  E[3] = rho * u[0] * u[1];
  E[4] = rho * u[0] * u[2];
  E[5] = rho * u[1] * u[2];
  const double p = dr / 3.0;
  double *s = sigma + 6 * (long long)t;
  for (int m = 0; m < 6; ++m) s[m] = (m < 3 ? -p : 0.0) - (1.0 - beta) * (P[m] - E[m]);
  if (L::D == 2) { s[2] = 0.0; s[4] = 0.0; s[5] = 0.0; }
}

// Signed area (2-D) / volume (3-D) of each body, for the outward normals.
__global__ void k_body_orientation(SurfaceDev s, double *acc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.ne) return;
  double v;
  if (s.dim == 2) {
    const double *a = s.x + 2 * s.e[2 * e], *b = s.x + 2 * s.e[2 * e + 1];
    v = 0.5 * (a[0] * b[1] - b[0] * a[1]);
  } else {
    const double *a = s.x + 3 * s.e[3 * e], *b = s.x + 3 * s.e[3 * e + 1], *c = s.x + 3 * s.e[3 * e + 2];
    v = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
         a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
  }
  atomicAdd(acc + s.eb[e], v);
}

// Element traction forces from the nearest boundary node's stress.
__global__ void k_element_traction(Grid g, SurfaceDev s, const BNode *__restrict__ bn,
                                   const int *__restrict__ nbn, int cap,
                                   const double *__restrict__ sigma,
                                   const double *__restrict__ orient, double *vforce,
                                   double *bforce) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.ne) return;
  const int n = *nbn < cap ? *nbn : cap;
  if (n == 0) return;
  const int dim = s.dim, body = s.eb[e];
  const double sg = orient[body] >= 0.0 ? 1.0 : -1.0;
  double xc[3] = {0, 0, 0}, nA[3] = {0, 0, 0};
  if (dim == 2) {
    const double *a = s.x + 2 * s.e[2 * e], *b = s.x + 2 * s.e[2 * e + 1];
    xc[0] = 0.5 * (a[0] + b[0]);
    xc[1] = 0.5 * (a[1] + b[1]);
    nA[0] = sg * (b[1] - a[1]);  // length x outward unit normal
    nA[1] = -sg * (b[0] - a[0]);
  } else {
    const double *a = s.x + 3 * s.e[3 * e], *b = s.x + 3 * s.e[3 * e + 1], *c = s.x + 3 * s.e[3 * e + 2];
    for (int q = 0; q < 3; ++q) xc[q] = (a[q] + b[q] + c[q]) / 3.0;
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    nA[0] = 0.5 * sg * (e1[1] * e2[2] - e1[2] * e2[1]);
    nA[1] = 0.5 * sg * (e1[2] * e2[0] - e1[0] * e2[2]);
    nA[2] = 0.5 * sg * (e1[0] * e2[1] - e1[1] * e2[0]);
  }
  int best = -1;
  long long bk = 0;
  double bd = 1e300;
  for (int t = 0; t < n; ++t) {
    const long long k = bn[t].k;
    int X, Y, Z;
    decompose(g, k, X, Y, Z);
    const double p[3] = {X - g.px + 0.5, Y - g.py + 0.5, Z - g.pz + 0.5};
    double d2 = 0.0;
    for (int q = 0; q < dim; ++q) d2 += (p[q] - xc[q]) * (p[q] - xc[q]);
    if (d2 < bd || (d2 == bd && k < bk)) {
      bd = d2;
      bk = k;
      best = t;
    }
  }
  const double *sv = sigma + 6 * (long long)best;
  const double Sm[3][3] = {{sv[0], sv[3], sv[4]}, {sv[3], sv[1], sv[5]}, {sv[4], sv[5], sv[2]}};
  double F[3];
  for (int a = 0; a < 3; ++a) F[a] = Sm[a][0] * nA[0] + Sm[a][1] * nA[1] + Sm[a][2] * nA[2];
  for (int a = 0; a < dim; ++a) {
    atomicAdd(bforce + 3 * body + a, F[a]);
    for (int m = 0; m < dim; ++m) atomicAdd(vforce + 3 * s.e[dim * e + m] + a, F[a] / dim);
  }
}

static cudaError_t launch_stress(int Q, int storage, const Grid &g, const void *f, const BNode *bn,
                                 const int *nbn, int cap, double beta, double *sigma,
                                 cudaStream_t s) {
  KBC_DISPATCH(Q, storage, {
    k_stress_nodes<QQ, SS><<<(cap + 127) / 128, 128, 0, s>>>(
        g, (const typename Store<SS>::T *)f, bn, nbn, cap, beta, sigma);
    return cudaGetLastError();
  });
}

cudaError_t launch_traction(int Q, int storage, const Grid &g, const void *f, const BNode *bn,
                            const int *nbn, int cap, double beta, const SurfaceDev &sd,
                            double *sigma, double *orient, double *vforce, double *bforce,
                            int nbodies, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(vforce, 0, sizeof(double) * 3 * (sd.nv > 0 ? sd.nv : 1), s)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(bforce, 0, sizeof(double) * 3 * nbodies, s)) != cudaSuccess) return e;
  if (cap <= 0 || sd.ne <= 0) return cudaSuccess;
  if ((e = cudaMemsetAsync(orient, 0, sizeof(double) * nbodies, s)) != cudaSuccess) return e;
  if ((e = launch_stress(Q, storage, g, f, bn, nbn, cap, beta, sigma, s)) != cudaSuccess) return e;
  k_body_orientation<<<(sd.ne + 127) / 128, 128, 0, s>>>(sd, orient);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_element_traction<<<(sd.ne + 127) / 128, 128, 0, s>>>(g, sd, bn, nbn, cap, sigma, orient,
                                                         vforce, bforce);
  return cudaGetLastError();
}

}  // namespace kbc
