// kbc_collide.cuh -- the KBC collision of one node in FP32 registers.
//
// Works on deviations g_i = f_i - W_i so that the O(u) content of each
// population keeps the full FP32 mantissa.  Steps (arXiv 1710.02375):
//   moments rho, j, P (deviation moments)           -- Eq. (conservationLaws)
//   entropic equilibrium, closed product form       -- Eq. (feq_min)
//       feq_i = rho prod_a W(c_ia) phi_a(c_ia),  phi(0) = 2 - S,
//       phi(+-1) = (2 - S)(S +- 2u)/(1 -+ u),    S = sqrt(1 + 3u^2),
//     evaluated as 1 + eps products so feq_i - W_i keeps relative accuracy;
//   shear part ds of f - feq from the trace-free second moments -- Eq. (popSplit)
//   dh = f - feq - ds (the kinematic part does not change)
//   gamma = 1/beta - (2 - 1/beta) <ds|dh>/<dh|dh>, <X|Y> = sum X Y / feq
//                                                   -- Eq. (gamma_min_approx)
//   f' = f - beta (2 ds + gamma dh)                 -- Eqs. (f_equations), (f_mirr)
// gamma = 2 (LBGK, omega = 2 beta) when <dh|dh> <= 1e-30 or BGK is requested;
// otherwise gamma is held in [0, 2/beta], where (1 - beta gamma) dh, the
// post-collision higher-order part, does not grow.
// The metric weights are evaluated up to the common factor 1/rho, so the
// degenerate-case threshold applies to rho <dh|dh>.
#pragma once
#include "kbc_common.cuh"

namespace kbc {

struct AxisEq {
  float e[3];   // phi(c) - 1 for c = -1, 0, +1
  float r[3];   // 1 / (w(c) phi(c)): per-axis factor of the entropic metric 1/feq
  float d;      // S - 1
};

__device__ __forceinline__ AxisEq axis_eq(float u) {
  AxisEq a;
  const float u2 = u * u;
  const float x = fmaf(3.0f, u2, 1.0f);
  const float S = x * rsqrtf(x);                       // sqrt(1 + 3u^2)
  const float d = __fdividef(3.0f * u2, 1.0f + S);     // S - 1 without cancellation
  const float om = 1.0f - d;                           // 2 - S
  const float ip = __fdividef(1.0f, 1.0f - u);
  const float im = __fdividef(1.0f, 1.0f + u);
  a.e[1] = -d;
  a.e[2] = fmaf(om, (d + 3.0f * u) * ip, -d);
  a.e[0] = fmaf(om, (d - 3.0f * u) * im, -d);
  a.r[0] = __fdividef(6.0f, 1.0f + a.e[0]);
  a.r[1] = __fdividef(1.5f, om);
  a.r[2] = __fdividef(6.0f, 1.0f + a.e[2]);
  a.d = d;
  return a;
}

// In-place collision of g[Q] (deviations g_i = f_i - W_i).  Returns rho.
//
// Sums are taken in the tensor-product structure of the lattice (rows of
// three x-neighbours, then planes), the equilibrium factors and the metric
// weights 1/feq_i (up to the common factor 1/rho, which cancels in gamma) as
// products of per-axis factors, and <ds|dh> grouped by the six distinct
// values of ds.
// CONSERVE: remove the FP32 rounding residue of mass and momentum from the
// non-equilibrium part (used with FP32 storage, where it would otherwise be
// the dominant error; with 16-bit storage the storage rounding dominates).
template <class L, bool CONSERVE = true>
__device__ __forceinline__ float collide(float (&g)[L::Q], float beta, bool bgk) {
  constexpr int Q = L::Q;
  constexpr int NR = Q / 3;  // rows of three x-neighbours (cy, cz)
  // ---- moments of the deviations (Eq. conservationLaws and second moments)
  float rs[NR], rd[NR], rm[NR];  // per row: g+ + g-, g+ - g-, g- + g0 + g+
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    rs[r] = g[3 * r + 2] + g[3 * r];
    rd[r] = g[3 * r + 2] - g[3 * r];
    rm[r] = rs[r] + g[3 * r + 1];
  }
  // row r has cy = r % 3 - 1, cz = r / 3 - 1
  float drho = 0.f, jx = 0.f, pxx = 0.f;
  float yp = 0.f, ym = 0.f, zp = 0.f, zm = 0.f;      // sums of rm over cy = +-1, cz = +-1
  float pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int cy = r % 3 - 1, cz = (L::D == 3) ? r / 3 - 1 : 0;
    drho += rm[r];
    jx += rd[r];
    pxx += rs[r];
    if (cy > 0) yp += rm[r];
    if (cy < 0) ym += rm[r];
    if (cz > 0) zp += rm[r];
    if (cz < 0) zm += rm[r];
    if (cy) pxy += cy * rd[r];
    if (cz) pxz += cz * rd[r];
    if (cy && cz) pyz += cy * cz * rm[r];
  }
  const float jy = yp - ym, pyy = yp + ym;
  const float jz = zp - zm, pzz = zp + zm;

  const float rho = 1.0f + drho;
  const float irho = __fdividef(1.0f, rho);
  const float ux = jx * irho, uy = jy * irho, uz = jz * irho;

  const AxisEq ax = axis_eq(ux), ay = axis_eq(uy);
  AxisEq az;
  if (L::D == 3) az = axis_eq(uz);

  // ---- shear part of f - feq from the deviatoric non-equilibrium stress
  // dPi_aa = P_aa - (drho + 2 rho d_a)/3, dPi_ab = P_ab - rho u_a u_b
  const float dxx = pxx - (drho + 2.f * rho * ax.d) * (1.f / 3.f);
  const float dyy = pyy - (drho + 2.f * rho * ay.d) * (1.f / 3.f);
  float sv[6];  // ds of the x, y, z faces and of the xy, xz, yz edges (sign +)
  if (L::D == 2) {
    const float N = dxx - dyy;
    sv[0] = 0.25f * N;
    sv[1] = -0.25f * N;
    sv[2] = 0.f;
    sv[3] = 0.25f * (pxy - rho * ux * uy);
    sv[4] = sv[5] = 0.f;
  } else {
    const float dzz = pzz - (drho + 2.f * rho * az.d) * (1.f / 3.f);
    const float Nxz = dxx - dzz, Nyz = dyy - dzz;
    sv[0] = (2.f * Nxz - Nyz) * (1.f / 6.f);
    sv[1] = (2.f * Nyz - Nxz) * (1.f / 6.f);
    sv[2] = -(Nxz + Nyz) * (1.f / 6.f);
    sv[3] = 0.25f * (pxy - rho * ux * uy);
    sv[4] = 0.25f * (pxz - rho * ux * uz);
    sv[5] = 0.25f * (pyz - rho * uy * uz);
  }

  // ---- per-direction non-equilibrium part and the entropic products
  // (1 + e_x)(1 + e_y) - 1 = e_x + e_y (1 + e_x), and likewise with e_z
  float exy[9], qxy[9], mxy[9];
  float px1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) px1[a] = 1.0f + ax.e[a];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      exy[3 * b + a] = fmaf(ay.e[b], px1[a], ax.e[a]);
      if (L::D == 3) qxy[3 * b + a] = 1.0f + exy[3 * b + a];
      mxy[3 * b + a] = ax.r[a] * ay.r[b];
    }
  float df[Q];
  float grp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // signed sums of m_i dh_i per ds group
  float hh = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    const int k2 = 3 * (cy + 1) + (cx + 1);
    float e = exy[k2], m = mxy[k2];
    if (L::D == 3) {
      e = fmaf(az.e[cz + 1], qxy[k2], e);
      m *= az.r[cz + 1];
    }
    // feq_i - W_i = W_i (drho + rho e_i);  df_i = g_i - (feq_i - W_i)
    const float d = fmaf(-(float)weight<L>(i), fmaf(rho, e, drho), g[i]);
    df[i] = d;
    const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
    int gi = -1, sg = 1;
    if (nnz == 1) gi = cx ? 0 : (cy ? 1 : 2);
    if (nnz == 2) {
      if (cx && cy) { gi = 3; sg = cx * cy; }
      else if (cx && cz) { gi = 4; sg = cx * cz; }
      else { gi = 5; sg = cy * cz; }
    }
    const float dh = (gi >= 0) ? d - sg * sv[gi < 0 ? 0 : gi] : d;
    const float t = m * dh;
    hh = fmaf(t, dh, hh);
    if (gi >= 0) grp[gi] += sg * t;
  }
  float sh = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) sh = fmaf(sv[k], grp[k], sh);

  const float ib = __fdividef(1.0f, beta);
  float gamma = 2.f;
  // <.|.> carries a common factor rho that cancels in the ratio
  if (!bgk && hh > 1e-30f) {
    gamma = ib - (2.f - ib) * __fdividef(sh, hh);
    // the vertex of the quadratic entropy norm clipped to the rates at which
    // the higher-order part does not grow, |1 - beta gamma| <= 1
    gamma = fminf(fmaxf(gamma, 0.f), 2.f * ib);
  }

  // ---- conservation of the FP32 update: df carries no mass or momentum in
  // exact arithmetic; its rounding residue (dm, dj) would otherwise leak into
  // the conserved moments every step, so it is removed along W_i (1, 3 c_i).
  float qm = 0.f, qx = 0.f, qyp = 0.f, qym = 0.f, qzp = 0.f, qzm = 0.f;
#pragma unroll
  for (int r = 0; r < (CONSERVE ? NR : 0); ++r) {
    const int cy = r % 3 - 1, cz = (L::D == 3) ? r / 3 - 1 : 0;
    const float m = df[3 * r] + df[3 * r + 1] + df[3 * r + 2];
    qm += m;
    qx += df[3 * r + 2] - df[3 * r];
    if (cy > 0) qyp += m;
    if (cy < 0) qym += m;
    if (cz > 0) qzp += m;
    if (cz < 0) qzm += m;
  }

  // ---- relaxation f' = f - beta (2 ds + gamma dh) = f - beta (gamma df + (2 - gamma) ds)
  const float bg = beta * gamma, b2g = beta * (2.f - gamma);
  const float A = bg * qm, Bx = 3.f * bg * qx, By = 3.f * bg * (qyp - qym),
              Bz = 3.f * bg * (qzp - qzm);
  float bs[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) bs[k] = b2g * sv[k];
  // projection term A + c_i.B built row by row: (cy, cz) part once per row
  float tyz[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int cy = r % 3 - 1, cz = (L::D == 3) ? r / 3 - 1 : 0;
    float t = A;
    if (cy) t += cy * By;
    if (cz) t += cz * Bz;
    tyz[r] = t;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
    float sds = 0.f;
    if (nnz == 1) sds = cx ? bs[0] : (cy ? bs[1] : bs[2]);
    if (nnz == 2) {
      if (cx && cy) sds = cx * cy * bs[3];
      else if (cx && cz) sds = cx * cz * bs[4];
      else sds = cy * cz * bs[5];
    }
    if (CONSERVE) {
      float t = tyz[i / 3];
      if (cx) t += cx * Bx;
      sds = fmaf(-(float)weight<L>(i), t, sds);
    }
    g[i] = g[i] - fmaf(bg, df[i], sds);
  }
  return rho;
}

}  // namespace kbc
