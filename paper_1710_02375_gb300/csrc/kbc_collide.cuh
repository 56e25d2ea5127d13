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
// gamma = 2 (LBGK, omega = 2 beta) when <dh|dh> <= 1e-30 or BGK is requested.
#pragma once
#include "kbc_common.cuh"

namespace kbc {

struct AxisEq {
  float e[3];   // phi(c) - 1 for c = -1, 0, +1
  float r[3];   // 1 / phi(c)
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
  a.r[0] = __fdividef(1.0f, 1.0f + a.e[0]);
  a.r[1] = __fdividef(1.0f, om);
  a.r[2] = __fdividef(1.0f, 1.0f + a.e[2]);
  a.d = d;
  return a;
}

// In-place collision of g[Q] (deviations).  Returns rho (for stability checks).
template <class L>
__device__ __forceinline__ float collide(float (&g)[L::Q], float beta, bool bgk) {
  constexpr int Q = L::Q;
  // ---- moments of the deviations
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    const float v = g[i];
    drho += v;
    if (cx) { jx += cx * v; pxx += v; }
    if (cy) { jy += cy * v; pyy += v; }
    if (cz) { jz += cz * v; pzz += v; }
    if (cx && cy) pxy += cx * cy * v;
    if (cx && cz) pxz += cx * cz * v;
    if (cy && cz) pyz += cy * cz * v;
  }
  const float rho = 1.0f + drho;
  const float irho = __fdividef(1.0f, rho);
  const float ux = jx * irho, uy = jy * irho, uz = jz * irho;

  const AxisEq ax = axis_eq(ux), ay = axis_eq(uy);
  AxisEq az;
  if (L::D == 3) az = axis_eq(uz);

  // ---- deviatoric non-equilibrium stress -> shear part (Eq. popSplit)
  // dPi_aa = P_aa - (drho + 2 rho d_a)/3, dPi_ab = P_ab - rho u_a u_b
  const float dxx = pxx - (drho + 2.f * rho * ax.d) * (1.f / 3.f);
  const float dyy = pyy - (drho + 2.f * rho * ay.d) * (1.f / 3.f);
  const float dxy = pxy - rho * ux * uy;
  float s_x, s_y, s_z = 0.f, s_xy, s_xz = 0.f, s_yz = 0.f;
  if (L::D == 2) {
    const float N = dxx - dyy;
    s_x = 0.25f * N;
    s_y = -0.25f * N;
    s_xy = 0.25f * dxy;
  } else {
    const float dzz = pzz - (drho + 2.f * rho * az.d) * (1.f / 3.f);
    const float Nxz = dxx - dzz, Nyz = dyy - dzz;
    s_x = (2.f * Nxz - Nyz) * (1.f / 6.f);
    s_y = (2.f * Nyz - Nxz) * (1.f / 6.f);
    s_z = -(Nxz + Nyz) * (1.f / 6.f);
    s_xy = 0.25f * dxy;
    s_xz = 0.25f * (pxz - rho * ux * uz);
    s_yz = 0.25f * (pyz - rho * uy * uz);
  }

  // ---- entropic products <ds|dh>, <dh|dh>
  float df[Q];
  float sh = 0.f, hh = 0.f;
  const float irho_w = irho;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    const float W = (float)weight<L>(i);
    const float iW = (float)(1.0 / weight<L>(i));
    // feq_i - W_i = W_i (drho + rho e_i), e_i = prod(1 + eps_a) - 1
    float e = ax.e[cx + 1];
    float r = ax.r[cx + 1];
    {
      const float ey = ay.e[cy + 1];
      e = e + ey + e * ey;
      r *= ay.r[cy + 1];
    }
    if (L::D == 3) {
      const float ez = az.e[cz + 1];
      e = e + ez + e * ez;
      r *= az.r[cz + 1];
    }
    const float feqdev = W * fmaf(rho, e, drho);
    const float invfeq = iW * irho_w * r;
    float ds = 0.f;
    const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
    if (nnz == 1) ds = cx ? s_x : (cy ? s_y : s_z);
    if (nnz == 2) {
      if (cx && cy) ds = cx * cy * s_xy;
      else if (cx && cz) ds = cx * cz * s_xz;
      else ds = cy * cz * s_yz;
    }
    const float d = g[i] - feqdev;
    df[i] = d;
    const float dh = d - ds;
    sh = fmaf(ds * dh, invfeq, sh);
    hh = fmaf(dh * dh, invfeq, hh);
  }
  const float ib = __fdividef(1.0f, beta);
  float gamma = 2.f;
  if (!bgk && hh > 1e-30f) gamma = ib - (2.f - ib) * __fdividef(sh, hh);

  // ---- relaxation f' = f - beta (2 ds + gamma dh) = f - beta ((2 - gamma) ds + gamma df)
  const float bg = beta * gamma, b2g = beta * (2.f - gamma);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    float ds = 0.f;
    const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
    if (nnz == 1) ds = cx ? s_x : (cy ? s_y : s_z);
    if (nnz == 2) {
      if (cx && cy) ds = cx * cy * s_xy;
      else if (cx && cz) ds = cx * cz * s_xz;
      else ds = cy * cz * s_yz;
    }
    g[i] = g[i] - fmaf(bg, df[i], b2g * ds);
  }
  return rho;
}

}  // namespace kbc
