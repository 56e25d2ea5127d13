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
// Forced form (multiphase model, Eq. (force_mp)): with a velocity increment
// du = F / rho the entropic products take the shifted metric 1 / feq(rho,
// u + du) and the relaxed state gains F_i = feq(rho, u + du) - feq(rho, u).
// gamma = 2 (LBGK, omega = 2 beta) when <dh|dh> <= 1e-30 or BGK is requested;
// otherwise gamma is held in [0, 2/beta], where (1 - beta gamma) dh, the
// post-collision higher-order part, does not grow.
// The metric weights are evaluated up to the common factor 1/rho, so the
// degenerate-case threshold applies to rho <dh|dh>.
#pragma once
#include "kbc_common.cuh"

namespace kbc {

// ---- arithmetic on one node (float) or on two nodes at once (f2) ----------
// f2 holds the same quantity of two nodes; its operations issue the paired
// FP32 instructions of sm_100+ (one instruction, two IEEE results), so the
// two-node sweep spends half the FP32 issue slots per node.  The special
// functions (reciprocal, reciprocal square root) stay one per value.
struct f2 {
  float2 v;
};
__device__ __forceinline__ f2 mk2(float a, float b) { return f2{make_float2(a, b)}; }
// scalar type of a value type (parameters such as beta)
template <class V>
struct ScalarOf {
  using type = float;
};
template <>
struct ScalarOf<double> {
  using type = double;
};
// a constant in the value type (constants are written in double and rounded
// once to FP32 for the FP32 forms)
template <class V>
__device__ __forceinline__ V vc(double a);
template <>
__device__ __forceinline__ float vc<float>(double a) { return (float)a; }
template <>
__device__ __forceinline__ f2 vc<f2>(double a) { return mk2((float)a, (float)a); }
template <>
__device__ __forceinline__ double vc<double>(double a) { return a; }

// The float forms are the IEEE operations of the paired ones (no contraction
// of a product into a following sum), so one-node and two-node sweeps agree
// to the last bit.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ f2 vadd(f2 a, f2 b) { return f2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
// a - b as fma(b, -1, a): exact product, one rounding, one paired instruction
__device__ __forceinline__ f2 vsub(f2 a, f2 b) {
  return f2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)};
}
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ f2 vmul(f2 a, f2 b) { return f2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return f2{__ffma2_rn(a.v, b.v, c.v)}; }
// FP64 forms (the F64 test storage)
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vrsqrt(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ double vdivf(double a, double b) { return a / b; }
__device__ __forceinline__ float vrsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ f2 vrsqrt(f2 a) { return mk2(rsqrtf(a.v.x), rsqrtf(a.v.y)); }
__device__ __forceinline__ float vdivf(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ f2 vdivf(f2 a, f2 b) {
  return mk2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}

template <class V>
struct AxisEqT {
  V e[3];  // phi(c) - 1 for c = -1, 0, +1
  V r[3];  // 1 / (w(c) phi(c)): per-axis factor of the entropic metric 1/feq
  V d;     // S - 1
};
using AxisEq = AxisEqT<float>;

template <class V>
__device__ __forceinline__ AxisEqT<V> axis_eq(V u) {
  AxisEqT<V> a;
  const V u2 = vmul(u, u);
  const V x = vfma(vc<V>(3.0f), u2, vc<V>(1.0f));
  const V S = vmul(x, vrsqrt(x));                                  // sqrt(1 + 3u^2)
  const V d = vdivf(vmul(vc<V>(3.0f), u2), vadd(vc<V>(1.0f), S));  // S - 1 without cancellation
  const V om = vsub(vc<V>(1.0f), d);                               // 2 - S
  const V ip = vdivf(vc<V>(1.0f), vsub(vc<V>(1.0f), u));
  const V im = vdivf(vc<V>(1.0f), vadd(vc<V>(1.0f), u));
  const V u3 = vmul(vc<V>(3.0f), u);
  const V nd = vsub(vc<V>(0.0f), d);
  a.e[1] = nd;
  a.e[2] = vfma(om, vmul(vadd(d, u3), ip), nd);
  a.e[0] = vfma(om, vmul(vsub(d, u3), im), nd);
  a.r[0] = vdivf(vc<V>(6.0f), vadd(vc<V>(1.0f), a.e[0]));
  a.r[1] = vdivf(vc<V>(1.5f), om);
  a.r[2] = vdivf(vc<V>(6.0f), vadd(vc<V>(1.0f), a.e[2]));
  a.d = d;
  return a;
}

// gamma of Eq. (gamma_min_approx) from the two entropic products, held in
// [0, 2/beta]; 2 (LBGK) when bgk or <dh|dh> <= 1e-30.
__device__ __forceinline__ float kbc_gamma(float sh, float hh, float ib, bool bgk) {
  float gamma = 2.f;
  if (!bgk && hh > 1e-30f) {
    gamma = ib - (2.f - ib) * __fdividef(sh, hh);
    // the vertex of the quadratic entropy norm clipped to the rates at which
    // the higher-order part does not grow, |1 - beta gamma| <= 1
    gamma = fminf(fmaxf(gamma, 0.f), 2.f * ib);
  }
  return gamma;
}
__device__ __forceinline__ float vgamma(float sh, float hh, float ib, bool bgk) {
  return kbc_gamma(sh, hh, ib, bgk);
}
__device__ __forceinline__ double vgamma(double sh, double hh, double ib, bool bgk) {
  double gamma = 2.0;
  if (!bgk && hh > 1e-30) {
    gamma = ib - (2.0 - ib) * (sh / hh);
    gamma = fmin(fmax(gamma, 0.0), 2.0 * ib);
  }
  return gamma;
}
__device__ __forceinline__ f2 vgamma(f2 sh, f2 hh, float ib, bool bgk) {
  return mk2(kbc_gamma(sh.v.x, hh.v.x, ib, bgk), kbc_gamma(sh.v.y, hh.v.y, ib, bgk));
}

// In-place collision of g[Q] (deviations g_i = f_i - W_i), of one node (V =
// float) or of two nodes (V = f2).  Returns rho.
//
// Sums are taken in the tensor-product structure of the lattice (rows of
// three x-neighbours, then planes), the equilibrium factors and the metric
// weights 1/feq_i (up to the common factor 1/rho, which cancels in gamma) as
// products of per-axis factors, and <ds|dh> grouped by the six distinct
// values of ds.
// CONSERVE: remove the FP32 rounding residue of mass and momentum from the
// non-equilibrium part (used with FP32 storage, where it would otherwise be
// the dominant error; with 16-bit storage the storage rounding dominates).
// FORCED: the forced form with velocity increment (dux, duy, duz), on
// deviations g_i = f_i - W_i ref from a reference density ref of the node
// (the moments and the update are unchanged in that form: only rho = ref +
// sum g_i); the unforced instantiations compile without any of its code.
template <class L, bool CONSERVE, class V, bool FORCED = false>
__device__ __forceinline__ V collide_v(V (&g)[L::Q], typename ScalarOf<V>::type beta, bool bgk,
                                       V dux = V(), V duy = V(), V duz = V(), V ref = V()) {
  using SC = typename ScalarOf<V>::type;
  constexpr int Q = L::Q;
  constexpr int NR = Q / 3;  // rows of three x-neighbours (cy, cz)
  const V zero = vc<V>(0.0);
  // ---- moments of the deviations (Eq. conservationLaws and second moments)
  V rs[NR], rd[NR], rm[NR];  // per row: g+ + g-, g+ - g-, g- + g0 + g+
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    rs[r] = vadd(g[3 * r + 2], g[3 * r]);
    rd[r] = vsub(g[3 * r + 2], g[3 * r]);
    rm[r] = vadd(rs[r], g[3 * r + 1]);
  }
  // row r has cy = r % 3 - 1, cz = r / 3 - 1
  V drho = zero, jx = zero, pxx = zero;
  V yp = zero, ym = zero, zp = zero, zm = zero;  // sums of rm over cy = +-1, cz = +-1
  V pxy = zero, pxz = zero, pyz = zero;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int cy = r % 3 - 1, cz = (L::D == 3) ? r / 3 - 1 : 0;
    drho = vadd(drho, rm[r]);
    jx = vadd(jx, rd[r]);
    pxx = vadd(pxx, rs[r]);
    if (cy > 0) yp = vadd(yp, rm[r]);
    if (cy < 0) ym = vadd(ym, rm[r]);
    if (cz > 0) zp = vadd(zp, rm[r]);
    if (cz < 0) zm = vadd(zm, rm[r]);
    if (cy > 0) pxy = vadd(pxy, rd[r]);
    if (cy < 0) pxy = vsub(pxy, rd[r]);
    if (cz > 0) pxz = vadd(pxz, rd[r]);
    if (cz < 0) pxz = vsub(pxz, rd[r]);
    if (cy * cz > 0) pyz = vadd(pyz, rm[r]);
    if (cy * cz < 0) pyz = vsub(pyz, rm[r]);
  }
  const V jy = vsub(yp, ym), pyy = vadd(yp, ym);
  const V jz = vsub(zp, zm), pzz = vadd(zp, zm);

  V rho;
  if constexpr (FORCED) rho = vadd(ref, drho);
  else rho = vadd(vc<V>(1.0f), drho);
  const V irho = vdivf(vc<V>(1.0f), rho);
  const V ux = vmul(jx, irho), uy = vmul(jy, irho), uz = vmul(jz, irho);

  const AxisEqT<V> ax = axis_eq(ux), ay = axis_eq(uy);
  AxisEqT<V> az;
  if (L::D == 3) az = axis_eq(uz);
  // equilibrium factors at the shifted velocity u + du (forced form)
  AxisEqT<V> sx, sy, sz;
  if constexpr (FORCED) {
    sx = axis_eq(vadd(ux, dux));
    sy = axis_eq(vadd(uy, duy));
    if (L::D == 3) sz = axis_eq(vadd(uz, duz));
  }

  // ---- shear part of f - feq from the deviatoric non-equilibrium stress
  // dPi_aa = P_aa - (drho + 2 rho d_a)/3, dPi_ab = P_ab - rho u_a u_b
  const V rho2 = vmul(vc<V>(2.f), rho);
  const V third = vc<V>(1.0 / 3.0);
  const V dxx = vsub(pxx, vmul(vfma(rho2, ax.d, drho), third));
  const V dyy = vsub(pyy, vmul(vfma(rho2, ay.d, drho), third));
  V sv[6];  // ds of the x, y, z faces and of the xy, xz, yz edges (sign +)
  const V quarter = vc<V>(0.25f);
  if (L::D == 2) {
    const V N = vsub(dxx, dyy);
    sv[0] = vmul(quarter, N);
    sv[1] = vmul(vc<V>(-0.25), N);
    sv[2] = zero;
    sv[3] = vmul(quarter, vsub(pxy, vmul(vmul(rho, ux), uy)));
    sv[4] = sv[5] = zero;
  } else {
    const V dzz = vsub(pzz, vmul(vfma(rho2, az.d, drho), third));
    const V Nxz = vsub(dxx, dzz), Nyz = vsub(dyy, dzz);
    const V sixth = vc<V>(1.0 / 6.0);
    sv[0] = vmul(vsub(vadd(Nxz, Nxz), Nyz), sixth);
    sv[1] = vmul(vsub(vadd(Nyz, Nyz), Nxz), sixth);
    sv[2] = vmul(vadd(Nxz, Nyz), vc<V>(-1.0 / 6.0));
    const V rux = vmul(rho, ux);
    sv[3] = vmul(quarter, vsub(pxy, vmul(rux, uy)));
    sv[4] = vmul(quarter, vsub(pxz, vmul(rux, uz)));
    sv[5] = vmul(quarter, vsub(pyz, vmul(vmul(rho, uy), uz)));
  }

  // ---- per-direction non-equilibrium part and the entropic products
  // (1 + e_x)(1 + e_y) - 1 = e_x + e_y (1 + e_x), and likewise with e_z.
  // Directions are visited by (c_x, c_y) pair k2 with c_z innermost, so the
  // x-y factors of a pair live only while its (up to) three directions are
  // processed; the non-equilibrium part df_i is not kept: the relaxation
  // below forms it again by the same operations (same value).
  V px1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) px1[a] = vadd(vc<V>(1.0f), ax.e[a]);
  V grp[6] = {zero, zero, zero, zero, zero, zero};  // signed sums of m_i dh_i per ds group
  V hh = zero;
  // mass and momentum of df (zero in exact arithmetic; see CONSERVE)
  V qm = zero, qx = zero, qy = zero, qz = zero;
#pragma unroll
  for (int k2 = 0; k2 < 9; ++k2) {
    const int a = k2 % 3, b = k2 / 3;  // a = cx + 1, b = cy + 1
    const V exy = vfma(ay.e[b], px1[a], ax.e[a]);
    const V qxy = vadd(vc<V>(1.0f), exy);
    V mxy;
    if constexpr (FORCED) mxy = vmul(sx.r[a], sy.r[b]);
    else mxy = vmul(ax.r[a], ay.r[b]);
#pragma unroll
    for (int zc = 0; zc < (L::D == 3 ? 3 : 1); ++zc) {
      const int i = (L::D == 3 ? 9 * zc : 0) + k2;
      const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
      V e = exy, m = mxy;
      if (L::D == 3) {
        e = vfma(az.e[cz + 1], qxy, e);
        if constexpr (FORCED) m = vmul(m, sz.r[cz + 1]);
        else m = vmul(m, az.r[cz + 1]);
      }
      // feq_i - W_i = W_i (drho + rho e_i);  df_i = g_i - (feq_i - W_i)
      const V d = vfma(vc<V>(-weight<L>(i)), vfma(rho, e, drho), g[i]);
      const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
      int gi = -1, sg = 1;
      if (nnz == 1) gi = cx ? 0 : (cy ? 1 : 2);
      if (nnz == 2) {
        if (cx && cy) { gi = 3; sg = cx * cy; }
        else if (cx && cz) { gi = 4; sg = cx * cz; }
        else { gi = 5; sg = cy * cz; }
      }
      V dh = d;
      if (gi >= 0) dh = (sg > 0) ? vsub(d, sv[gi]) : vadd(d, sv[gi]);
      const V t = vmul(m, dh);
      hh = vfma(t, dh, hh);
      if (gi >= 0) grp[gi] = (sg > 0) ? vadd(grp[gi], t) : vsub(grp[gi], t);
      if (CONSERVE) {
        qm = vadd(qm, d);
        if (cx > 0) qx = vadd(qx, d);
        if (cx < 0) qx = vsub(qx, d);
        if (cy > 0) qy = vadd(qy, d);
        if (cy < 0) qy = vsub(qy, d);
        if (cz > 0) qz = vadd(qz, d);
        if (cz < 0) qz = vsub(qz, d);
      }
    }
  }
  V sh = zero;
#pragma unroll
  for (int k = 0; k < 6; ++k) sh = vfma(sv[k], grp[k], sh);

  const SC ib = vdivf((SC)1, beta);
  // <.|.> carries a common factor rho that cancels in the ratio
  const V gamma = vgamma(sh, hh, ib, bgk);

  // ---- relaxation f' = f - beta (2 ds + gamma dh) = f - beta (gamma df + (2 - gamma) ds).
  // Conservation of the FP32 update (CONSERVE): df carries no mass or
  // momentum in exact arithmetic; its rounding residue (qm, q) would otherwise
  // leak into the conserved moments every step, so it is removed along
  // W_i (1, 3 c_i).
  const V bg = vmul(vc<V>(beta), gamma);
  const V b2g = vmul(vc<V>(beta), vsub(vc<V>(2.f), gamma));
  const V bg3 = vmul(vc<V>(3.f), bg);
  const V A = vmul(bg, qm), Bx = vmul(bg3, qx), By = vmul(bg3, qy), Bz = vmul(bg3, qz);
  V bs[6], nbs[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    bs[k] = vmul(b2g, sv[k]);
    nbs[k] = vsub(zero, bs[k]);
  }
#pragma unroll
  for (int k2 = 0; k2 < 9; ++k2) {
    const int a = k2 % 3, b = k2 / 3;
    const V exy = vfma(ay.e[b], px1[a], ax.e[a]);
    const V qxy = vadd(vc<V>(1.0f), exy);
    V sxy = zero, sqxy = zero;  // shifted x-y factors (forced form)
    if constexpr (FORCED) {
      sxy = vfma(sy.e[b], vadd(vc<V>(1.0f), sx.e[a]), sx.e[a]);
      sqxy = vadd(vc<V>(1.0f), sxy);
    }
#pragma unroll
    for (int zc = 0; zc < (L::D == 3 ? 3 : 1); ++zc) {
      const int i = (L::D == 3 ? 9 * zc : 0) + k2;
      const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
      V e = exy;
      if (L::D == 3) e = vfma(az.e[cz + 1], qxy, e);
      const V d = vfma(vc<V>(-weight<L>(i)), vfma(rho, e, drho), g[i]);
      const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
      V sds = zero;
      int gk = -1, sg = 1;
      if (nnz == 1) gk = cx ? 0 : (cy ? 1 : 2);
      if (nnz == 2) {
        if (cx && cy) { gk = 3; sg = cx * cy; }
        else if (cx && cz) { gk = 4; sg = cx * cz; }
        else { gk = 5; sg = cy * cz; }
      }
      if (gk >= 0) sds = (sg > 0) ? bs[gk] : nbs[gk];
      if (CONSERVE) {
        V t = A;
        if (cx > 0) t = vadd(t, Bx);
        if (cx < 0) t = vsub(t, Bx);
        if (cy > 0) t = vadd(t, By);
        if (cy < 0) t = vsub(t, By);
        if (cz > 0) t = vadd(t, Bz);
        if (cz < 0) t = vsub(t, Bz);
        sds = vfma(vc<V>(-weight<L>(i)), t, sds);
      }
      g[i] = vsub(g[i], vfma(bg, d, sds));
      if constexpr (FORCED) {
        // F_i = feq(rho, u + du) - feq(rho, u) = W_i rho (e_i(u + du) - e_i(u))
        V es = sxy;
        if (L::D == 3) es = vfma(sz.e[cz + 1], sqxy, es);
        g[i] = vfma(vc<V>(weight<L>(i)), vmul(rho, vsub(es, e)), g[i]);
      }
    }
  }
  return rho;
}

// One node in FP32 (the form every single-node kernel uses).
template <class L, bool CONSERVE = true>
__device__ __forceinline__ float collide(float (&g)[L::Q], float beta, bool bgk) {
  return collide_v<L, CONSERVE, float>(g, beta, bgk);
}

}  // namespace kbc
