// multiphase.cu -- the multiphase KBC step (arXiv 1710.02375, section
// "Extensions to fluid-structure interaction in multiphase flow").
//
// Per time step, on a fully periodic lattice:
//   1. density pass: rho(x) = sum_i f_i(x - c_i) of the pulled populations
//      and phi(x) = sqrt(max(rho c_s^2 - p(rho), 0)) with p of Eq. (eos);
//   2. Laplacian pass: lap rho(x) = 6 sum_i W_i (rho(x + c_i) - rho(x));
//   3. forced sweep: the pull-stream of the populations, the mean-field force
//        F = 2 phi d(phi) + kappa rho d(lap rho) (+ rho g),
//      (Eqs. (force1), (Korteweg); the sign of the capillary term is that of
//      the divergence of the Korteweg tensor), with the isotropic lattice
//      gradient d_a psi(x) = 3 sum_i W_i c_ia psi(x + c_i), the velocity
//      increment du = F / rho of the exact difference method, and the KBC
//      collision in its forced form (kbc_collide.cuh): gamma in the shifted
//      entropic product, F_i = feq(rho, u + du) - feq(rho, u) added,
//      Eq. (force_mp).
// Passes 1 and 2 write one density and one (phi, lap) pair per node; the
// sweep reads its node's 27 (9) populations from HBM and the 26 (8)
// neighbouring (phi, lap) pairs mostly from L1/L2, where neighbouring rows of
// the same CTA and the previous CTAs keep them.
//
// Storage relative to the local density.  Populations are kept as
// deviations g_i = f_i - W_i R(x) from the node's density R(x) of the step
// that wrote them (two density buffers alternate: the reference of the
// stored state and the density of the step being computed).  In the liquid
// (f_i ~ 7.5 W_i) a deviation from W_i alone would be ~6.5 W_i and every
// FP32 update would round at that magnitude; in a quasi-steady two-phase
// state those roundings repeat every step and add up to a net force on a
// periodic box.  With the local reference the stored values are O(u) W_i R
// in both phases.  The sweep brings the pulled values to its own node's
// reference, g_i + W_i (R(x - c_i) - R(x)), which is small except across the
// interface.
//
// Momentum balance.  Over a periodic box the mean-field force sums to zero
// in exact arithmetic (both terms are discrete divergences), so the total
// momentum changes by M g per step (M the mass).  In FP32 the roundings of
// the force, of the forcing term and of the stored values repeat from step
// to step in a quasi-steady state and add up to a net force: a liquid slab
// at rest accelerates by ~1e-9 per step.  Each sweep therefore sums the
// momentum of the populations it stores (one partial per CTA, reduced in a
// fixed order during the next step), and an acceleration a_c, whose force rho
// a_c is subtracted at every node in the next step, integrates the error:
//     a_c <- a_c + (P(t) - P(t-1) - M g) / M,
// so the momentum error of step t + 1 is the change of the rounding between
// consecutive steps and the error over many steps stays that of one step.
// (Taken per unit mass, the correction moves both phases alike.)  In exact
// arithmetic a_c stays zero.
//
// The fields stay valid until the next step; the force of the last step and
// the fluid velocity (j - F/2) / rho of its post-collision state are
// computed from them on request.
#include "kbc_collide.cuh"
#include "lbm_internal.h"
#include "sweep_io.cuh"

namespace kbc {

template <class C>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
};

// p(rho) of Eq. (eos) (a polynomial of degree six without constant term,
// evaluated by Horner's rule), or the ideal gas rho c_s^2 (then phi = 0).
template <class C>
__device__ __forceinline__ C mp_pressure(C r, int eos) {
  if (eos == MP_EOS_IDEAL) return r * (C)(1.0 / 3.0);
  C p = (C)1.2746947442749278e-5;
  p = p * r + (C)-1.4552652965531227e-4;
  p = p * r + (C)3.748484095210317e-4;
  p = p * r + (C)4.139745482116095e-3;
  p = p * r + (C)-3.818183621928911e-2;
  p = p * r + (C)5.3e-2;
  return p * r;
}

// Stored-space offsets of the three x columns, y rows and z planes around
// stored node (X, Y, Z) (periodic wrap): node (X + cx, Y + cy, Z + cz) is at
// xo[cx + 1] + yo[cy + 1] + zo[cz + 1].
template <int D, typename IX>
struct Nbhd {
  IX xo[3], yo[3], zo[3];
  __device__ __forceinline__ Nbhd(const Grid &g, int X, int Y, int Z) {
    xo[0] = (IX)nbr(X, -1, g.NX);
    xo[1] = (IX)X;
    xo[2] = (IX)nbr(X, 1, g.NX);
    yo[0] = (IX)nbr(Y, -1, g.NY) * (IX)g.pitch;
    yo[1] = (IX)Y * (IX)g.pitch;
    yo[2] = (IX)nbr(Y, 1, g.NY) * (IX)g.pitch;
    const IX plane = (IX)g.NY * (IX)g.pitch;
    zo[1] = (IX)Z * plane;
    zo[0] = zo[2] = zo[1];
    if (D == 3) {
      zo[0] = (IX)nbr(Z, -1, g.NZ) * plane;
      zo[2] = (IX)nbr(Z, 1, g.NZ) * plane;
    }
  }
  __device__ __forceinline__ IX at(int cx, int cy, int cz) const {
    return zo[cz + 1] + yo[cy + 1] + xo[cx + 1];
  }
};

// ---------------------------------------------------------------- momentum controller
// The sweep of step t leaves one (momentum, mass) partial per CTA; during
// step t + 1 the first CTAs of the density pass sum them in groups of
// kMpGroup (fixed order), and CTA 0 of the Laplacian pass sums the groups
// and updates the controller before the sweep of step t + 1 reads it.
// Stream order makes each stage's writes visible to the next: no atomics,
// no fences, a deterministic result.
// ctl: [0..2] the correcting acceleration a_c used by the current step,
// [6..8] the momentum of the step before, [9] the number of sweeps whose
// partials exist (0, 1, 2 = enough for an update), [10..11] a_c in FP32
// (three floats).
constexpr int kMpPartial = kMpPartialDoubles;  // per CTA: momentum (3), mass
constexpr int kMpGroup = kMpGroupCtas;

// Fixed-order sum of n values v[j * stride] (n <= kMpGroup) by the CTA into
// red[q]; every thread of the CTA calls it.
__device__ __forceinline__ void cta_sum_group(const double *__restrict__ src, long long stride,
                                              int n, double (&red)[kMpPartial][kMpGroup],
                                              double (&out)[kMpPartial]) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int q = 0; q < kMpPartial; ++q)
    for (int j = tid; j < kMpGroup; j += nthr) red[q][j] = j < n ? src[q * stride + j] : 0.0;
  __syncthreads();
  for (int h = kMpGroup / 2; h > 0; h >>= 1) {
    for (int q = 0; q < kMpPartial; ++q)
      for (int j = tid; j < h; j += nthr) red[q][j] += red[q][j + h];
    __syncthreads();
  }
  for (int q = 0; q < kMpPartial; ++q) out[q] = red[q][0];
}

// Stage 1 (density pass, CTAs b < ngroups): group sums of the CTA partials.
__device__ __forceinline__ void mp_stage1(const double *__restrict__ partial, long long nblk,
                                          double *__restrict__ gpart, long long blk) {
  const long long ngroups = (nblk + kMpGroup - 1) / kMpGroup;
  if (blk >= ngroups) return;
  __shared__ double red[kMpPartial][kMpGroup];
  double out[kMpPartial];
  const int n = (int)min((long long)kMpGroup, nblk - blk * kMpGroup);
  cta_sum_group(partial + blk * kMpGroup, nblk, n, red, out);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid < kMpPartial) gpart[tid * ngroups + blk] = out[tid];
}

// Stage 2 (Laplacian pass, CTA 0): total momentum and mass of the last
// sweep, controller update a_c <- a_c + (P(t) - P(t-1) - M g) / M.
__device__ __forceinline__ void mp_stage2(const double *__restrict__ gpart, long long nblk,
                                          double gx, double gy, double gz, double *ctl,
                                          long long blk) {
  if (blk != 0) return;
  const long long ngroups = (nblk + kMpGroup - 1) / kMpGroup;
  __shared__ double red[kMpPartial][kMpGroup];
  double tot[kMpPartial] = {0, 0, 0, 0};
  for (long long g0 = 0; g0 < ngroups; g0 += kMpGroup) {
    double part[kMpPartial];
    cta_sum_group(gpart + g0, ngroups, (int)min((long long)kMpGroup, ngroups - g0), red, part);
    for (int q = 0; q < kMpPartial; ++q) tot[q] += part[q];
    __syncthreads();
  }
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid == 0) {
    const double have = ctl[9];
    if (have >= 1.0) {
      const double M = tot[3], gg[3] = {gx, gy, gz};
      for (int a = 0; a < 3; ++a) {
        if (have >= 2.0) ctl[a] += (tot[a] - ctl[6 + a] - M * gg[a]) / M;
        ctl[6 + a] = tot[a];
      }
    }
    ctl[9] = have >= 1.0 ? 2.0 : 1.0;
    float *acf = reinterpret_cast<float *>(ctl + 10);  // FP32 copy for the sweep
    for (int a = 0; a < 3; ++a) acf[a] = (float)ctl[a];
  }
}

// The correcting acceleration of the current step in the compute type
// (FP32 sweeps read the FP32 copy at ctl[10..11]).
template <class C>
__device__ __forceinline__ C mp_ac(const double *ctl, int a);
template <>
__device__ __forceinline__ float mp_ac<float>(const double *ctl, int a) {
  return reinterpret_cast<const float *>(ctl + 10)[a];
}
template <>
__device__ __forceinline__ double mp_ac<double>(const double *ctl, int a) {
  return ctl[a];
}

// ---------------------------------------------------------------- walls
// Two planar walls half a cell outside the faces normal to axis wa (stored
// rows lo and hi are the first and last interior rows; the ghost rows lo - 1
// and hi + 1 hold, for the stencils, the fields of the row across the wall,
// and in their population slots the Grad-filled populations of the wall
// nodes).  kw: wetting strength.
template <class C>
struct MpWallT {
  int wa, lo, hi;
  C kw;
};
// -1 / +1 on the first / last interior row along the wall axis, else 0
template <class C>
__device__ __forceinline__ int mp_side(const MpWallT<C> &w, int X, int Y, int Z) {
  if (w.wa < 0) return 0;
  const int p = w.wa == 0 ? X : (w.wa == 1 ? Y : Z);
  return p == w.lo ? -1 : (p == w.hi ? 1 : 0);
}
// stored-index step along the wall axis
template <class C>
__device__ __forceinline__ long long mp_wall_stride(const Grid &g, const MpWallT<C> &w) {
  return w.wa == 0 ? 1LL : (w.wa == 1 ? (long long)g.pitch : (long long)g.pitch * g.NY);
}
// Wetting force F_s = kw rho sum_i W_i s(x + c_i) c_i: on the first row the
// ghost neighbours (c_wa = -1) weigh 1/6 in total, so F_s = -kw rho / 6
// along the wall normal; +kw rho / 6 on the last row.
template <class C>
__device__ __forceinline__ void mp_wet(const MpWallT<C> &w, int side, C r, C (&F)[3]) {
  if (side) F[w.wa] += (C)side * w.kw * r * (C)(1.0 / 6.0);
}

// ---------------------------------------------------------------- pass 1
// Pulled populations of a node as deviations from W_i R0 (R0 the node's new
// reference), the sources stored relative to their own references rref.
template <int Q, int S, typename IX>
__device__ __forceinline__ void mp_gather(const Grid &g, const typename Store<S>::T *__restrict__ fin,
                                          const typename Store<S>::C *__restrict__ rref,
                                          const Nbhd<Lat<Q>::D, IX> &nb, typename Store<S>::C R0,
                                          typename Store<S>::C (&v)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const IX N = (IX)g.N;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const IX src = nb.at(-L::cx(i), -L::cy(i), -L::cz(i));
    const C w = (C)weight<L>(i);
    v[i] = St::load(fin + ((IX)i * N + src), w) + w * (__ldg(rref + src) - R0);
  }
}

// WALL: the wall terms (ghost-row mirrors; the periodic instantiation
// compiles without them).
template <int Q, int S, typename IX, bool WALL>
__global__ void __launch_bounds__(128)
    k_mp_density(Grid g, const typename Store<S>::T *__restrict__ fin,
                 const typename Store<S>::C *__restrict__ rref,
                 typename Store<S>::C *__restrict__ rho,
                 typename Vec2<typename Store<S>::C>::T *__restrict__ pl, int eos,
                 const double *__restrict__ partial, double *__restrict__ gpart, long long nblk,
                 MpWallT<typename Store<S>::C> wl, int *__restrict__ err) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x < g.nx && y < g.ny) {
    using L = Lat<Q>;
    using St = Store<S>;
    const Nbhd<L::D, IX> nb(g, x + g.px, y + g.py, z + g.pz);
    const IX k = nb.at(0, 0, 0);
    // rho = sum_i g_i(x - c_i) + sum_i W_i R(x - c_i); the second sum is
    // the weighted neighbourhood mean of the reference densities, which the
    // Laplacian pass of the step that wrote them left at the node:
    // sum_i W_i R(x - c_i) = R(x) + lap R(x) / 6 (W_i = W_-i)
    const C R = rref[k];
    const C mean_ref = R + pl[k].y * (C)(1.0 / 6.0);
    const IX N = (IX)g.N;
    C d = (C)0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      d += St::load(fin + ((IX)i * N + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))), (C)weight<L>(i));
    const C r = mean_ref + d;
    if (!(r > (C)0 && r < (C)1e30)) atomicOr(err, 1);
    const C s = r * (C)(1.0 / 3.0) - mp_pressure(r, eos);
    const C ph = s > (C)0 ? sqrt(s) : (C)0;
    rho[k] = r;
    pl[k].x = ph;
    // the ghost row across a wall mirrors the first / last row
    if constexpr (WALL) {
      const int side = mp_side(wl, x + g.px, y + g.py, z + g.pz);
      if (side) {
        const long long kg = (long long)k + side * mp_wall_stride(g, wl);
        rho[kg] = r;
        pl[kg].x = ph;
      }
    }
  }
  mp_stage1(partial, nblk, gpart,
            ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------- pass 2
// lap rho = 6 (sum_i W_i rho(x + c_i) - rho(x)), the sum in tensor-product
// form: rows of three x-neighbours weighted by the D1Q3 weights w(c), then
// the rows by w(cy) w(cz).
template <int Q, class C, typename IX, bool WALL>
__device__ __forceinline__ void mp_lap_node(const Grid &g, const C *__restrict__ rho,
                                            typename Vec2<C>::T *__restrict__ pl, int x, int y,
                                            int z, const MpWallT<C> &wl) {
  using L = Lat<Q>;
  const Nbhd<L::D, IX> nb(g, x + g.px, y + g.py, z + g.pz);
  const IX k = nb.at(0, 0, 0);
  const C r0 = rho[k];
  C acc = (C)0;
#pragma unroll
  for (int cz = (L::D == 3 ? -1 : 0); cz <= (L::D == 3 ? 1 : 0); ++cz)
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy) {
      const IX row = nb.zo[cz + 1] + nb.yo[cy + 1];
      const C sw = (C)(1.0 / 6.0) * (__ldg(rho + row + nb.xo[0]) + __ldg(rho + row + nb.xo[2])) +
                   (C)(2.0 / 3.0) * __ldg(rho + row + nb.xo[1]);
      acc += (C)((L::D == 3 ? w1d(cz) : 1.0) * w1d(cy)) * sw;
    }
  const C lp = (C)6 * (acc - r0);
  pl[k].y = lp;
  if constexpr (WALL) {
    const int side = mp_side(wl, x + g.px, y + g.py, z + g.pz);
    if (side) pl[(long long)k + side * mp_wall_stride(g, wl)].y = lp;
  }
}

template <int Q, class C, typename IX, bool WALL>
__global__ void __launch_bounds__(128)
    k_mp_lap(Grid g, const C *__restrict__ rho, typename Vec2<C>::T *__restrict__ pl,
             const double *__restrict__ gpart, long long nblk, double gx, double gy, double gz,
             double *__restrict__ ctl, MpWallT<C> wl) {
  using L = Lat<Q>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x < g.nx && y < g.ny) mp_lap_node<Q, C, IX, WALL>(g, rho, pl, x, y, z, wl);
  // walls take momentum: the controller runs on fully periodic lattices only
  if constexpr (!WALL)
    mp_stage2(gpart, nblk, gx, gy, gz, ctl,
              ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// D3Q27 form marching along z: a thread takes a column of up to kz nodes of
// one (x, y) and keeps the weighted plane sums P(z) = sum_{cy} w(cy) S(cy, z)
// of three consecutive planes in registers, so each node costs the 9 loads of
// one new plane instead of 27 (lap rho = 6 (sum_cz w(cz) P(z + cz) - rho)).
template <class C, typename IX, bool WALL>
__global__ void __launch_bounds__(128)
    k_mp_lap_z(Grid g, const C *__restrict__ rho, typename Vec2<C>::T *__restrict__ pl,
               const double *__restrict__ gpart, long long nblk, double gx, double gy, double gz,
               double *__restrict__ ctl, MpWallT<C> wl, int kz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z0 = blockIdx.z * kz;
  if (x < g.nx && y < g.ny) {
    const int X = x + g.px, Y = y + g.py;
    const IX xo[3] = {(IX)nbr(X, -1, g.NX), (IX)X, (IX)nbr(X, 1, g.NX)};
    const IX yo[3] = {(IX)nbr(Y, -1, g.NY) * (IX)g.pitch, (IX)Y * (IX)g.pitch,
                      (IX)nbr(Y, 1, g.NY) * (IX)g.pitch};
    const IX plane = (IX)g.NY * (IX)g.pitch;
    auto psum = [&](int Zs) -> C {
      const IX base = (IX)Zs * plane;
      C acc = (C)0;
#pragma unroll
      for (int cy = 0; cy < 3; ++cy) {
        const IX row = base + yo[cy];
        const C sw = (C)(1.0 / 6.0) * (__ldg(rho + row + xo[0]) + __ldg(rho + row + xo[2])) +
                     (C)(2.0 / 3.0) * __ldg(rho + row + xo[1]);
        acc += (C)w1d(cy - 1) * sw;
      }
      return acc;
    };
    const int zend = min(z0 + kz, g.nz);
    C pm = psum(nbr(z0 + g.pz, -1, g.NZ)), p0 = psum(z0 + g.pz);
    for (int z = z0; z < zend; ++z) {
      const int Z = z + g.pz;
      const C pp = psum(nbr(Z, 1, g.NZ));
      const IX k = (IX)Z * plane + yo[1] + xo[1];
      const C lp = (C)6 * ((C)(1.0 / 6.0) * (pm + pp) + (C)(2.0 / 3.0) * p0 - rho[k]);
      pl[k].y = lp;
      if constexpr (WALL) {
        const int side = mp_side(wl, X, Y, Z);
        if (side) pl[(long long)k + side * mp_wall_stride(g, wl)].y = lp;
      }
      pm = p0;
      p0 = pp;
    }
  }
  if constexpr (!WALL)
    mp_stage2(gpart, nblk, gx, gy, gz, ctl,
              ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// F at a node from the fields: 2 phi d(phi) + kappa rho d(lap rho) + rho g.
// The lattice gradient d_a psi = 3 sum_i W_i c_ia psi(x + c_i) in
// tensor-product form (3 W_i c_ix = c_ix w(cy) w(cz) / 2):
//   d_x psi = 1/2 sum_{cy,cz} w(cy) w(cz) (psi(+1, cy, cz) - psi(-1, cy, cz)),
//   d_y psi = 1/2 sum_cz w(cz) (S(+1, cz) - S(-1, cz)),
//   d_z psi = 1/2 sum_cy w(cy) (S(cy, +1) - S(cy, -1)),
// S(cy, cz) = sum_cx w(cx) psi(cx, cy, cz) the weighted row sums.
template <int Q, class C, typename IX>
__device__ __forceinline__ void mp_force(const C *__restrict__ rho,
                                         const typename Vec2<C>::T *__restrict__ pl,
                                         const Nbhd<Lat<Q>::D, IX> &nb, C kappa, C gx, C gy,
                                         C gz, C &r, C (&F)[3]) {
  using L = Lat<Q>;
  using C2 = typename Vec2<C>::T;
  C dp[3] = {(C)0, (C)0, (C)0}, dl[3] = {(C)0, (C)0, (C)0};
#pragma unroll
  for (int cz = (L::D == 3 ? -1 : 0); cz <= (L::D == 3 ? 1 : 0); ++cz)
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy) {
      const IX row = nb.zo[cz + 1] + nb.yo[cy + 1];
      const C2 qm = __ldg(pl + row + nb.xo[0]);
      const C2 qp = __ldg(pl + row + nb.xo[2]);
      const C wyz = (C)(w1d(cy) * (L::D == 3 ? w1d(cz) : 1.0));
      dp[0] += wyz * (qp.x - qm.x);
      dl[0] += wyz * (qp.y - qm.y);
      if (cy == 0 && cz == 0) continue;  // the centre row enters d_x only
      const C2 q0 = __ldg(pl + row + nb.xo[1]);
      const C spx = (C)(1.0 / 6.0) * (qm.x + qp.x) + (C)(2.0 / 3.0) * q0.x;
      const C slx = (C)(1.0 / 6.0) * (qm.y + qp.y) + (C)(2.0 / 3.0) * q0.y;
      if (cy != 0) {
        const C w = (C)(cy * (L::D == 3 ? w1d(cz) : 1.0));
        dp[1] += w * spx;
        dl[1] += w * slx;
      }
      if (cz != 0) {
        const C w = (C)(cz * w1d(cy));
        dp[2] += w * spx;
        dl[2] += w * slx;
      }
    }
  const IX k = nb.at(0, 0, 0);
  r = rho[k];
  const C phi = pl[k].x;
  const C gg[3] = {gx, gy, gz};
#pragma unroll
  for (int a = 0; a < 3; ++a) F[a] = phi * dp[a] + (C)0.5 * kappa * r * dl[a] + r * gg[a];
  if (L::D == 2) F[2] = (C)0;
}

// ---------------------------------------------------------------- pass 3
// Sum of a[4] over the CTA into out[q * stride], fixed order: within each
// warp in the compute type A (FP64 arithmetic is scarce on this GPU; a
// rounding that repeats from step to step cancels in the controller's
// P(t) - P(t-1)), across the warps in FP64.
template <class A>
__device__ __forceinline__ void cta_sum4(A (&a)[kMpPartial], double *out, long long stride) {
  __shared__ double red[kMpPartial][32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < kMpPartial; ++q) {
    for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_down_sync(0xffffffffu, a[q], o);
    if (lane == 0) red[q][warp] = (double)a[q];
  }
  __syncthreads();
  if (tid < kMpPartial) {
    double t = 0;
    for (int w = 0; w < nw; ++w) t += red[tid][w];
    out[tid * stride] = t;
  }
}

// Resident 128-thread CTAs per SM the one-node forced sweep's registers
// are sized for (measured on the 320 x 250 x 320 droplet: 4 / 5 CTAs ->
// 2.63 / 2.68 ms per step; 5 spills ~130 bytes to L1).
#ifndef KBC_MP_CTAS
#define KBC_MP_CTAS 4
#endif
template <int Q, int S, typename IX, bool WALL>
__global__ void __launch_bounds__(128, KBC_MP_CTAS)
    k_mp_sweep(Grid g, const typename Store<S>::T *__restrict__ fin,
               typename Store<S>::T *__restrict__ fout, const typename Store<S>::C *__restrict__ rref,
               const typename Store<S>::C *__restrict__ rho,
               const typename Vec2<typename Store<S>::C>::T *__restrict__ pl,
               typename Store<S>::C beta, typename Store<S>::C kappa, typename Store<S>::C gx,
               typename Store<S>::C gy, typename Store<S>::C gz, int bgk,
               const double *__restrict__ ctl, double *__restrict__ partial, long long nblk,
               MpWallT<typename Store<S>::C> wl, int *__restrict__ err) {
  using L = Lat<Q>;
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool active = x < g.nx && y < g.ny;
  C part[kMpPartial] = {(C)0, (C)0, (C)0, (C)0};
  if (active) {
    const Nbhd<L::D, IX> nb(g, x + g.px, y + g.py, z + g.pz);
    const C ac[3] = {mp_ac<C>(ctl, 0), mp_ac<C>(ctl, 1), mp_ac<C>(ctl, 2)};
    C r, F[3];
    mp_force<Q, C, IX>(rho, pl, nb, kappa, gx, gy, gz, r, F);
    if constexpr (WALL) mp_wet(wl, mp_side(wl, x + g.px, y + g.py, z + g.pz), r, F);
    const C ir = (C)1 / r;
    C v[Q];
    // the new reference of the node: its density of this step
    mp_gather<Q, S, IX>(g, fin, rref, nb, r, v);
    // du = F / rho - a_c
    const C rc = collide_v<L, S == STORE_F32, C, true>(
        v, beta, bgk != 0, F[0] * ir - ac[0], F[1] * ir - ac[1],
        L::D == 3 ? F[2] * ir - ac[2] : (C)0, r);
    if (!(rc > (C)0 && rc < (C)1e30)) atomicOr(err, 1);
    sweep_scatter<Q, S, IX>(g, fout, nb.at(0, 0, 0), v);
    // momentum of the stored values (the reference carries none), by rows
    // of three x-neighbours
    C jx = (C)0, jy = (C)0, jz = (C)0;
#pragma unroll
    for (int rw = 0; rw < Q / 3; ++rw) {
      const int cy = L::cy(3 * rw), cz = L::cz(3 * rw);
      jx += v[3 * rw + 2] - v[3 * rw];
      if (cy || cz) {
        const C sm = v[3 * rw] + v[3 * rw + 1] + v[3 * rw + 2];
        if (cy > 0) jy += sm;
        if (cy < 0) jy -= sm;
        if (cz > 0) jz += sm;
        if (cz < 0) jz -= sm;
      }
    }
    part[0] = jx;
    part[1] = jy;
    part[2] = jz;
    part[3] = r;
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  cta_sum4(part, partial + blk, nblk);
}

// Two-node form of the forced sweep (FP32 storage): each thread takes the
// columns (X, X + 1), X even, of one row and collides both nodes on the
// paired FP32 instructions (collide_v with V = f2).  The c_x = 0 sources and
// the references of a pair are aligned two-element loads.  When X + 1 is
// past the row's last node the second lane repeats the first node's inputs
// and is never stored.
#ifndef KBC_MP_PAIR_CTAS
#define KBC_MP_PAIR_CTAS 2
#endif
template <int Q, typename IX, bool WALL>
__global__ void __launch_bounds__(128, KBC_MP_PAIR_CTAS)
    k_mp_sweep2(Grid g, const float *__restrict__ fin, float *__restrict__ fout,
                const float *__restrict__ rref, const float *__restrict__ rho,
                const float2 *__restrict__ pl, float beta, float kappa, float gx, float gy,
                float gz, int bgk, const double *__restrict__ ctl, double *__restrict__ partial,
                long long nblk, MpWallT<float> wl, int *__restrict__ err) {
  using L = Lat<Q>;
  using St = Store<STORE_F32>;
  const int x = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool ia = x < g.nx && y < g.ny;
  const bool ib = ia && x + 1 < g.nx;
  float part[kMpPartial] = {0.f, 0.f, 0.f, 0.f};
  if (ia) {
    const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
    const Nbhd<L::D, IX> na(g, X, Y, Z), nb(g, ib ? X + 1 : X, Y, Z);
    float ra, rb, Fa[3], Fb[3];
    mp_force<Q, float, IX>(rho, pl, na, kappa, gx, gy, gz, ra, Fa);
    mp_force<Q, float, IX>(rho, pl, nb, kappa, gx, gy, gz, rb, Fb);
    // the pair shares Y and Z, and walls normal to x are not paired
    if constexpr (WALL) {
      mp_wet(wl, mp_side(wl, X, Y, Z), ra, Fa);
      mp_wet(wl, mp_side(wl, ib ? X + 1 : X, Y, Z), rb, Fb);
    }
    const IX N = (IX)g.N;
    f2 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
      const float w = (float)weight<L>(i);
      const IX sa = na.at(-cx, -cy, -cz);
      float pa, pb, qa, qb;
      if (cx == 0 && ib) {
        // sources (X, X + 1) of the same row: one aligned pair each
        const float2 p2 = St::load2(fin + ((IX)i * N + sa), w);
        const float2 q2 = __ldg(reinterpret_cast<const float2 *>(rref + sa));
        pa = p2.x; pb = p2.y; qa = q2.x; qb = q2.y;
      } else {
        const IX sb = nb.at(-cx, -cy, -cz);
        pa = St::load(fin + ((IX)i * N + sa), w);
        pb = St::load(fin + ((IX)i * N + sb), w);
        qa = __ldg(rref + sa);
        qb = __ldg(rref + sb);
      }
      v[i] = mk2(fmaf(w, qa - ra, pa), fmaf(w, qb - rb, pb));
    }
    const float ia_r = 1.f / ra, ib_r = 1.f / rb;
    const float c0 = mp_ac<float>(ctl, 0), c1 = mp_ac<float>(ctl, 1), c2 = mp_ac<float>(ctl, 2);
    const f2 dux = mk2(Fa[0] * ia_r - c0, Fb[0] * ib_r - c0);
    const f2 duy = mk2(Fa[1] * ia_r - c1, Fb[1] * ib_r - c1);
    const f2 duz = L::D == 3 ? mk2(Fa[2] * ia_r - c2, Fb[2] * ib_r - c2) : mk2(0.f, 0.f);
    const f2 rc = collide_v<L, true, f2, true>(v, beta, bgk != 0, dux, duy, duz, mk2(ra, rb));
    if (!(rc.v.x > 0.f && rc.v.x < 1e30f) || (ib && !(rc.v.y > 0.f && rc.v.y < 1e30f)))
      atomicOr(err, 1);
    const IX k = na.at(0, 0, 0);
    if (ib) {
#pragma unroll
      for (int i = 0; i < Q; ++i) St::store2(fout + ((IX)i * N + k), v[i].v, 1.f);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) St::store(fout + ((IX)i * N + k), v[i].v.x, 1.f);
    }
    // momentum of the stored values, by rows of three x-neighbours
    f2 jx = mk2(0.f, 0.f), jy = jx, jz = jx;
#pragma unroll
    for (int rw = 0; rw < Q / 3; ++rw) {
      const int cy = L::cy(3 * rw), cz = L::cz(3 * rw);
      jx = vadd(jx, vsub(v[3 * rw + 2], v[3 * rw]));
      if (cy || cz) {
        const f2 sm = vadd(vadd(v[3 * rw], v[3 * rw + 1]), v[3 * rw + 2]);
        if (cy > 0) jy = vadd(jy, sm);
        if (cy < 0) jy = vsub(jy, sm);
        if (cz > 0) jz = vadd(jz, sm);
        if (cz < 0) jz = vsub(jz, sm);
      }
    }
    part[0] = jx.v.x + (ib ? jx.v.y : 0.f);
    part[1] = jy.v.x + (ib ? jy.v.y : 0.f);
    part[2] = jz.v.x + (ib ? jz.v.y : 0.f);
    part[3] = ra + (ib ? rb : 0.f);
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  cta_sum4(part, partial + blk, nblk);
}

// Read-out of the stored state for interior nodes [begin, begin + count),
// output index j = node - begin.
//   F (optional): the force of the last step, F[a * stride + j], FP64;
//   rho_out, u (optional): density R + sum g_i and fluid velocity
//     (j - F/2) / rho of the stored post-collision state (F = 0 when
//     !have_force), u[a * stride + j];
//   fabs (optional): absolute populations f_i = g_i + W_i R of the interface
//     layout, fabs[i * stride + j], FP64.
template <int Q, int S, class O>
__global__ void k_mp_read(Grid g, const typename Store<S>::T *__restrict__ f,
                          const typename Store<S>::C *__restrict__ rref,
                          const typename Vec2<typename Store<S>::C>::T *__restrict__ pl,
                          typename Store<S>::C kappa, typename Store<S>::C gx,
                          typename Store<S>::C gy, typename Store<S>::C gz, int have_force,
                          const double *__restrict__ mean, MpWallT<typename Store<S>::C> wl,
                          long long begin, long long count, long long stride, double *F,
                          O *rho_out, O *u, double *fabs) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= count) return;
  const long long n = begin + j;
  const int X = (int)(n % g.nx) + g.px;
  const int Y = (int)((n / g.nx) % g.ny) + g.py;
  const int Z = (int)(n / ((long long)g.nx * g.ny)) + g.pz;
  const long long k = sidx(g, X, Y, Z);
  C Fv[3] = {(C)0, (C)0, (C)0}, rdummy;
  if (have_force) {
    const Nbhd<L::D, long long> nb(g, X, Y, Z);
    mp_force<Q, C, long long>(rref, pl, nb, kappa, gx, gy, gz, rdummy, Fv);
    mp_wet(wl, mp_side(wl, X, Y, Z), rdummy, Fv);
    // the correcting force the step used
    for (int a = 0; a < L::D; ++a) Fv[a] -= rdummy * (C)mean[a];
  }
  if (F)
    for (int a = 0; a < 3; ++a) F[a * stride + j] = (double)Fv[a];
  const C R = rref[k];
  if (fabs)
    for (int i = 0; i < Q; ++i)
      fabs[i * stride + j] = (double)St::load(f + (long long)i * g.N + k, (C)weight<L>(i)) +
                             weight<L>(i) * (double)R;
  if (rho_out) {
    double d = 0, jx = 0, jy = 0, jz = 0;
    for (int i = 0; i < Q; ++i) {
      const double v = (double)St::load(f + (long long)i * g.N + k, (C)weight<L>(i));
      d += v;
      jx += L::cx(i) * v;
      jy += L::cy(i) * v;
      jz += L::cz(i) * v;
    }
    const double r = (double)R + d;
    rho_out[j] = (O)r;
    const double ja[3] = {jx, jy, jz};
    for (int a = 0; a < L::D; ++a) u[a * stride + j] = (O)((ja[a] - 0.5 * (double)Fv[a]) / r);
  }
}

// Reference changes of the stored state: g_i += W_i (R(x) - Rnew) in place,
// and R(x) := Rnew (1 when a state is set from outside or the model is
// switched off, so that the single-phase kernels read it).
template <int Q, int S>
__global__ void k_mp_rebase(Grid g, typename Store<S>::T *__restrict__ f,
                            typename Store<S>::C *__restrict__ rref, typename Store<S>::C Rnew,
                            int shift_populations) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= (long long)g.nx * g.ny * g.nz) return;
  const int X = (int)(n % g.nx) + g.px;
  const int Y = (int)((n / g.nx) % g.ny) + g.py;
  const int Z = (int)(n / ((long long)g.nx * g.ny)) + g.pz;
  const long long k = sidx(g, X, Y, Z);
  const C R = rref[k];
  if (shift_populations)
    for (int i = 0; i < Q; ++i) {
      const C w = (C)weight<L>(i);
      St::store(f + (long long)i * g.N + k, St::load(f + (long long)i * g.N + k, w) + w * (R - Rnew),
                (C)(1.0 / weight<L>(i)));
    }
  rref[k] = Rnew;
}

// rref := Rnew over every stored node (ghost rows and row padding included:
// the ghost slots of a wall are filled relative to their reference).
template <class C>
__global__ void k_mp_fill_ref(C *__restrict__ rref, long long N, C Rnew) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < N) rref[k] = Rnew;
}

// ---------------------------------------------------------------- wall fill
// Grad's approximation for the populations that the wall nodes (first and
// last interior rows along the wall axis) miss, written into the ghost slots
// they pull from.  Readings (as for face walls at q = 1/2, at rest): rho_t =
// the known pulled populations plus the node's own stored f'_opp(i); u_t =
// mean over the missing set of u(x_b + c_i) / 3, minus F_prev(x_b) / (2
// rho_t) (the pulled populations carry rho u - F/2); grad u of the fluid
// velocity by central differences along the wall, one-sided second order
// across it; Pi = rho c_s^2 I + rho u u - rho c_s^2/(2 beta)(grad u + grad
// u^T).  u(x) = (j' - F_prev/2) / rho' of the stored state, F_prev the force
// of the step that produced it (zero without one).
//
// Band scratch: band[((s * 3 + r) * 6 + q) * plane + p], side s (0: first
// rows, 1: last rows), row r from the wall, q = 0..2 the velocity and 3..5
// the force, p = t1 + n[a1] t2 over the two other axes a1 < a2.
struct MpPlane {
  int wa, a1, a2, n[3], pad[3];
  long long plane;
};
__device__ __forceinline__ void mp_plane_node(const MpPlane &pl, int s, int r, long long p,
                                              int (&X)[3]) {
  const int t1 = (int)(p % pl.n[pl.a1]), t2 = (int)(p / pl.n[pl.a1]);
  X[pl.a1] = t1 + pl.pad[pl.a1];
  X[pl.a2] = t2 + pl.pad[pl.a2];
  X[pl.wa] = pl.pad[pl.wa] + (s == 0 ? r : pl.n[pl.wa] - 1 - r);
}

template <int Q, int S, typename IX>
__global__ void __launch_bounds__(128)
    k_mp_wall_band(Grid g, const typename Store<S>::T *__restrict__ f,
                   const typename Store<S>::C *__restrict__ rref,
                   const typename Vec2<typename Store<S>::C>::T *__restrict__ fields,
                   typename Store<S>::C kappa, typename Store<S>::C gx, typename Store<S>::C gy,
                   typename Store<S>::C gz, MpWallT<typename Store<S>::C> wl, MpPlane mpl,
                   int have_force, typename Store<S>::C *__restrict__ band) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 2 * kMpBandRows * mpl.plane) return;
  const int sr = (int)(t / mpl.plane);
  const int s = sr / kMpBandRows, r = sr % kMpBandRows;
  const long long p = t % mpl.plane;
  int X[3];
  mp_plane_node(mpl, s, r, p, X);
  const Nbhd<L::D, IX> nb(g, X[0], X[1], X[2]);
  const IX k = nb.at(0, 0, 0);
  C d = (C)0, j[3] = {(C)0, (C)0, (C)0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const C v = St::load(f + ((IX)i * (IX)g.N + k), (C)weight<L>(i));
    d += v;
    j[0] += (C)L::cx(i) * v;
    j[1] += (C)L::cy(i) * v;
    j[2] += (C)L::cz(i) * v;
  }
  const C rs = rref[k] + d;  // density of the stored state
  C F[3] = {(C)0, (C)0, (C)0};
  if (have_force) {
    C rf;
    mp_force<Q, C, IX>(rref, fields, nb, kappa, gx, gy, gz, rf, F);
    mp_wet(wl, mp_side(wl, X[0], X[1], X[2]), rf, F);
  }
  C *out = band + (long long)sr * 6 * mpl.plane + p;
  for (int a = 0; a < 3; ++a) {
    out[a * mpl.plane] = (j[a] - (C)0.5 * F[a]) / rs;
    out[(3 + a) * mpl.plane] = F[a];
  }
}

template <int Q, int S, typename IX>
__global__ void __launch_bounds__(128)
    k_mp_wall_fill(Grid g, typename Store<S>::T *__restrict__ f,
                   const typename Store<S>::C *__restrict__ rref,
                   const typename Store<S>::C *__restrict__ band, MpPlane mpl,
                   typename Store<S>::C beta) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 2 * mpl.plane) return;
  const int s = (int)(t / mpl.plane);
  const long long p = t % mpl.plane;
  int X[3];
  mp_plane_node(mpl, s, 0, p, X);
  const Nbhd<L::D, IX> nb(g, X[0], X[1], X[2]);
  const IX k = nb.at(0, 0, 0);
  const IX N = (IX)g.N;
  const int inward = s == 0 ? 1 : -1;  // stored-coordinate direction away from the wall
  const int t1 = (int)(p % mpl.n[mpl.a1]), t2 = (int)(p / mpl.n[mpl.a1]);
  // band value q of row r at tangential offsets (o1, o2), periodic along the wall
  auto bv = [&](int r, int o1, int o2, int q) -> C {
    int u1 = t1 + o1, u2 = t2 + o2;
    const int n1 = mpl.n[mpl.a1], n2 = mpl.n[mpl.a2];
    u1 = u1 < 0 ? u1 + n1 : (u1 >= n1 ? u1 - n1 : u1);
    u2 = u2 < 0 ? u2 + n2 : (u2 >= n2 ? u2 - n2 : u2);
    return band[((long long)(s * kMpBandRows + r) * 6 + q) * mpl.plane + u1 +
                (long long)n1 * u2];
  };
  auto cax = [&](int i, int a) { return a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i)); };
  const C R = rref[k];
  C rho_t = (C)0, ut[3] = {(C)0, (C)0, (C)0};
  int nmiss = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const C w = (C)weight<L>(i);
    if (cax(i, mpl.wa) == inward) {  // the source x_b - c_i lies beyond the wall
      ++nmiss;
      rho_t += St::load(f + ((IX)(Q - 1 - i) * N + k), w) + w * R;
      for (int a = 0; a < 3; ++a)
        ut[a] += bv(1, cax(i, mpl.a1), cax(i, mpl.a2), a) * (C)(1.0 / 3.0);
    } else {
      const IX src = nb.at(-L::cx(i), -L::cy(i), -L::cz(i));
      rho_t += St::load(f + ((IX)i * N + src), w) + w * __ldg(rref + src);
    }
  }
  const C im = (C)1 / (C)nmiss;
  for (int a = 0; a < 3; ++a) ut[a] = ut[a] * im - (C)0.5 * bv(0, 0, 0, 3 + a) / rho_t;
  // grad u, G[a][b] = d u_a / d x_b
  C G[3][3] = {{(C)0, (C)0, (C)0}, {(C)0, (C)0, (C)0}, {(C)0, (C)0, (C)0}};
  for (int b = 0; b < L::D; ++b)
    for (int a = 0; a < 3; ++a) {
      if (b == mpl.wa) {
        const C u0 = bv(0, 0, 0, a), u1 = bv(1, 0, 0, a), u2 = bv(2, 0, 0, a);
        G[a][b] = (C)(0.5 * inward) * ((C)-3 * u0 + (C)4 * u1 - u2);
      } else {
        const int o1 = b == mpl.a1 ? 1 : 0, o2 = b == mpl.a2 ? 1 : 0;
        G[a][b] = (C)0.5 * (bv(0, o1, o2, a) - bv(0, -o1, -o2, a));
      }
    }
  const C cs2 = (C)(1.0 / 3.0);
  C Pn[3][3];  // Pi - rho c_s^2 I
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Pn[a][b] = rho_t * ut[a] * ut[b] - rho_t * cs2 / ((C)2 * beta) * (G[a][b] + G[b][a]);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (cax(i, mpl.wa) != inward) continue;
    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
    C cu = (C)0, contr = (C)0;
    for (int a = 0; a < 3; ++a) cu += (C)c[a] * ut[a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        contr += Pn[a][b] * ((C)(c[a] * c[b]) - (a == b ? cs2 : (C)0));
    const C w = (C)weight<L>(i);
    const C fs = w * (rho_t + rho_t * cu / cs2 + contr / ((C)2 * cs2 * cs2));
    const IX src = nb.at(-c[0], -c[1], -c[2]);  // the ghost slot it is pulled from
    St::store(f + ((IX)i * N + src), fs - w * __ldg(rref + src), (C)(1.0 / weight<L>(i)));
  }
}

// ---------------------------------------------------------------- launchers
static dim3 mp_block(const Grid &g) {
  const MpGrid m = mp_grid(g.nx, g.ny, g.nz);
  return dim3(m.bx, m.by, 1);
}

// Wall description of a grid for the kernels (wa < 0: fully periodic).
template <class C>
static MpWallT<C> mp_wall_of(const Grid &g, const MpParams &mp) {
  MpWallT<C> w;
  w.wa = mp.wall;
  w.kw = (C)mp.kappa_w;
  w.lo = w.hi = -1;
  if (mp.wall >= 0) {
    const int n[3] = {g.nx, g.ny, g.nz}, pad[3] = {g.px, g.py, g.pz};
    w.lo = pad[mp.wall];
    w.hi = pad[mp.wall] + n[mp.wall] - 1;
  }
  return w;
}
static MpPlane mp_plane_of(const Grid &g, int wa) {
  MpPlane m;
  m.wa = wa;
  m.a1 = wa == 0 ? 1 : 0;
  m.a2 = wa == 2 ? 1 : 2;
  m.n[0] = g.nx; m.n[1] = g.ny; m.n[2] = g.nz;
  m.pad[0] = g.px; m.pad[1] = g.py; m.pad[2] = g.pz;
  m.plane = (long long)m.n[m.a1] * m.n[m.a2];
  return m;
}

// z-nodes per thread of the marching Laplacian pass
#ifndef KBC_MP_LAP_COLUMN
#define KBC_MP_LAP_COLUMN 16
#endif
constexpr int kMpLapColumn = KBC_MP_LAP_COLUMN;

template <int Q, int S, typename IX, bool WALL>
static void mp_launch_all(const Grid &g, void *fin, void *fout, const void *rref, void *rho,
                          void *pl, double *ctl, double *partial, double *gpart, void *band,
                          int have_force, const MpParams &mp, double beta, int bgk, int *err,
                          cudaStream_t s) {
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  using C2 = typename Vec2<C>::T;
  const MpWallT<C> wl = mp_wall_of<C>(g, mp);
  const dim3 b = mp_block(g);
  const dim3 grid((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
  const long long nblk = (long long)grid.x * grid.y * grid.z;
  // the sweep: two-node form for FP32 storage when x is periodic (its pairs
  // start on even stored columns), with its own CTA grid
  const bool pair = S == STORE_F32 && mp.pair && g.px == 0;
  const int npairs = (g.nx + 1) / 2;
  const dim3 b2 = npairs >= 128 ? dim3(128, 1, 1) : dim3(32, 4, 1);
  const dim3 grid2((npairs + b2.x - 1) / b2.x, (g.ny + b2.y - 1) / b2.y, g.nz);
  const long long nblk_sweep = pair ? (long long)grid2.x * grid2.y * grid2.z : nblk;
  if constexpr (WALL) {
    // Grad fill of the wall nodes' missing populations (into fin's ghost slots)
    const MpPlane mpl = mp_plane_of(g, mp.wall);
    const long long nb_band = 2 * kMpBandRows * mpl.plane, nb_fill = 2 * mpl.plane;
    k_mp_wall_band<Q, S, IX><<<(unsigned)((nb_band + 127) / 128), 128, 0, s>>>(
        g, (const T *)fin, (const C *)rref, (const C2 *)pl, (C)mp.kappa, (C)mp.g[0], (C)mp.g[1],
        (C)mp.g[2], wl, mpl, have_force, (C *)band);
    k_mp_wall_fill<Q, S, IX><<<(unsigned)((nb_fill + 127) / 128), 128, 0, s>>>(
        g, (T *)fin, (const C *)rref, (const C *)band, mpl, (C)beta);
  }
  k_mp_density<Q, S, IX, WALL><<<grid, b, 0, s>>>(g, (const T *)fin, (const C *)rref, (C *)rho,
                                            (C2 *)pl, mp.eos, partial, gpart, nblk_sweep, wl, err);
  if (Q == 27 && g.nz >= 2 * kMpLapColumn) {
    const dim3 gz(grid.x, grid.y, (g.nz + kMpLapColumn - 1) / kMpLapColumn);
    k_mp_lap_z<C, IX, WALL><<<gz, b, 0, s>>>(g, (const C *)rho, (C2 *)pl, gpart, nblk_sweep,
                                             mp.g[0], mp.g[1], mp.g[2], ctl, wl, kMpLapColumn);
  } else {
    k_mp_lap<Q, C, IX, WALL><<<grid, b, 0, s>>>(g, (const C *)rho, (C2 *)pl, gpart, nblk_sweep,
                                                mp.g[0], mp.g[1], mp.g[2], ctl, wl);
  }
  if (pair) {
    if constexpr (S == STORE_F32)
      k_mp_sweep2<Q, IX, WALL><<<grid2, b2, 0, s>>>(
          g, (const float *)fin, (float *)fout, (const float *)rref, (const float *)rho,
          (const float2 *)pl, (float)beta, (float)mp.kappa, (float)mp.g[0], (float)mp.g[1],
          (float)mp.g[2], bgk, ctl, partial, nblk_sweep, wl, err);
  } else {
    k_mp_sweep<Q, S, IX, WALL><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, (const C *)rref,
                                            (const C *)rho, (const C2 *)pl, (C)beta, (C)mp.kappa,
                                            (C)mp.g[0], (C)mp.g[1], (C)mp.g[2], bgk, ctl, partial,
                                            nblk_sweep, wl, err);
  }
}

template <int Q, int S>
static cudaError_t mp_step_t(const Grid &g, void *fin, void *fout, const void *rref, void *rho,
                             void *pl, double *ctl, double *partial, void *band, int have_force,
                             const MpParams &mp, double beta, int bgk, int *err, cudaStream_t s) {
  // partial: [4][nblk] CTA sums of the sweep, then [4][ngroups] group sums
  double *gpart = partial + kMpPartial * mp_grid(g.nx, g.ny, g.nz).blocks;
  // 32-bit offsets when every population offset fits
  const bool narrow = (long long)Q * g.N < (1LL << 31);
  if (narrow && mp.wall < 0)
    mp_launch_all<Q, S, int, false>(g, fin, fout, rref, rho, pl, ctl, partial, gpart, band,
                                    have_force, mp, beta, bgk, err, s);
  else if (narrow)
    mp_launch_all<Q, S, int, true>(g, fin, fout, rref, rho, pl, ctl, partial, gpart, band,
                                   have_force, mp, beta, bgk, err, s);
  else if (mp.wall < 0)
    mp_launch_all<Q, S, long long, false>(g, fin, fout, rref, rho, pl, ctl, partial, gpart, band,
                                          have_force, mp, beta, bgk, err, s);
  else
    mp_launch_all<Q, S, long long, true>(g, fin, fout, rref, rho, pl, ctl, partial, gpart, band,
                                         have_force, mp, beta, bgk, err, s);
  return cudaGetLastError();
}

#define MP_DISPATCH(Q, storage, ...)                                                  \
  do {                                                                                \
    if (Q == 9 && storage == STORE_F32) { constexpr int QQ = 9, SS = STORE_F32; __VA_ARGS__; }   \
    if (Q == 9 && storage == STORE_F64) { constexpr int QQ = 9, SS = STORE_F64; __VA_ARGS__; }   \
    if (Q == 27 && storage == STORE_F32) { constexpr int QQ = 27, SS = STORE_F32; __VA_ARGS__; } \
    return cudaErrorInvalidValue;                                                     \
  } while (0)

cudaError_t launch_mp_step(int Q, int storage, const Grid &g, void *fin, void *fout,
                           const void *rref, void *rho, void *pl, double *ctl, double *partial,
                           void *band, int have_force, const MpParams &mp, double beta, int bgk,
                           int *err, cudaStream_t s) {
  MP_DISPATCH(Q, storage, return (mp_step_t<QQ, SS>(g, fin, fout, rref, rho, pl, ctl, partial,
                                                    band, have_force, mp, beta, bgk, err, s)));
}

template <int Q, int S, class O>
static cudaError_t mp_read_t(const Grid &g, const void *f, const void *rref, const void *pl,
                             const MpParams &mp, int have_force, const double *mean,
                             long long begin, long long count,
                             long long stride, double *F, O *rho_out, O *u, double *fabs,
                             cudaStream_t s) {
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  using C2 = typename Vec2<C>::T;
  if (count <= 0) return cudaSuccess;
  const int b = 256;
  k_mp_read<Q, S, O><<<(unsigned)((count + b - 1) / b), b, 0, s>>>(
      g, (const T *)f, (const C *)rref, (const C2 *)pl, (C)mp.kappa, (C)mp.g[0], (C)mp.g[1],
      (C)mp.g[2], have_force, mean, mp_wall_of<C>(g, mp), begin, count, stride, F, rho_out, u,
      fabs);
  return cudaGetLastError();
}

cudaError_t launch_mp_read(int Q, int storage, const Grid &g, const void *f, const void *rref,
                           const void *pl, const MpParams &mp, int have_force,
                           const double *mean, long long begin,
                           long long count, long long stride, double *F, double *rho_out,
                           double *u, float *rho32, float *u32, double *fabs, cudaStream_t s) {
  if (rho32)
    MP_DISPATCH(Q, storage, return (mp_read_t<QQ, SS, float>(g, f, rref, pl, mp, have_force, mean, begin,
                                                             count, stride, F, rho32, u32, fabs, s)));
  MP_DISPATCH(Q, storage, return (mp_read_t<QQ, SS, double>(g, f, rref, pl, mp, have_force, mean, begin,
                                                            count, stride, F, rho_out, u, fabs, s)));
}

cudaError_t launch_mp_rebase(int Q, int storage, const Grid &g, void *f, void *rref, double Rnew,
                             int shift_populations, cudaStream_t s) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const int b = 256;
  const unsigned nb = (unsigned)((n + b - 1) / b);
  MP_DISPATCH(Q, storage, {
    using T = typename Store<SS>::T;
    using C = typename Store<SS>::C;
    k_mp_rebase<QQ, SS><<<nb, b, 0, s>>>(g, (T *)f, (C *)rref, (C)Rnew, shift_populations);
    k_mp_fill_ref<C><<<(unsigned)((g.N + b - 1) / b), b, 0, s>>>((C *)rref, g.N, (C)Rnew);
    return cudaGetLastError();
  });
}

}  // namespace kbc
