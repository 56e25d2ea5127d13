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
// momentum of the populations it stores (per-CTA partials in FP64, one CTA
// reducing them in a fixed order), and an acceleration a_c, whose force rho
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

// ---------------------------------------------------------------- pass 1
// Pulled populations of stored node (X, Y, Z) as deviations from W_i R0 (R0
// the node's new reference; R0 = 0 gives absolute values), the sources
// stored relative to their own references rref.
template <int Q, int S>
__device__ __forceinline__ void mp_gather(const Grid &g, const typename Store<S>::T *__restrict__ fin,
                                          const typename Store<S>::C *__restrict__ rref, int X,
                                          int Y, int Z, typename Store<S>::C R0,
                                          typename Store<S>::C (&v)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
  using C = typename St::C;
  const int xs[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};  // source x for cx = -1, 0, +1
  const int ys[3] = {nbr(Y, 1, g.NY), Y, nbr(Y, -1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, 1, g.NZ);
    zs[2] = nbr(Z, -1, g.NZ);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long src = ((long long)zs[L::cz(i) + 1] * g.NY + ys[L::cy(i) + 1]) * g.pitch +
                          xs[L::cx(i) + 1];
    const C w = (C)weight<L>(i);
    v[i] = St::load(fin + ((long long)i * g.N + src), w) + w * (__ldg(rref + src) - R0);
  }
}

template <int Q, int S>
__global__ void __launch_bounds__(128)
    k_mp_density(Grid g, const typename Store<S>::T *__restrict__ fin,
                 const typename Store<S>::C *__restrict__ rref,
                 typename Store<S>::C *__restrict__ rho,
                 typename Vec2<typename Store<S>::C>::T *__restrict__ pl, int eos,
                 int *__restrict__ err) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
  const long long k = sidx(g, X, Y, Z);
  // deviations from the node's own old reference keep the sum small
  const C R = rref[k];
  C v[Q];
  mp_gather<Q, S>(g, fin, rref, X, Y, Z, R, v);
  C d = (C)0;
#pragma unroll
  for (int i = 0; i < Q; ++i) d += v[i];
  const C r = R + d;
  if (!(r > (C)0 && r < (C)1e30)) atomicOr(err, 1);
  const C s = r * (C)(1.0 / 3.0) - mp_pressure(r, eos);
  rho[k] = r;
  pl[k].x = s > (C)0 ? sqrt(s) : (C)0;
}

// ---------------------------------------------------------------- pass 2
template <int Q, class C>
__global__ void __launch_bounds__(128)
    k_mp_lap(Grid g, const C *__restrict__ rho, typename Vec2<C>::T *__restrict__ pl) {
  using L = Lat<Q>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
  const int xs[3] = {nbr(X, -1, g.NX), X, nbr(X, 1, g.NX)};  // x + c for c = -1, 0, +1
  const int ys[3] = {nbr(Y, -1, g.NY), Y, nbr(Y, 1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, -1, g.NZ);
    zs[2] = nbr(Z, 1, g.NZ);
  }
  const long long k = sidx(g, X, Y, Z);
  const C r0 = rho[k];
  C acc = (C)0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
    const long long kn = sidx(g, xs[L::cx(i) + 1], ys[L::cy(i) + 1], zs[L::cz(i) + 1]);
    acc += (C)weight<L>(i) * (__ldg(rho + kn) - r0);
  }
  pl[k].y = (C)6 * acc;
}

// F at stored node (X, Y, Z) from the fields: 2 phi d(phi) + kappa rho
// d(lap rho) + rho g.  The lattice gradient in tensor-product form:
// d_x psi = 1/2 sum_{cy,cz} w(cy) w(cz) (psi(x+1, .) - psi(x-1, .)), w the
// D1Q3 weights (3 W_i c_ix = c_ix w(cy) w(cz) / 2).
template <int Q, class C>
__device__ __forceinline__ void mp_force(const Grid &g, const C *__restrict__ rho,
                                         const typename Vec2<C>::T *__restrict__ pl, C kappa,
                                         C gx, C gy, C gz, int X, int Y, int Z, C &r, C (&F)[3]) {
  using L = Lat<Q>;
  const int xs[3] = {nbr(X, -1, g.NX), X, nbr(X, 1, g.NX)};
  const int ys[3] = {nbr(Y, -1, g.NY), Y, nbr(Y, 1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, -1, g.NZ);
    zs[2] = nbr(Z, 1, g.NZ);
  }
  C gp[3] = {(C)0, (C)0, (C)0}, gl[3] = {(C)0, (C)0, (C)0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    if (cx == 0 && cy == 0 && cz == 0) continue;
    const long long kn = sidx(g, xs[cx + 1], ys[cy + 1], zs[cz + 1]);
    const typename Vec2<C>::T q = __ldg(pl + kn);
    const C w3 = (C)(3.0 * weight<L>(i));
    if (cx) { gp[0] += (C)cx * w3 * q.x; gl[0] += (C)cx * w3 * q.y; }
    if (cy) { gp[1] += (C)cy * w3 * q.x; gl[1] += (C)cy * w3 * q.y; }
    if (cz) { gp[2] += (C)cz * w3 * q.x; gl[2] += (C)cz * w3 * q.y; }
  }
  const long long k = sidx(g, X, Y, Z);
  r = rho[k];
  const C phi = pl[k].x;
  const C gg[3] = {gx, gy, gz};
#pragma unroll
  for (int a = 0; a < 3; ++a) F[a] = (C)2 * phi * gp[a] + kappa * r * gl[a] + r * gg[a];
  if (L::D == 2) F[2] = (C)0;
}

// ---------------------------------------------------------------- pass 3
// Sum of a[4] over the CTA into out[4] (FP64, fixed order).
constexpr int kMpPartial = kMpPartialDoubles;  // per CTA: momentum (3), mass
__device__ __forceinline__ void cta_sum4(double (&a)[kMpPartial], double *out) {
  __shared__ double red[kMpPartial][32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < kMpPartial; ++q) {
    for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_down_sync(0xffffffffu, a[q], o);
    if (lane == 0) red[q][warp] = a[q];
  }
  __syncthreads();
  if (tid < kMpPartial) {
    double t = 0;
    for (int w = 0; w < nw; ++w) t += red[tid][w];
    out[tid] = t;
  }
}

template <int Q, int S>
__global__ void __launch_bounds__(128, 4)
    k_mp_sweep(Grid g, const typename Store<S>::T *__restrict__ fin,
               typename Store<S>::T *__restrict__ fout, const typename Store<S>::C *__restrict__ rref,
               const typename Store<S>::C *__restrict__ rho,
               const typename Vec2<typename Store<S>::C>::T *__restrict__ pl,
               typename Store<S>::C beta, typename Store<S>::C kappa, typename Store<S>::C gx,
               typename Store<S>::C gy, typename Store<S>::C gz, int bgk,
               const double *__restrict__ ctl, double *__restrict__ partial,
               int *__restrict__ err) {
  using L = Lat<Q>;
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool active = x < g.nx && y < g.ny;
  double part[kMpPartial] = {0, 0, 0, 0};
  if (active) {
    const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
    C r, F[3];
    mp_force<Q, C>(g, rho, pl, kappa, gx, gy, gz, X, Y, Z, r, F);
    const C ir = (C)1 / r;
    C v[Q];
    // the new reference of the node: its density of this step
    mp_gather<Q, S>(g, fin, rref, X, Y, Z, r, v);
    // du = F / rho - a_c
    const C rc = collide_v<L, S == STORE_F32, C, true>(
        v, beta, bgk != 0, F[0] * ir - (C)ctl[0], F[1] * ir - (C)ctl[1],
        L::D == 3 ? F[2] * ir - (C)ctl[2] : (C)0, r);
    if (!(rc > (C)0 && rc < (C)1e30)) atomicOr(err, 1);
    sweep_scatter<Q, S, long long>(g, fout, sidx(g, X, Y, Z), v);
    // momentum of the stored values (the reference carries none)
    C jx = (C)0, jy = (C)0, jz = (C)0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::cx(i)) jx += (C)L::cx(i) * v[i];
      if (L::cy(i)) jy += (C)L::cy(i) * v[i];
      if (L::cz(i)) jz += (C)L::cz(i) * v[i];
    }
    part[0] = (double)jx;
    part[1] = (double)jy;
    part[2] = (double)jz;
    part[3] = (double)r;
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  cta_sum4(part, partial + kMpPartial * blk);
}

// Momentum controller (one CTA, fixed order).  ctl: [0..2] the correcting
// acceleration a_c of the next step, [3..5] the one the last step used,
// [6..8] the momentum P of the previous step, [9] 1 once P is recorded.
__global__ void __launch_bounds__(256) k_mp_control(const double *__restrict__ partial,
                                                    long long nblk, double gx,
                                                    double gy, double gz, double *__restrict__ ctl) {
  __shared__ double red[kMpPartial][256];
  double t[kMpPartial] = {0, 0, 0, 0};
  for (long long b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int q = 0; q < kMpPartial; ++q) t[q] += partial[kMpPartial * b + q];
  for (int q = 0; q < kMpPartial; ++q) red[q][threadIdx.x] = t[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < kMpPartial; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double M = red[3][0], gg[3] = {gx, gy, gz};
    const bool have_prev = ctl[9] != 0.0;
    for (int a = 0; a < 3; ++a) {
      const double P = red[a][0];
      ctl[3 + a] = ctl[a];
      if (have_prev) ctl[a] += (P - ctl[6 + a] - M * gg[a]) / M;
      ctl[6 + a] = P;
    }
    ctl[9] = 1.0;
  }
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
                          const double *__restrict__ mean, long long begin, long long count,
                          long long stride, double *F, O *rho_out, O *u, double *fabs) {
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
    mp_force<Q, C>(g, rref, pl, kappa, gx, gy, gz, X, Y, Z, rdummy, Fv);
    // the correcting force the step used
    for (int a = 0; a < L::D; ++a) Fv[a] -= rdummy * (C)mean[3 + a];
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

// ---------------------------------------------------------------- launchers
static dim3 mp_block(const Grid &g) {
  const MpGrid m = mp_grid(g.nx, g.ny, g.nz);
  return dim3(m.bx, m.by, 1);
}

template <int Q, int S>
static cudaError_t mp_step_t(const Grid &g, const void *fin, void *fout, const void *rref,
                             void *rho, void *pl, double *ctl, double *partial,
                             const MpParams &mp, double beta, int bgk, int *err, cudaStream_t s) {
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  using C2 = typename Vec2<C>::T;
  const dim3 b = mp_block(g);
  const dim3 grid((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
  k_mp_density<Q, S><<<grid, b, 0, s>>>(g, (const T *)fin, (const C *)rref, (C *)rho, (C2 *)pl,
                                        mp.eos, err);
  k_mp_lap<Q, C><<<grid, b, 0, s>>>(g, (const C *)rho, (C2 *)pl);
  k_mp_sweep<Q, S><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, (const C *)rref,
                                      (const C *)rho, (const C2 *)pl, (C)beta, (C)mp.kappa,
                                      (C)mp.g[0], (C)mp.g[1], (C)mp.g[2], bgk, ctl, partial, err);
  const long long nblk = (long long)grid.x * grid.y * grid.z;
  k_mp_control<<<1, 256, 0, s>>>(partial, nblk, mp.g[0], mp.g[1], mp.g[2], ctl);
  return cudaGetLastError();
}

#define MP_DISPATCH(Q, storage, ...)                                                  \
  do {                                                                                \
    if (Q == 9 && storage == STORE_F32) { constexpr int QQ = 9, SS = STORE_F32; __VA_ARGS__; }   \
    if (Q == 9 && storage == STORE_F64) { constexpr int QQ = 9, SS = STORE_F64; __VA_ARGS__; }   \
    if (Q == 27 && storage == STORE_F32) { constexpr int QQ = 27, SS = STORE_F32; __VA_ARGS__; } \
    return cudaErrorInvalidValue;                                                     \
  } while (0)

cudaError_t launch_mp_step(int Q, int storage, const Grid &g, const void *fin, void *fout,
                           const void *rref, void *rho, void *pl, double *ctl, double *partial,
                           const MpParams &mp, double beta, int bgk, int *err, cudaStream_t s) {
  MP_DISPATCH(Q, storage, return (mp_step_t<QQ, SS>(g, fin, fout, rref, rho, pl, ctl, partial, mp,
                                                    beta, bgk, err, s)));
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
      (C)mp.g[2], have_force, mean, begin, count, stride, F, rho_out, u, fabs);
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
    return cudaGetLastError();
  });
}

}  // namespace kbc
