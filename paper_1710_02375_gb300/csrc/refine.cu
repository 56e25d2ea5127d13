// refine.cu -- two-level grid refinement (D2Q9): a periodic coarse lattice
// and a fine patch at half the spacing, two fine steps per coarse step
// (arXiv 1710.02375 uses multi-domain refinement in its validation cases and
// cites its algorithm; the reading implemented here, the same as the
// oracle's or_refine_step):
//   coarse -> fine: at the fine nodes whose pull reaches outside the patch,
//     those populations are Grad's approximation, Eq. (grad), Pi = rho c_s^2
//     I + rho u u - rho c_s^2/(2 beta_f)(grad u + grad u^T), of the coarse
//     rho, u = j / rho and grad u (central differences; half in fine units)
//     interpolated bicubically to the node and linearly in time to the fine
//     time of the pull (t + 1/2, t + 1); written into the ghost slots the
//     fine sweep pulls them from;
//   fine -> coarse: each covered coarse cell takes the cubic midpoint values
//     (weights -1, 9, 9, -1 over 16 per axis) of the fine density and
//     momentum, the velocity gradient from the midpoint differences of the
//     fine velocity (doubled to coarse units; the ghost ring holds the
//     coarse values of t + 1), Grad's approximation with beta_c and the
//     coarse KBC collision: its stored post-collision state.
// Order per coarse step: the coarse sweep over all cells; one sampling pass
// (the coarse fields at t and t + 1 interpolated to the fine boundary nodes,
// those at t + 1 to the ring around the patch); two fine steps (fill,
// sweep); the restriction, with the fine moments of each tile staged in
// shared memory.
#include "kbc_collide.cuh"
#include "lbm_internal.h"

namespace kbc {

// Lagrange weights of the four nodes -1, 0, 1, 2 at the offset t in [0, 1)
template <class C>
__device__ __forceinline__ void ref_cubic_w(C t, C (&w)[4]) {
  w[0] = -t * (t - (C)1) * (t - (C)2) / (C)6;
  w[1] = (t + (C)1) * (t - (C)1) * (t - (C)2) / (C)2;
  w[2] = -(t + (C)1) * t * (t - (C)2) / (C)2;
  w[3] = (t + (C)1) * t * (t - (C)1) / (C)6;
}

// the k-th of those weights (selected, not indexed: k varies across lanes)
template <class C>
__device__ __forceinline__ C ref_cubic_wk(C t, int k) {
  C w[4];
  ref_cubic_w(t, w);
  return k == 0 ? w[0] : (k == 1 ? w[1] : (k == 2 ? w[2] : w[3]));
}

__device__ __forceinline__ int ref_wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// D2Q9 weight of direction i in the compute type (selects, so a runtime i
// costs no double-precision arithmetic)
template <class C>
__device__ __forceinline__ C ref_weight(int i) {
  using L = Lat<9>;
  const C a = L::cx(i) == 0 ? (C)(2.0 / 3.0) : (C)(1.0 / 6.0);
  const C b = L::cy(i) == 0 ? (C)(2.0 / 3.0) : (C)(1.0 / 6.0);
  return a * b;
}

// Grad's approximation of direction i (D2Q9) for rho = 1 + drho, u and Pi -
// rho c_s^2 I, less the weight W_i (the stored deviation).
template <class C>
__device__ __forceinline__ C ref_grad_dev(int i, C drho, C rho, const C (&u)[2],
                                          const C (&Pn)[2][2]) {
  using L = Lat<9>;
  const int c[2] = {L::cx(i), L::cy(i)};
  const C cs2 = (C)(1.0 / 3.0);
  C cu = (C)0, contr = (C)0;
  for (int a = 0; a < 2; ++a) cu += (C)c[a] * u[a];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) contr += Pn[a][b] * ((C)(c[a] * c[b]) - (a == b ? cs2 : (C)0));
  return ref_weight<C>(i) * (drho + rho * cu / cs2 + contr / ((C)2 * cs2 * cs2));
}
template <class C>
__device__ __forceinline__ void ref_pn(C rho, const C (&u)[2], const C (&G)[2][2], C beta,
                                       C (&Pn)[2][2]) {
  const C cs2 = (C)(1.0 / 3.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      Pn[a][b] = rho * u[a] * u[b] - rho * cs2 / ((C)2 * beta) * (G[a][b] + G[b][a]);
}


// ---------------------------------------------------------------- node lists
// Fill nodes: the perimeter of the fine patch (p along x, q along y), bottom
// row, top row, then the left and right columns without their corners.
__host__ __device__ inline int ref_nfill(int nfx, int nfy) { return 2 * nfx + 2 * (nfy - 2); }
__device__ __forceinline__ void ref_fill_node(int t, int nfx, int nfy, int &p, int &q) {
  if (t < nfx) { p = t; q = 0; }
  else if (t < 2 * nfx) { p = t - nfx; q = nfy - 1; }
  else if (t < 2 * nfx + nfy - 2) { p = 0; q = t - 2 * nfx + 1; }
  else { p = nfx - 1; q = t - (2 * nfx + nfy - 2) + 1; }
}
// Ring nodes: the perimeter of the patch extended by one node, p in [-1,
// nfx], q in [-1, nfy]: the row q = -1, the row q = nfy, then the columns p =
// -1 and p = nfx over q in [0, nfy).
__host__ __device__ inline int ref_nring(int nfx, int nfy) { return 2 * (nfx + 2) + 2 * nfy; }
__device__ __forceinline__ void ref_ring_node(int t, int nfx, int nfy, int &p, int &q) {
  const int rw = nfx + 2;
  if (t < rw) { p = t - 1; q = -1; }
  else if (t < 2 * rw) { p = t - rw - 1; q = nfy; }
  else if (t < 2 * rw + nfy) { p = -1; q = t - 2 * rw; }
  else { p = nfx; q = t - 2 * rw - nfy; }
}
__device__ __forceinline__ int ref_ring_index(int p, int q, int nfx, int nfy) {
  const int rw = nfx + 2;
  if (q == -1) return p + 1;
  if (q == nfy) return rw + p + 1;
  if (p == -1) return 2 * rw + q;
  return 2 * rw + nfy + q;
}

// Sampled values: fill node n holds (rho - 1, u_x, u_y, G_xx, G_xy, G_yx,
// G_yy) at t, then at t + 1 (G[a][b] = d u_a / d x_b in coarse units), ring
// node m holds (rho - 1, u_x, u_y) at t + 1; structure of arrays.
constexpr int kRefFillVals = 14, kRefRingVals = 3;

// rho - 1 and u = j / rho of coarse cell (x, y) from its stored populations
template <int S>
__device__ __forceinline__ void ref_cell(const Grid &g, const typename Store<S>::T *__restrict__ f,
                                         int x, int y, typename Store<S>::C &d,
                                         typename Store<S>::C (&u)[2]) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  const long long s = sidx(g, x + g.px, y + g.py, 0);
  C dd = (C)0, jx = (C)0, jy = (C)0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const C v = St::load(f + (long long)i * g.N + s, (C)weight<L>(i));
    dd += v;
    jx += (C)L::cx(i) * v;
    jy += (C)L::cy(i) * v;
  }
  d = dd;
  u[0] = jx / ((C)1 + dd);
  u[1] = jy / ((C)1 + dd);
}

// ---------------------------------------------------------------- fine fill
// Grad's approximation of direction i at fill node (p, q) from the sampled
// coarse fields v (kRefFillVals values) at time t + w, into the ghost slot
// the node's pull reads when that direction is missing (no sweep writes
// ghost slots).
template <int S>
__device__ __forceinline__ void ref_fill_dir(const Grid &gf, typename Store<S>::T *__restrict__ ff,
                                             int p, int q, int i,
                                             const typename Store<S>::C (&v)[kRefFillVals],
                                             typename Store<S>::C w, typename Store<S>::C beta_f) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  const int ps = p - L::cx(i), qs = q - L::cy(i);
  if (ps >= 0 && ps < gf.nx && qs >= 0 && qs < gf.ny) return;
  const C drho = ((C)1 - w) * v[0] + w * v[7], rho = (C)1 + drho;
  C u[2], G[2][2], Pn[2][2];
  for (int c = 0; c < 2; ++c) u[c] = ((C)1 - w) * v[1 + c] + w * v[8 + c];
  for (int c = 0; c < 2; ++c)
    for (int d = 0; d < 2; ++d)
      G[c][d] = (C)0.5 * (((C)1 - w) * v[3 + 2 * c + d] + w * v[10 + 2 * c + d]);
  ref_pn(rho, u, G, beta_f, Pn);
  const long long s = sidx(gf, ps + gf.px, qs + gf.py, 0);
  // FP32 and FP64 storage keep f - W unscaled: the scale argument is unused
  St::store(ff + (long long)i * gf.N + s, ref_grad_dev(i, drho, rho, u, Pn), (C)1);
}

// ---------------------------------------------------------------- sampling
// One warp per sampled node.  The node at (X, Y) in coarse-cell coordinates
// interpolates over the 4 x 4 cells floor(X - 1/2) - 1 .. + 2 per axis
// (wrapped onto the periodic grid); their central differences reach one
// cell further.  The 32 lanes take the 6 x 6 block around the stencil less
// its corners (lane -> block cell (cx, cy): row cy = 0 cx = 1..4, rows 1..4
// cx = 0..5, row 5 cx = 1..4), each forms its cell's rho - 1 and u from the
// coarse populations at t (fc0) and t + 1 (fc1), the 16 stencil lanes take
// grad u from their neighbours' u by shuffles, and the weighted values are
// summed over the warp.  A fill node then writes the ghost slots of both
// fine steps, one (time, direction) per lane: t + 1/2 into fa (read by the
// first fine sweep), t + 1 into fb (read by the second); a ring node stores
// its fields at t + 1 for the restriction.
__device__ __forceinline__ void ref_block_cell(int lane, int &cx, int &cy) {
  if (lane < 4) { cx = lane + 1; cy = 0; }
  else if (lane < 28) { cx = (lane - 4) % 6; cy = (lane - 4) / 6 + 1; }
  else { cx = lane - 27; cy = 5; }
}
__device__ __forceinline__ int ref_block_lane(int cx, int cy) {
  return cy == 0 ? cx - 1 : (cy == 5 ? cx + 27 : 4 + (cy - 1) * 6 + cx);
}

template <int S>
__global__ void __launch_bounds__(256)
    k_ref_sample(Grid gc, const typename Store<S>::T *__restrict__ fc0,
                 const typename Store<S>::T *__restrict__ fc1, Grid gf,
                 typename Store<S>::T *__restrict__ fa, typename Store<S>::T *__restrict__ fb,
                 int i0, int j0, typename Store<S>::C beta_f,
                 typename Store<S>::C *__restrict__ sring) {
  using C = typename Store<S>::C;
  const int nfx = gf.nx, nfy = gf.ny;
  const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int nfill = ref_nfill(nfx, nfy), nring = ref_nring(nfx, nfy);
  if (node >= nfill + nring) return;  // the whole warp
  const bool fill = node < nfill;
  int p, q;
  if (fill) ref_fill_node(node, nfx, nfy, p, q);
  else ref_ring_node(node - nfill, nfx, nfy, p, q);
  // X - 1/2 = i0 + (2 p - 1) / 4 exactly: stencil origin and offset in
  // quarter cells, in integers (floor by arithmetic shift)
  const int nx4 = 4 * i0 + 2 * p - 1, ny4 = 4 * j0 + 2 * q - 1;
  const int ix = nx4 >> 2, iy = ny4 >> 2;
  const C tx = (C)0.25 * (C)(nx4 & 3), ty = (C)0.25 * (C)(ny4 & 3);
  int cx, cy;
  ref_block_cell(lane, cx, cy);
  const bool inner = cx >= 1 && cx <= 4 && cy >= 1 && cy <= 4;
  const C w = inner ? ref_cubic_wk(tx, cx - 1) * ref_cubic_wk(ty, cy - 1) : (C)0;
  const int x = ref_wrap(ix - 2 + cx, gc.nx), y = ref_wrap(iy - 2 + cy, gc.ny);
  // neighbour lanes of a stencil lane (own lane elsewhere: unused)
  const int le = inner ? ref_block_lane(cx + 1, cy) : lane, lw = inner ? ref_block_lane(cx - 1, cy) : lane;
  const int ln = inner ? ref_block_lane(cx, cy + 1) : lane, ls = inner ? ref_block_lane(cx, cy - 1) : lane;
  // both time levels' loads first (ring nodes: t + 1 only)
  C dt[2] = {(C)0, (C)0}, ut[2][2] = {{(C)0, (C)0}, {(C)0, (C)0}};
  if (fill) ref_cell<S>(gc, fc0, x, y, dt[0], ut[0]);
  ref_cell<S>(gc, fc1, x, y, dt[1], ut[1]);
  C acc[kRefFillVals];
#pragma unroll
  for (int tt = 0; tt < 2; ++tt) {
    C *o = acc + 7 * tt;
    const C d = dt[tt], u[2] = {ut[tt][0], ut[tt][1]};
    o[0] = w * d;
    o[1] = w * u[0];
    o[2] = w * u[1];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const C ue = __shfl_sync(0xffffffffu, u[c], le), uw = __shfl_sync(0xffffffffu, u[c], lw);
      const C un = __shfl_sync(0xffffffffu, u[c], ln), us = __shfl_sync(0xffffffffu, u[c], ls);
      o[3 + 2 * c] = w * ((C)0.5 * (ue - uw));
      o[4 + 2 * c] = w * ((C)0.5 * (un - us));
    }
  }
#pragma unroll
  for (int k = 0; k < kRefFillVals; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  // every lane holds the sums: lanes 0..17 write one (time, direction) each
  if (fill) {
    if (lane < 18) {
      const bool second = lane >= 9;
      ref_fill_dir<S>(gf, second ? fb : fa, p, q, second ? lane - 9 : lane, acc,
                      second ? (C)1 : (C)0.5, beta_f);
    }
  } else if (lane < kRefRingVals) {
    const int m = node - nfill;
    sring[(long long)lane * nring + m] = lane == 0 ? acc[7] : (lane == 1 ? acc[8] : acc[9]);
  }
}

// ---------------------------------------------------------------- restriction
// A CTA restricts a tile of kRefTX x kRefTY covered coarse cells.  It first
// stages (rho - 1, j_x, j_y, u_x, u_y) of the fine nodes the tile's cubic
// stencils reach, 2 I0 - 1 .. 2 (I0 + kRefTX) along x and the same along y
// (ring nodes beyond the patch from the sampled coarse fields at t + 1),
// then each thread takes one cell (I, J): the cubic midpoint values, Grad's
// approximation with beta_c, the coarse collision, the stored state.
constexpr int kRefTX = 32, kRefTY = 8;
constexpr int kRefEX = 2 * kRefTX + 2, kRefEY = 2 * kRefTY + 2;

template <int S>
__global__ void __launch_bounds__(kRefTX * kRefTY)
    k_ref_restrict(Grid gc, typename Store<S>::T *__restrict__ fc, Grid gf,
                   const typename Store<S>::T *__restrict__ ff,
                   const typename Store<S>::C *__restrict__ sring, int i0, int j0,
                   typename Store<S>::C beta_c, int bgk) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  __shared__ C sm[5][kRefEY][kRefEX];
  const int nfx = gf.nx, nfy = gf.ny, mx = nfx / 2, my = nfy / 2;
  const int nring = ref_nring(nfx, nfy);
  const int I0 = blockIdx.x * kRefTX, J0 = blockIdx.y * kRefTY;
  const int p0 = 2 * I0 - 1, q0 = 2 * J0 - 1;  // fine node of sm[.][0][0]
  constexpr int kPer = (kRefEX * kRefEY + kRefTX * kRefTY - 1) / (kRefTX * kRefTY);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = threadIdx.x + k * kRefTX * kRefTY;
    if (e >= kRefEX * kRefEY) continue;
    const int ex = e % kRefEX, ey = e / kRefEX;
    const int p = p0 + ex, q = q0 + ey;
    C d = (C)0, j[2] = {(C)0, (C)0}, u[2] = {(C)0, (C)0};
    if (p >= 0 && p < nfx && q >= 0 && q < nfy) {
      const long long s = sidx(gf, p + gf.px, q + gf.py, 0);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C v = St::load(ff + (long long)i * gf.N + s, (C)weight<L>(i));
        d += v;
        j[0] += (C)L::cx(i) * v;
        j[1] += (C)L::cy(i) * v;
      }
      u[0] = j[0] / ((C)1 + d);
      u[1] = j[1] / ((C)1 + d);
    } else if (p >= -1 && p <= nfx && q >= -1 && q <= nfy) {
      const int m = ref_ring_index(p, q, nfx, nfy);
      d = sring[m];
      u[0] = sring[nring + m];
      u[1] = sring[2 * nring + m];
      j[0] = ((C)1 + d) * u[0];
      j[1] = ((C)1 + d) * u[1];
    }
    sm[0][ey][ex] = d;
    sm[1][ey][ex] = j[0];
    sm[2][ey][ex] = j[1];
    sm[3][ey][ex] = u[0];
    sm[4][ey][ex] = u[1];
  }
  __syncthreads();
  const int tx = threadIdx.x % kRefTX, ty = threadIdx.x / kRefTX;
  const int I = I0 + tx, J = J0 + ty;
  if (I >= mx || J >= my) return;
  const int lx = 2 * tx, ly = 2 * ty;  // sm position of fine node (2 I - 1, 2 J - 1)
  const C wm[4] = {(C)(-1.0 / 16.0), (C)(9.0 / 16.0), (C)(9.0 / 16.0), (C)(-1.0 / 16.0)};
  C d = (C)0, j[2] = {(C)0, (C)0};
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const C w = wm[a] * wm[b];
      d += w * sm[0][ly + b][lx + a];
      j[0] += w * sm[1][ly + b][lx + a];
      j[1] += w * sm[2][ly + b][lx + a];
    }
  C G[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    C dx = (C)0, dy = (C)0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      // d/dx: the pairs (2I, 2I + 1) on the rows 2J - 1 .. 2J + 2; d/dy: the
      // pairs (2J, 2J + 1) on the columns 2I - 1 .. 2I + 2
      dx += wm[b] * (sm[3 + c][ly + b][lx + 2] - sm[3 + c][ly + b][lx + 1]);
      dy += wm[b] * (sm[3 + c][ly + 2][lx + b] - sm[3 + c][ly + 1][lx + b]);
    }
    G[c][0] = (C)2 * dx;
    G[c][1] = (C)2 * dy;
  }
  const C r = (C)1 + d;
  const C u[2] = {j[0] / r, j[1] / r};
  C Pn[2][2];
  ref_pn(r, u, G, beta_c, Pn);
  C v[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = ref_grad_dev(i, d, r, u, Pn);
  collide_v<L, S == STORE_F32, C>(v, beta_c, bgk != 0);
  const long long s = sidx(gc, i0 + I + gc.px, j0 + J + gc.py, 0);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    St::store(fc + (long long)i * gc.N + s, v[i], (C)(1.0 / weight<L>(i)));
}

// ---------------------------------------------------------------- launchers
// Coarse cells that need no coarse step: those more than kRefKeep cells
// inside the patch edge (the restriction replaces them, and no stencil of
// the sampling reads them).
constexpr int kRefKeep = 3;
__global__ void k_ref_skip(Grid gc, uint8_t *__restrict__ skip, int x0, int x1, int y0, int y1) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int w = x1 - x0;
  if (t >= (long long)w * (y1 - y0)) return;
  const int x = x0 + (int)(t % w), y = y0 + (int)(t / w);
  skip[sidx(gc, x + gc.px, y + gc.py, 0)] = NODE_GHOST;
}

static size_t ref_ring_bytes(int storage, int nfx, int nfy) {
  const size_t cb = storage == STORE_F64 ? 8 : 4;
  return (cb * kRefRingVals * (size_t)ref_nring(nfx, nfy) + 255) / 256 * 256;
}

template <int S>
static cudaError_t ref_step_t(const RefLaunch &R, cudaStream_t s) {
  static_assert(S == STORE_F32 || S == STORE_F64, "unscaled deviations (the fill's stores)");
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  const Grid &gc = R.gc, &gf = R.gf;
  const int nfill = ref_nfill(gf.nx, gf.ny), nring = ref_nring(gf.nx, gf.ny);
  C *sring = (C *)R.fields;
  const uint8_t *skip = (const uint8_t *)R.fields + ref_ring_bytes(S, gf.nx, gf.ny);
  cudaError_t e = launch_sweep(9, S, gc, R.fc_in, R.fc_out, skip, R.beta_c, R.bgk, R.err_c, s,
                               R.variant);
  if (e != cudaSuccess) return e;
  void *fa = R.ff[R.cur_f], *fb = R.ff[1 - R.cur_f];
  const long long nthr = 32LL * (nfill + nring);
  k_ref_sample<S><<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(
      gc, (const T *)R.fc_in, (const T *)R.fc_out, gf, (T *)fa, (T *)fb, R.i0, R.j0, (C)R.beta_f,
      sring);
  for (int k = 0; k < 2; ++k) {
    e = launch_sweep(9, S, gf, fa, fb, R.flags_f, R.beta_f, R.bgk, R.err_f, s, R.variant);
    if (e != cudaSuccess) return e;
    void *tmp = fa;
    fa = fb;
    fb = tmp;
  }
  const dim3 grid((unsigned)((gf.nx / 2 + kRefTX - 1) / kRefTX),
                  (unsigned)((gf.ny / 2 + kRefTY - 1) / kRefTY));
  k_ref_restrict<S><<<grid, kRefTX * kRefTY, 0, s>>>(gc, (T *)R.fc_out, gf, (const T *)fa, sring,
                                                     R.i0, R.j0, (C)R.beta_c, R.bgk);
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const RefLaunch &R, cudaStream_t s) {
  if (R.storage == STORE_F32) return ref_step_t<STORE_F32>(R, s);
  if (R.storage == STORE_F64) return ref_step_t<STORE_F64>(R, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_refine_init(const RefLaunch &R, cudaStream_t s) {
  uint8_t *skip = (uint8_t *)R.fields + ref_ring_bytes(R.storage, R.gf.nx, R.gf.ny);
  cudaError_t e = cudaMemsetAsync(skip, NODE_FLUID, (size_t)R.gc.N, s);
  if (e != cudaSuccess) return e;
  const int mx = R.gf.nx / 2, my = R.gf.ny / 2;
  const int x0 = R.i0 + kRefKeep, x1 = R.i0 + mx - kRefKeep;
  const int y0 = R.j0 + kRefKeep, y1 = R.j0 + my - kRefKeep;
  if (x1 <= x0 || y1 <= y0) return cudaSuccess;
  const long long n = (long long)(x1 - x0) * (y1 - y0);
  k_ref_skip<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R.gc, skip, x0, x1, y0, y1);
  return cudaGetLastError();
}

size_t refine_workspace_bytes(int storage, const Grid &gc, int nfx, int nfy) {
  return ref_ring_bytes(storage, nfx, nfy) + (size_t)gc.N;
}

}  // namespace kbc
