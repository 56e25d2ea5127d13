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
// Order per coarse step: coarse fields at t, the coarse sweep over all cells,
// coarse fields at t + 1, two fine steps (fill, sweep), the fine fields on
// the ghost-extended patch, the restriction.
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

__device__ __forceinline__ int ref_wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Coarse fields at a position (X, Y) in coarse-cell coordinates: the density
// deviation rho - 1, u[2], G[2][2] (coarse units), bicubic over the periodic
// coarse grid.  The density is carried as its deviation from 1 in every
// field and sum (the weights sum to 1), so FP32 keeps its precision.
template <class C>
struct RefSample {
  C drho, u[2], G[2][2];
};
template <class C>
__device__ __forceinline__ RefSample<C> ref_sample(const C *__restrict__ drho,
                                                   const C *__restrict__ u,
                                                   const C *__restrict__ G, int nx, int ny,
                                                   double X, double Y) {
  const double sx = X - 0.5, sy = Y - 0.5;
  const int ix = (int)floor(sx), iy = (int)floor(sy);
  C wx[4], wy[4];
  ref_cubic_w((C)(sx - ix), wx);
  ref_cubic_w((C)(sy - iy), wy);
  const long long n = (long long)nx * ny;
  RefSample<C> s;
  s.drho = (C)0;
  s.u[0] = s.u[1] = (C)0;
  s.G[0][0] = s.G[0][1] = s.G[1][0] = s.G[1][1] = (C)0;
  for (int b = 0; b < 4; ++b) {
    const long long row = (long long)ref_wrap(iy - 1 + b, ny) * nx;
    for (int a = 0; a < 4; ++a) {
      const long long k = row + ref_wrap(ix - 1 + a, nx);
      const C w = wx[a] * wy[b];
      s.drho += w * drho[k];
      s.u[0] += w * u[k];
      s.u[1] += w * u[n + k];
      for (int q = 0; q < 4; ++q) s.G[q / 2][q % 2] += w * G[q * n + k];
    }
  }
  return s;
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
  return (C)weight<L>(i) * (drho + rho * cu / cs2 + contr / ((C)2 * cs2 * cs2));
}
template <class C>
__device__ __forceinline__ void ref_pn(C rho, const C (&u)[2], const C (&G)[2][2], C beta,
                                       C (&Pn)[2][2]) {
  const C cs2 = (C)(1.0 / 3.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      Pn[a][b] = rho * u[a] * u[b] - rho * cs2 / ((C)2 * beta) * (G[a][b] + G[b][a]);
}

// ---------------------------------------------------------------- coarse fields
// The interpolation reads the coarse fields only within a few cells of the
// patch edge: the fine boundary nodes and the ring sit within 1/4 of a cell
// of it, their bicubic stencils reach 2 cells across it, the central
// differences of grad u one more.  A RefBand is the frame of cells [x0, x0 +
// w) x [y0, y0 + h) (coordinates wrapped onto the periodic grid) less the
// inner rectangle [ix0, ix1) x [iy0, iy1), which no stencil reaches.
struct RefBand {
  int x0, y0, w, h;
  int ix0, ix1, iy0, iy1;
};
// The band of the cells whose fields (margin 3: rho, u) or gradients (margin 2)
// are read, for the patch of mx x my cells from (i0, j0).
static RefBand ref_band(int nxc, int nyc, int i0, int j0, int mx, int my, int margin) {
  RefBand b;
  b.w = mx + 2 * margin;
  b.h = my + 2 * margin;
  b.x0 = i0 - margin;
  b.y0 = j0 - margin;
  if (b.w >= nxc) { b.w = nxc; b.x0 = 0; }
  if (b.h >= nyc) { b.h = nyc; b.y0 = 0; }
  b.ix0 = i0 + margin;
  b.ix1 = i0 + mx - margin;
  b.iy0 = j0 + margin;
  b.iy1 = j0 + my - margin;
  return b;
}
// Cell t of the band's frame, or false for the inner rectangle and the
// threads past the frame.
__device__ __forceinline__ bool band_cell(const RefBand &b, int nx, int ny, long long t, int &x,
                                          int &y) {
  if (t >= (long long)b.w * b.h) return false;
  const int lx = (int)(t % b.w), ly = (int)(t / b.w);
  const int ux = b.x0 + lx, uy = b.y0 + ly;  // unwrapped
  if (ux >= b.ix0 && ux < b.ix1 && uy >= b.iy0 && uy < b.iy1) return false;
  x = ref_wrap(ux, nx);
  y = ref_wrap(uy, ny);
  return true;
}

// rho - 1 and u = j / rho of the coarse state over a band (linear index k =
// y nx + x of the coarse grid)
template <int S>
__global__ void k_ref_coarse_fields(Grid g, RefBand band, const typename Store<S>::T *__restrict__ f,
                                    typename Store<S>::C *__restrict__ drho,
                                    typename Store<S>::C *__restrict__ u) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  int x, y;
  if (!band_cell(band, g.nx, g.ny, blockIdx.x * (long long)blockDim.x + threadIdx.x, x, y)) return;
  const long long n = (long long)g.nx * g.ny;
  const long long k = (long long)y * g.nx + x;
  const long long s = sidx(g, x + g.px, y + g.py, 0);
  C d = (C)0, jx = (C)0, jy = (C)0;
  for (int i = 0; i < 9; ++i) {
    const C v = St::load(f + (long long)i * g.N + s, (C)weight<L>(i));
    d += v;
    jx += (C)L::cx(i) * v;
    jy += (C)L::cy(i) * v;
  }
  const C r = (C)1 + d;
  drho[k] = d;
  u[k] = jx / r;
  u[n + k] = jy / r;
}

// G[a][b] = d u_a / d x_b by central differences (periodic), coarse units,
// over a band
template <class C>
__global__ void k_ref_coarse_grad(int nx, int ny, RefBand band, const C *__restrict__ u,
                                  C *__restrict__ G) {
  int x, y;
  if (!band_cell(band, nx, ny, blockIdx.x * (long long)blockDim.x + threadIdx.x, x, y)) return;
  const long long n = (long long)nx * ny;
  const long long k = (long long)y * nx + x;
  const long long xp = (long long)y * nx + ref_wrap(x + 1, nx), xm = (long long)y * nx + ref_wrap(x - 1, nx);
  const long long yp = (long long)ref_wrap(y + 1, ny) * nx + x, ym = (long long)ref_wrap(y - 1, ny) * nx + x;
  for (int a = 0; a < 2; ++a) {
    G[(2 * a) * n + k] = (C)0.5 * (u[a * n + xp] - u[a * n + xm]);
    G[(2 * a + 1) * n + k] = (C)0.5 * (u[a * n + yp] - u[a * n + ym]);
  }
}

// ---------------------------------------------------------------- fine fill
// One thread per fine boundary node (the patch perimeter, p along x, q
// along y): Grad's approximation at the node from the coarse fields at time
// t + w, into the ghost slots of the directions it misses.
template <int S>
__global__ void k_ref_fill(Grid gf, typename Store<S>::T *__restrict__ ff, int nxc, int nyc,
                           const typename Store<S>::C *__restrict__ r0,
                           const typename Store<S>::C *__restrict__ u0,
                           const typename Store<S>::C *__restrict__ G0,
                           const typename Store<S>::C *__restrict__ r1,
                           const typename Store<S>::C *__restrict__ u1,
                           const typename Store<S>::C *__restrict__ G1, int i0, int j0,
                           typename Store<S>::C w, typename Store<S>::C beta_f) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  const int nfx = gf.nx, nfy = gf.ny;
  const int nper = 2 * nfx + 2 * (nfy - 2);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nper) return;
  int p, q;
  if (t < nfx) { p = t; q = 0; }
  else if (t < 2 * nfx) { p = t - nfx; q = nfy - 1; }
  else if (t < 2 * nfx + nfy - 2) { p = 0; q = t - 2 * nfx + 1; }
  else { p = nfx - 1; q = t - (2 * nfx + nfy - 2) + 1; }
  const double X = i0 + 0.5 * (p + 0.5), Y = j0 + 0.5 * (q + 0.5);
  const RefSample<C> a = ref_sample(r0, u0, G0, nxc, nyc, X, Y);
  const RefSample<C> b = ref_sample(r1, u1, G1, nxc, nyc, X, Y);
  const C drho = ((C)1 - w) * a.drho + w * b.drho, rho = (C)1 + drho;
  C u[2], G[2][2], Pn[2][2];
  for (int c = 0; c < 2; ++c) u[c] = ((C)1 - w) * a.u[c] + w * b.u[c];
  for (int c = 0; c < 2; ++c)
    for (int d = 0; d < 2; ++d) G[c][d] = (C)0.5 * (((C)1 - w) * a.G[c][d] + w * b.G[c][d]);
  ref_pn(rho, u, G, beta_f, Pn);
  for (int i = 0; i < 9; ++i) {
    const int ps = p - L::cx(i), qs = q - L::cy(i);
    if (ps >= 0 && ps < nfx && qs >= 0 && qs < nfy) continue;
    // the ghost slot of direction i that the node pulls from
    const long long s = sidx(gf, ps + gf.px, qs + gf.py, 0);
    St::store(ff + (long long)i * gf.N + s, ref_grad_dev(i, drho, rho, u, Pn),
              (C)(1.0 / weight<L>(i)));
  }
}

// ---------------------------------------------------------------- restriction
// Fine fields on the patch extended by one ring: rho - 1, j[2], u[2] at (p, q) in
// [-1, nfx] x [-1, nfy], index (q + 1) * (nfx + 2) + (p + 1); the ring from the
// coarse fields at t + 1.
template <int S>
__global__ void k_ref_fine_fields(Grid gf, const typename Store<S>::T *__restrict__ ff, int nxc,
                                  int nyc, const typename Store<S>::C *__restrict__ r1,
                                  const typename Store<S>::C *__restrict__ u1,
                                  const typename Store<S>::C *__restrict__ G1, int i0, int j0,
                                  typename Store<S>::C *__restrict__ ext) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  const int ex = gf.nx + 2, ey = gf.ny + 2;
  const long long ne = (long long)ex * ey;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ne) return;
  const int p = (int)(t % ex) - 1, q = (int)(t / ex) - 1;
  C d, j[2], u[2];
  if (p >= 0 && p < gf.nx && q >= 0 && q < gf.ny) {
    const long long s = sidx(gf, p + gf.px, q + gf.py, 0);
    d = (C)0;
    j[0] = j[1] = (C)0;
    for (int i = 0; i < 9; ++i) {
      const C v = St::load(ff + (long long)i * gf.N + s, (C)weight<L>(i));
      d += v;
      j[0] += (C)L::cx(i) * v;
      j[1] += (C)L::cy(i) * v;
    }
    u[0] = j[0] / ((C)1 + d);
    u[1] = j[1] / ((C)1 + d);
  } else {
    const RefSample<C> c = ref_sample(r1, u1, G1, nxc, nyc, i0 + 0.5 * (p + 0.5), j0 + 0.5 * (q + 0.5));
    d = c.drho;
    u[0] = c.u[0];
    u[1] = c.u[1];
    j[0] = ((C)1 + d) * u[0];
    j[1] = ((C)1 + d) * u[1];
  }
  ext[t] = d;
  ext[ne + t] = j[0];
  ext[2 * ne + t] = j[1];
  ext[3 * ne + t] = u[0];
  ext[4 * ne + t] = u[1];
}

// One thread per covered coarse cell (I, J): cubic midpoint values, Grad's
// approximation with beta_c, the coarse collision, the stored state.
template <int S>
__global__ void k_ref_restrict(Grid gc, typename Store<S>::T *__restrict__ fc, int nfx, int nfy,
                               const typename Store<S>::C *__restrict__ ext, int i0, int j0,
                               typename Store<S>::C beta_c, int bgk) {
  using L = Lat<9>;
  using St = Store<S>;
  using C = typename St::C;
  const int mx = nfx / 2, my = nfy / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mx * my) return;
  const int I = t % mx, J = t / mx;
  const int ex = nfx + 2;
  const long long ne = (long long)ex * (nfy + 2);
  const C wm[4] = {(C)(-1.0 / 16.0), (C)(9.0 / 16.0), (C)(9.0 / 16.0), (C)(-1.0 / 16.0)};
  auto at = [&](int f, int p, int q) -> C { return ext[f * ne + (long long)(q + 1) * ex + (p + 1)]; };
  C d = (C)0, j[2] = {(C)0, (C)0};
  for (int b = 0; b < 4; ++b)
    for (int a = 0; a < 4; ++a) {
      const int p = 2 * I - 1 + a, q = 2 * J - 1 + b;
      const C w = wm[a] * wm[b];
      d += w * at(0, p, q);
      j[0] += w * at(1, p, q);
      j[1] += w * at(2, p, q);
    }
  C G[2][2];
  for (int c = 0; c < 2; ++c) {
    C dx = (C)0, dy = (C)0;
    for (int b = 0; b < 4; ++b) {
      const int q = 2 * J - 1 + b, p = 2 * I - 1 + b;
      dx += wm[b] * (at(3 + c, 2 * I + 1, q) - at(3 + c, 2 * I, q));
      dy += wm[b] * (at(3 + c, p, 2 * J + 1) - at(3 + c, p, 2 * J));
    }
    G[c][0] = (C)2 * dx;
    G[c][1] = (C)2 * dy;
  }
  const C r = (C)1 + d;
  const C u[2] = {j[0] / r, j[1] / r};
  C Pn[2][2];
  ref_pn(r, u, G, beta_c, Pn);
  C v[9];
  for (int i = 0; i < 9; ++i) v[i] = ref_grad_dev(i, d, r, u, Pn);
  collide_v<L, S == STORE_F32, C>(v, beta_c, bgk != 0);
  const long long s = sidx(gc, i0 + I + gc.px, j0 + J + gc.py, 0);
  for (int i = 0; i < 9; ++i)
    St::store(fc + (long long)i * gc.N + s, v[i], (C)(1.0 / weight<L>(i)));
}

// ---------------------------------------------------------------- launchers
template <int S>
static cudaError_t ref_step_t(const RefLaunch &R, cudaStream_t s) {
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  const Grid &gc = R.gc, &gf = R.gf;
  const long long nc = (long long)gc.nx * gc.ny;
  C *r0 = (C *)R.fields, *u0 = r0 + nc, *G0 = u0 + 2 * nc;
  C *r1 = G0 + 4 * nc, *u1 = r1 + nc, *G1 = u1 + 2 * nc;
  C *ext = G1 + 4 * nc;
  const int b = 256;
  const int mx = gf.nx / 2, my = gf.ny / 2;
  const RefBand bu = ref_band(gc.nx, gc.ny, R.i0, R.j0, mx, my, 3);
  const RefBand bg = ref_band(gc.nx, gc.ny, R.i0, R.j0, mx, my, 2);
  const unsigned nbu = (unsigned)(((long long)bu.w * bu.h + b - 1) / b);
  const unsigned nbg = (unsigned)(((long long)bg.w * bg.h + b - 1) / b);
  k_ref_coarse_fields<S><<<nbu, b, 0, s>>>(gc, bu, (const T *)R.fc_in, r0, u0);
  k_ref_coarse_grad<C><<<nbg, b, 0, s>>>(gc.nx, gc.ny, bg, u0, G0);
  cudaError_t e = launch_sweep(9, S, gc, R.fc_in, R.fc_out, nullptr, R.beta_c, R.bgk, R.err_c, s,
                               R.variant);
  if (e != cudaSuccess) return e;
  k_ref_coarse_fields<S><<<nbu, b, 0, s>>>(gc, bu, (const T *)R.fc_out, r1, u1);
  k_ref_coarse_grad<C><<<nbg, b, 0, s>>>(gc.nx, gc.ny, bg, u1, G1);
  const int nper = 2 * gf.nx + 2 * (gf.ny - 2);
  void *fa = R.ff[R.cur_f], *fb = R.ff[1 - R.cur_f];
  for (int k = 0; k < 2; ++k) {
    k_ref_fill<S><<<(nper + 127) / 128, 128, 0, s>>>(gf, (T *)fa, gc.nx, gc.ny, r0, u0, G0, r1, u1,
                                                     G1, R.i0, R.j0, (C)(0.5 * (k + 1)),
                                                     (C)R.beta_f);
    e = launch_sweep(9, S, gf, fa, fb, R.flags_f, R.beta_f, R.bgk, R.err_f, s, R.variant);
    if (e != cudaSuccess) return e;
    void *tmp = fa;
    fa = fb;
    fb = tmp;
  }
  const long long ne = (long long)(gf.nx + 2) * (gf.ny + 2);
  k_ref_fine_fields<S><<<(unsigned)((ne + b - 1) / b), b, 0, s>>>(gf, (const T *)fa, gc.nx, gc.ny,
                                                                  r1, u1, G1, R.i0, R.j0, ext);
  const int ncov = (gf.nx / 2) * (gf.ny / 2);
  k_ref_restrict<S><<<(ncov + 127) / 128, 128, 0, s>>>(gc, (T *)R.fc_out, gf.nx, gf.ny, ext, R.i0,
                                                       R.j0, (C)R.beta_c, R.bgk);
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const RefLaunch &R, cudaStream_t s) {
  if (R.storage == STORE_F32) return ref_step_t<STORE_F32>(R, s);
  if (R.storage == STORE_F64) return ref_step_t<STORE_F64>(R, s);
  return cudaErrorInvalidValue;
}

size_t refine_workspace_bytes(int storage, int nxc, int nyc, int nfx, int nfy) {
  const size_t cb = storage == STORE_F64 ? 8 : 4;
  const size_t nc = (size_t)nxc * nyc, ne = (size_t)(nfx + 2) * (nfy + 2);
  return cb * (14 * nc + 5 * ne);
}

}  // namespace kbc
