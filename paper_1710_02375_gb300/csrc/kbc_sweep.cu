// kbc_sweep.cu -- the fused pull-stream + KBC collision sweep and the
// population conversion kernels.
//
// One thread per interior node, x fastest across the warp so that all Q loads
// and Q stores of a warp are coalesced (the +-x neighbours are one element
// off and come from the same L1/L2 lines).  The sweep reads Q populations and
// writes Q populations per node: 2 Q bytes_per_population of algorithmic HBM
// traffic, Eq. (f_equations); the collision (kbc_collide.cuh) stays in
// registers.  No tensor cores: there is no contraction on this path.
#include "kbc_collide.cuh"
#include "lbm_internal.h"

namespace kbc {

template <int Q, int S, bool FLAGS>
__global__ void __launch_bounds__(256, 2)
    k_sweep(Grid g, const typename Store<S>::T *__restrict__ fin,
            typename Store<S>::T *__restrict__ fout, const uint8_t *__restrict__ flags,
            float beta, int bgk, int *__restrict__ err) {
  using L = Lat<Q>;
  using St = Store<S>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
  const long long k = sidx(g, X, Y, Z);
  if (FLAGS && flags[k] != NODE_FLUID) return;

  const int xs[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};  // source x for cx = -1, 0, +1
  const int ys[3] = {nbr(Y, 1, g.NY), Y, nbr(Y, -1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, 1, g.NZ);
    zs[2] = nbr(Z, -1, g.NZ);
  }
  float v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long src = ((long long)zs[L::cz(i) + 1] * g.NY + ys[L::cy(i) + 1]) * g.NX +
                          xs[L::cx(i) + 1];
    v[i] = St::load(fin + (long long)i * g.N + src, (float)weight<L>(i));
  }
  const float rho = collide<L>(v, beta, bgk != 0);
  if (!(rho > 0.f && rho < 1e30f)) atomicOr(err, 1);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    St::store(fout + (long long)i * g.N + k, v[i], (float)(1.0 / weight<L>(i)));
}

static dim3 sweep_block(const Grid &g) {
  if (g.nx >= 128) return dim3(128, 2, 1);
  if (g.nx >= 64) return dim3(64, 4, 1);
  return dim3(32, 8, 1);
}

template <int Q, int S>
static cudaError_t sweep_t(const Grid &g, const void *fin, void *fout, const uint8_t *flags,
                           float beta, int bgk, int *err, cudaStream_t s) {
  using T = typename Store<S>::T;
  dim3 b = sweep_block(g);
  dim3 grid((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
  if (flags)
    k_sweep<Q, S, true><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  else
    k_sweep<Q, S, false><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  return cudaGetLastError();
}

#define KBC_DISPATCH(Q, storage, ...)                                               \
  do {                                                                              \
    if (Q == 9) {                                                                   \
      if (storage == STORE_F32) { constexpr int QQ = 9, SS = STORE_F32; __VA_ARGS__; }     \
      if (storage == STORE_F16) { constexpr int QQ = 9, SS = STORE_F16; __VA_ARGS__; }     \
      if (storage == STORE_BF16) { constexpr int QQ = 9, SS = STORE_BF16; __VA_ARGS__; }   \
    } else if (Q == 27) {                                                           \
      if (storage == STORE_F32) { constexpr int QQ = 27, SS = STORE_F32; __VA_ARGS__; }    \
      if (storage == STORE_F16) { constexpr int QQ = 27, SS = STORE_F16; __VA_ARGS__; }    \
      if (storage == STORE_BF16) { constexpr int QQ = 27, SS = STORE_BF16; __VA_ARGS__; }  \
    }                                                                               \
    return cudaErrorInvalidValue;                                                   \
  } while (0)

cudaError_t launch_sweep(int Q, int storage, const Grid &g, const void *fin, void *fout,
                         const uint8_t *flags, float beta, int bgk, int *err, cudaStream_t s) {
  KBC_DISPATCH(Q, storage, return (sweep_t<QQ, SS>(g, fin, fout, flags, beta, bgk, err, s)));
}

// ---------------------------------------------------------------- conversions
// Linear interior index -> stored index.
__device__ __forceinline__ long long interior_to_stored(const Grid &g, long long n) {
  const int x = (int)(n % g.nx);
  const long long r = n / g.nx;
  const int y = (int)(r % g.ny);
  const int z = (int)(r / g.ny);
  return sidx(g, x + g.px, y + g.py, z + g.pz);
}

// Entropic equilibrium in FP64 (product form of the minimiser of Eq. feq_min).
template <class L>
__device__ double feq_fp64(int i, double rho, double ux, double uy, double uz) {
  double p = rho;
  const double u[3] = {ux, uy, uz};
  const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const double S = sqrt(1.0 + 3.0 * u[a] * u[a]);
    double f = w1d(c[a]) * (2.0 - S);
    if (c[a] == 1) f *= (2.0 * u[a] + S) / (1.0 - u[a]);
    if (c[a] == -1) f *= (S - 2.0 * u[a]) / (1.0 + u[a]);
    p *= f;
  }
  return p;
}

template <int Q, int S>
__global__ void k_init_eq(Grid g, const double *__restrict__ rho, const double *__restrict__ u,
                          long long ustride, long long begin, long long count,
                          typename Store<S>::T *__restrict__ f) {
  using L = Lat<Q>;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long k = interior_to_stored(g, begin + t);
  const double r = rho[t], ux = u[t], uy = u[ustride + t], uz = (L::D == 3) ? u[2 * ustride + t] : 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double w = weight<L>(i);
    f[(long long)i * g.N + k] = Store<S>::encode(feq_fp64<L>(i, r, ux, uy, uz) - w, w);
  }
}

template <int Q, int S>
__global__ void k_set_pop(Grid g, int i, const double *__restrict__ src, long long begin,
                          long long count, typename Store<S>::T *__restrict__ f) {
  using L = Lat<Q>;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long k = interior_to_stored(g, begin + t);
  double w = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j)
    if (j == i) w = weight<L>(j);
  f[(long long)i * g.N + k] = Store<S>::encode(src[t] - w, w);
}

template <int Q, int S>
__global__ void k_get_pop(Grid g, int i, double *__restrict__ dst, long long begin,
                          long long count, const typename Store<S>::T *__restrict__ f) {
  using L = Lat<Q>;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long k = interior_to_stored(g, begin + t);
  double w = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j)
    if (j == i) w = weight<L>(j);
  dst[t] = w + Store<S>::decode(f[(long long)i * g.N + k], w);
}

template <int Q, int S>
__global__ void k_macros(Grid g, const typename Store<S>::T *__restrict__ f,
                         const uint8_t *__restrict__ flags, double *__restrict__ rho,
                         double *__restrict__ u, long long ustride, long long begin,
                         long long count) {
  using L = Lat<Q>;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long k = interior_to_stored(g, begin + t);
  double r = 0, jx = 0, jy = 0, jz = 0;
  if (!flags || flags[k] == NODE_FLUID) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double w = weight<L>(i);
      const double v = w + Store<S>::decode(f[(long long)i * g.N + k], w);
      r += v;
      jx += L::cx(i) * v;
      jy += L::cy(i) * v;
      jz += L::cz(i) * v;
    }
    jx /= r; jy /= r; jz /= r;
  }
  rho[t] = r;
  u[t] = jx;
  u[ustride + t] = jy;
  if (L::D == 3) u[2 * ustride + t] = jz;
}

static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_init_eq(int Q, int storage, const Grid &g, const double *rho, const double *u,
                           long long ustride, long long begin, long long count, void *f,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    k_init_eq<QQ, SS><<<nblk(count, 256), 256, 0, s>>>(g, rho, u, ustride, begin, count,
                                                       (typename Store<SS>::T *)f);
    return cudaGetLastError();
  });
}

cudaError_t launch_set_pop(int Q, int storage, const Grid &g, int i, const double *src,
                           long long begin, long long count, void *f, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    k_set_pop<QQ, SS><<<nblk(count, 256), 256, 0, s>>>(g, i, src, begin, count,
                                                       (typename Store<SS>::T *)f);
    return cudaGetLastError();
  });
}

cudaError_t launch_get_pop(int Q, int storage, const Grid &g, int i, double *dst,
                           long long begin, long long count, const void *f, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    k_get_pop<QQ, SS><<<nblk(count, 256), 256, 0, s>>>(g, i, dst, begin, count,
                                                       (const typename Store<SS>::T *)f);
    return cudaGetLastError();
  });
}

cudaError_t launch_macros(int Q, int storage, const Grid &g, const void *f, const uint8_t *flags,
                          double *rho, double *u, long long ustride, long long begin,
                          long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    k_macros<QQ, SS><<<nblk(count, 256), 256, 0, s>>>(
        g, (const typename Store<SS>::T *)f, flags, rho, u, ustride, begin, count);
    return cudaGetLastError();
  });
}

}  // namespace kbc
