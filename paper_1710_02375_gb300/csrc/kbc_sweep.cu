// kbc_sweep.cu -- the fused pull-stream + KBC collision sweep and the
// population conversion kernels.
//
// One thread per interior node, x fastest across the warp so that all Q loads
// and Q stores of a warp are coalesced (the +-x neighbours are one element
// off and come from the same L1/L2 lines).  The sweep reads Q populations and
// writes Q populations per node: 2 Q bytes_per_population of algorithmic HBM
// traffic, Eq. (f_equations); the collision (kbc_collide.cuh) stays in
// registers.  No tensor cores: there is no contraction on this path.
#include "bulk.cuh"
#include "kbc_collide.cuh"
#include "lbm_internal.h"
#include "sweep_io.cuh"

#include <string.h>

// Resident CTAs per SM the register allocation is sized for (128 threads
// each): five keep the D3Q27 kernels at <= 96 registers without spills.
#ifndef KBC_MIN_CTAS
#define KBC_MIN_CTAS 5
#endif

namespace kbc {

// One node (interior coordinates x, y, z) of the fused sweep.  IX: index
// type of the population offsets (32-bit when Q N < 2^31: fewer address
// instructions per load and store).
template <int Q, int S, bool FLAGS, typename IX = long long>
__device__ __forceinline__ void sweep_node(const Grid &g,
                                           const typename Store<S>::T *__restrict__ fin,
                                           typename Store<S>::T *__restrict__ fout,
                                           const uint8_t *__restrict__ flags,
                                           typename Store<S>::C beta, int bgk,
                                           int *__restrict__ err, int x, int y, int z) {
  using L = Lat<Q>;
  using C = typename Store<S>::C;
  const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
  const IX k = (IX)sidx(g, X, Y, Z);
  if (FLAGS && flags[k] != NODE_FLUID) return;
  C v[Q];
  sweep_gather<Q, S, IX>(g, fin, X, Y, Z, v);
  // the conservation projection removes FP32 rounding residue (FP32 storage)
  const C rho = collide_v<L, S == STORE_F32, C>(v, beta, bgk != 0);
  if (!(rho > 0.f && rho < 1e30f)) atomicOr(err, 1);
  sweep_scatter<Q, S, IX>(g, fout, k, v);
}

// Resident CTAs per SM for the direct sweep, measured on the periodic 128^3
// D3Q27 lattice: FP32 storage 5 / 6 / 7 / 8 CTAs -> 84.6 / 81.9 / 84.4 /
// 88.8 us per sweep (6: 80 registers, a few bytes of spills to L1); 16-bit
// storage 72.0 / 69.6 / 68.7 / 70.5 us.
template <int Q, int S>
struct SweepOcc {
  static constexpr int ctas = (Q == 27 && S != STORE_F32) ? 7 : 6;
};

template <int Q, int S, bool FLAGS, typename IX>
__global__ void __launch_bounds__(128, SweepOcc<Q, S>::ctas)
    k_sweep(Grid g, const typename Store<S>::T *__restrict__ fin,
            typename Store<S>::T *__restrict__ fout, const uint8_t *__restrict__ flags,
            typename Store<S>::C beta, int bgk, int *__restrict__ err) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  sweep_node<Q, S, FLAGS, IX>(g, fin, fout, flags, beta, bgk, err, x, y, z);
}


// ---------------------------------------------------------------- two-node sweep
// Each thread takes the stored columns (X, X + 1), X even, of one row: the
// c_x = 0 sources of both nodes are one aligned two-element load, the c_x =
// +-1 sources two single loads, and the collision of both nodes runs on the
// paired FP32 instructions (collide_v with V = f2).  Nodes of the pair that
// are ghosts, solid or in the row padding are computed on whatever their
// slots hold and never stored (their loads stay inside the row: x sources
// wrap with nbr), so the written populations are those of the one-node
// sweep.  Pairs of a row: X = 0, 2, .. covering the interior columns
// [px, px + nx).
template <int Q, int S, typename IX>
__device__ __forceinline__ void sweep_pair_gather(const Grid &g,
                                                  const typename Store<S>::T *__restrict__ fin,
                                                  int X, int Y, int Z, f2 (&v)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
  // source x of the first / second node for cx = -1, 0, +1
  const int xa[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};
  const int xb[3] = {nbr(X + 1, 1, g.NX), X + 1, X};
  const int ys[3] = {nbr(Y, 1, g.NY), Y, nbr(Y, -1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, 1, g.NZ);
    zs[2] = nbr(Z, -1, g.NZ);
  }
  const IX N = (IX)g.N;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::cx(i);
    const IX row = ((IX)zs[L::cz(i) + 1] * (IX)g.NY + (IX)ys[L::cy(i) + 1]) * (IX)g.pitch + (IX)i * N;
    const float w = (float)weight<L>(i);
    if (cx == 0) {
      v[i] = f2{St::load2(fin + (row + (IX)X), w)};
    } else {
      v[i] = mk2(St::load(fin + (row + (IX)xa[cx + 1]), w), St::load(fin + (row + (IX)xb[cx + 1]), w));
    }
  }
}

// Resident 128-thread CTAs per SM the two-node D3Q27 kernel's registers are
// sized for.
#ifndef KBC_PAIR_CTAS27
#define KBC_PAIR_CTAS27 3
#endif
template <int Q, int S>
struct Sweep2Occ {
  static constexpr int ctas = Q == 27 ? KBC_PAIR_CTAS27 : 5;
};

template <int Q, int S, bool FLAGS, typename IX>
__global__ void __launch_bounds__(128, Sweep2Occ<Q, S>::ctas)
    k_sweep2(Grid g, const typename Store<S>::T *__restrict__ fin,
             typename Store<S>::T *__restrict__ fout, const uint8_t *__restrict__ flags, float beta,
             int bgk, int *__restrict__ err) {
  using L = Lat<Q>;
  using St = Store<S>;
  const int X = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (X >= g.px + g.nx || y >= g.ny) return;
  const int Y = y + g.py, Z = z + g.pz;
  const IX k = (IX)sidx(g, X, Y, Z);
  bool ia = X >= g.px, ib = X + 1 < g.px + g.nx;
  if (FLAGS) {
    const uint16_t fl = *reinterpret_cast<const uint16_t *>(flags + k);
    ia = ia && (fl & 0xFFu) == NODE_FLUID;
    ib = ib && (fl >> 8) == NODE_FLUID;
    if (!ia && !ib) return;
  }
  f2 v[Q];
  sweep_pair_gather<Q, S, IX>(g, fin, X, Y, Z, v);
  const f2 rho = collide_v<L, S == STORE_F32, f2>(v, beta, bgk != 0);
  if ((ia && !(rho.v.x > 0.f && rho.v.x < 1e30f)) || (ib && !(rho.v.y > 0.f && rho.v.y < 1e30f)))
    atomicOr(err, 1);
  const IX N = (IX)g.N;
  if (ia && ib) {
#pragma unroll
    for (int i = 0; i < Q; ++i) St::store2(fout + ((IX)i * N + k), v[i].v, (float)(1.0 / weight<L>(i)));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float iw = (float)(1.0 / weight<L>(i));
      if (ia) St::store(fout + ((IX)i * N + k), v[i].v.x, iw);
      if (ib) St::store(fout + ((IX)i * N + k + 1), v[i].v.y, iw);
    }
  }
}

static dim3 sweep2_block(int npairs) {
  if (npairs >= 128) return dim3(128, 1, 1);
  if (npairs >= 64) return dim3(64, 2, 1);
  return dim3(32, 4, 1);
}

template <int Q, int S>
static cudaError_t sweep2_t(const Grid &g, const void *fin, void *fout, const uint8_t *flags,
                            float beta, int bgk, int *err, cudaStream_t s) {
  using T = typename Store<S>::T;
  const int npairs = (g.px + g.nx + 1) / 2;
  const dim3 b = sweep2_block(npairs);
  const dim3 grid((npairs + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
  const bool narrow = (long long)Q * g.N < (1LL << 31);
  if (flags && narrow)
    k_sweep2<Q, S, true, int><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  else if (flags)
    k_sweep2<Q, S, true, long long><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk,
                                                       err);
  else if (narrow)
    k_sweep2<Q, S, false, int><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  else
    k_sweep2<Q, S, false, long long><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta,
                                                        bgk, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- row-staged sweep
// Persistent form of the same sweep.  A CTA walks output rows (y, z) of the
// interior; for each it fetches, with the bulk-copy engine, the Q source rows
// (direction i, row (y - cy_i, z - cz_i)) into a shared-memory stage, so each
// input row crosses HBM exactly once and the memory pipeline runs ahead of the
// collision by `stages - 1` rows without holding registers.  Threads read
// their node's Q populations from the stage (x shift and periodic wrap
// resolved in shared memory), collide in registers and store coalesced.
constexpr uint32_t kMaxSpins = 1u << 22;  // bounded mbarrier waits

template <int Q, int S, bool FLAGS>
__global__ void __launch_bounds__(128, KBC_MIN_CTAS)
    k_sweep_rows(Grid g, const typename Store<S>::T *__restrict__ fin,
                 typename Store<S>::T *__restrict__ fout, const uint8_t *__restrict__ flags,
                 float beta, int bgk, int *__restrict__ err, int row_bytes, int stages) {
  using L = Lat<Q>;
  using St = Store<S>;
  using T = typename St::T;
  extern __shared__ __align__(128) unsigned char smem[];
  // per stage: a "full" barrier (bulk copies landed) and an "empty" barrier
  // (every warp has read the stage); no CTA-wide barrier inside the loop
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * Q * row_bytes);
  uint64_t *empty = full + stages;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nwarps = (int)blockDim.x >> 5;
  const int nrows = g.ny * g.nz;
  if ((int)blockIdx.x >= nrows) return;
  const int my_rows = (nrows - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int row_elems = row_bytes / (int)sizeof(T);

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nwarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int j, int s) {
    const int r = (int)blockIdx.x + j * (int)gridDim.x;
    const int Y = r % g.ny + g.py, Z = r / g.ny + g.pz;
    mbar_arrive_expect_tx(&full[s], (uint32_t)(Q * row_bytes));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int Ys = nbr(Y, -L::cy(i), g.NY);
      const int Zs = (L::D == 3) ? nbr(Z, -L::cz(i), g.NZ) : Z;
      const T *src = fin + (long long)i * g.N + ((long long)Zs * g.NY + Ys) * g.pitch;
      bulk_g2s(smem + ((size_t)s * Q + i) * row_bytes, src, (uint32_t)row_bytes, &full[s]);
    }
  };

  if (tid == 0) {
    const int pre = my_rows < stages ? my_rows : stages;
    for (int j = 0; j < pre; ++j) issue(j, j);
  }
  const int groups = (g.nx + (int)blockDim.x - 1) / (int)blockDim.x;
  bool timed_out = false;

  for (int j = 0; j < my_rows; ++j) {
    const int s = j % stages;
    if (!mbar_wait_bounded(&full[s], (uint32_t)((j / stages) & 1), kMaxSpins)) timed_out = true;
    // refill the stage released one row earlier (its readers are past it)
    if (tid == 0 && j >= 1 && j - 1 + stages < my_rows) {
      const int sp = (j - 1) % stages;
      if (!mbar_wait_bounded(&empty[sp], (uint32_t)(((j - 1) / stages) & 1), kMaxSpins))
        timed_out = true;
      fence_proxy_async_smem();
      issue(j - 1 + stages, sp);
    }
    const int r = (int)blockIdx.x + j * (int)gridDim.x;
    const int Y = r % g.ny + g.py, Z = r / g.ny + g.pz;
    const long long k0 = sidx(g, 0, Y, Z);
    const T *stage = reinterpret_cast<const T *>(smem + (size_t)s * Q * row_bytes);

    for (int grp = 0; grp < groups; ++grp) {
      const int x = grp * (int)blockDim.x + tid;
      const bool active = x < g.nx;
      const int X = (active ? x : 0) + g.px;
      const int xs[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};
      float v[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i)
        v[i] = St::load_smem(stage + i * row_elems + xs[L::cx(i) + 1], (float)weight<L>(i));
      if (grp == groups - 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
      }
      if (active && (!FLAGS || flags[k0 + X] == NODE_FLUID)) {
        const float rho = collide<L, S == STORE_F32>(v, beta, bgk != 0);
        if (!(rho > 0.f && rho < 1e30f)) atomicOr(err, 1);
        T *po = fout + k0 + X;
#pragma unroll
        for (int i = 0; i < Q; ++i, po += g.N) St::store(po, v[i], (float)(1.0 / weight<L>(i)));
      }
    }
  }
  if (timed_out) atomicOr(err, 2);
  // a copy can only still be in flight after a timed-out wait: let it land
  // (bounded) before the CTA's shared memory is released
  if (tid == 0 && timed_out)
    for (int s = 0; s < stages; ++s) {
      const int jl = my_rows - 1 - ((my_rows - 1 - s) % stages + stages) % stages;
      if (jl >= 0) mbar_wait_bounded(&full[s], (uint32_t)((jl / stages) & 1), kMaxSpins);
    }
}

struct RowPlan {
  int ok = 0, stages = 0, blocks = 0, row_bytes = 0;
  size_t smem = 0;
};

template <int Q, int S, bool FLAGS>
static RowPlan plan_rows(const Grid &g) {
  RowPlan p;
  using T = typename Store<S>::T;
  p.row_bytes = (int)(((size_t)g.NX * sizeof(T) + 15) / 16 * 16);
  int dev = 0, sms = 0, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  auto kern = k_sweep_rows<Q, S, FLAGS>;
  int best_score = 0;
  for (int st = 4; st >= 2; --st) {
    const size_t smem = (size_t)st * Q * p.row_bytes + 2 * (size_t)st * sizeof(uint64_t);
    if (smem > (size_t)smem_optin) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 128, smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int score = nb * (st - 1) * 4 + nb;  // rows in flight, then resident warps
    if (nb >= 2 && score > best_score) {
      best_score = score;
      p.ok = 1;
      p.stages = st;
      p.blocks = nb * sms;
      p.smem = smem;
    }
  }
  if (p.ok) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  return p;
}

template <int Q, int S>
static cudaError_t sweep_rows_t(const Grid &g, const void *fin, void *fout, const uint8_t *flags,
                                float beta, int bgk, int *err, cudaStream_t s, bool *used) {
  using T = typename Store<S>::T;
  // plans are cached per (template, lattice shape)
  static thread_local Grid last_g[2] = {};
  static thread_local RowPlan last_p[2] = {};
  const int fi = flags ? 1 : 0;
  if (memcmp(&last_g[fi], &g, sizeof(Grid)) != 0 || !last_p[fi].ok) {
    last_p[fi] = flags ? plan_rows<Q, S, true>(g) : plan_rows<Q, S, false>(g);
    last_g[fi] = g;
  }
  const RowPlan &p = last_p[fi];
  *used = p.ok != 0;
  if (!p.ok) return cudaSuccess;
  const int nrows = g.ny * g.nz;
  const int grid = p.blocks < nrows ? p.blocks : nrows;
  if (flags)
    k_sweep_rows<Q, S, true><<<grid, 128, p.smem, s>>>(g, (const T *)fin, (T *)fout, flags, beta,
                                                       bgk, err, p.row_bytes, p.stages);
  else
    k_sweep_rows<Q, S, false><<<grid, 128, p.smem, s>>>(g, (const T *)fin, (T *)fout, flags, beta,
                                                        bgk, err, p.row_bytes, p.stages);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- prefetching sweep
// FP32 form with per-thread double buffering: while a thread collides the
// node of row j, cp.async copies of the 27 source values of its node in row
// j+1 are already in flight into shared memory, so the memory pipeline stays
// full without holding registers.  A CTA owns one x-segment of 128 nodes over
// `rows_per_cta` consecutive interior rows; no CTA barriers.
template <int Q, bool FLAGS>
__global__ void __launch_bounds__(128, KBC_MIN_CTAS)
    k_sweep_async(Grid g, const float *__restrict__ fin, float *__restrict__ fout,
                  const uint8_t *__restrict__ flags, float beta, int bgk, int *__restrict__ err,
                  int rows_per_cta) {
  using L = Lat<Q>;
  __shared__ float buf[2][Q][128];
  const int tid = threadIdx.x;
  const int x = blockIdx.x * 128 + tid;
  const bool active = x < g.nx;
  const int X = (active ? x : 0) + g.px;
  const int xs[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};
  const int nrows = g.ny * g.nz;
  const int r0 = blockIdx.y * rows_per_cta;
  const int rend = min(r0 + rows_per_cta, nrows);

  auto prefetch = [&](int r, int b) {
    const int Y = r % g.ny + g.py, Z = r / g.ny + g.pz;
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
      cp_async4(&buf[b][i][tid], fin + (long long)i * g.N + src);
    }
  };

  if (r0 < rend) prefetch(r0, 0);
  cp_async_commit();
  for (int r = r0; r < rend; ++r) {
    const int b = (r - r0) & 1;
    if (r + 1 < rend) prefetch(r + 1, b ^ 1);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of row r have landed
    float v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = buf[b][i][tid];
    const int Y = r % g.ny + g.py, Z = r / g.ny + g.pz;
    const long long k = sidx(g, X, Y, Z);
    if (active && (!FLAGS || flags[k] == NODE_FLUID)) {
      const float rho = collide<L, true>(v, beta, bgk != 0);
      if (!(rho > 0.f && rho < 1e30f)) atomicOr(err, 1);
      float *po = fout + k;
#pragma unroll
      for (int i = 0; i < Q; ++i, po += g.N) *po = v[i];
    }
  }
}

template <int Q>
static cudaError_t sweep_async_t(const Grid &g, const void *fin, void *fout, const uint8_t *flags,
                                 float beta, int bgk, int *err, cudaStream_t s) {
  const int rows_per_cta = 8;
  const int nrows = g.ny * g.nz;
  dim3 grid((g.nx + 127) / 128, (nrows + rows_per_cta - 1) / rows_per_cta, 1);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (flags)
    k_sweep_async<Q, true><<<grid, 128, 0, s>>>(g, (const float *)fin, (float *)fout, flags, beta,
                                                bgk, err, rows_per_cta);
  else
    k_sweep_async<Q, false><<<grid, 128, 0, s>>>(g, (const float *)fin, (float *)fout, flags, beta,
                                                 bgk, err, rows_per_cta);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched sweep
// Persistent CTAs take tiles (lattice, first row, x segment of 128 nodes)
// from an atomic ticket until the list is exhausted; lattices of any shape
// share one launch.  Block 0 also advances every lattice's inlet-ramp clock
// (this kernel runs after the boundary fill of the step).
// Up to R consecutive interior rows (r0 .. r0 + m - 1) of one x column:
// every row's populations are gathered before the first collision, so a
// thread keeps R nodes' loads in flight (the D2Q9 node has little arithmetic
// to hide a load's latency behind).
template <int Q, int S, int R>
__device__ __forceinline__ void sweep_rows(const Grid &g, const typename Store<S>::T *__restrict__ fin,
                                           typename Store<S>::T *__restrict__ fout,
                                           const uint8_t *__restrict__ flags,
                                           typename Store<S>::C beta, int bgk,
                                           int *__restrict__ err, int x, int r0, int m) {
  using L = Lat<Q>;
  using C = typename Store<S>::C;
  C v[R][Q];
  int k[R];
  bool live[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = r0 + q;
    const int X = x + g.px, Y = r % g.ny + g.py, Z = r / g.ny + g.pz;
    k[q] = (int)sidx(g, X, Y, Z);
    live[q] = q < m && flags[k[q]] == NODE_FLUID;
    if (live[q]) sweep_gather<Q, S, int>(g, fin, X, Y, Z, v[q]);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (!live[q]) continue;
    const C rho = collide_v<L, S == STORE_F32, C>(v[q], beta, bgk != 0);
    if (!(rho > 0.f && rho < 1e30f)) atomicOr(err, 1);
    sweep_scatter<Q, S, int>(g, fout, k[q], v[q]);
  }
}

template <int Q, int S>
__global__ void __launch_bounds__(128, KBC_MIN_CTAS)
    k_sweep_batch(const InstDesc *__restrict__ d, int n, const int4 *__restrict__ tiles,
                  int ntiles, int *ticket, int parity, int rows_per_tile) {
  using T = typename Store<S>::T;
  __shared__ int s_tile;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (d[i].bp.ramp_steps > 0 && d[i].bp.step) atomicAdd((int *)d[i].bp.step, 1);
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= ntiles) break;
    const int4 tl = tiles[tile];
    const InstDesc &b = d[tl.x];
    const T *fin = (const T *)b.f[(b.cur0 + parity) & 1];
    T *fout = (T *)b.f[(b.cur0 + parity + 1) & 1];
    const int x = tl.z * 128 + threadIdx.x;
    const int nrows = b.g.ny * b.g.nz;
    const int rend = min(tl.y + rows_per_tile, nrows);
    if (x < b.g.nx) {
      if (Q == 9 && b.narrow) {
        for (int r = tl.y; r < rend; r += 4)
          sweep_rows<Q, S, 4>(b.g, fin, fout, b.flags, (typename Store<S>::C)b.beta, b.bgk, b.err,
                              x, r, rend - r);
      } else {
        for (int r = tl.y; r < rend; ++r)
          sweep_node<Q, S, true>(b.g, fin, fout, b.flags, (typename Store<S>::C)b.beta, b.bgk,
                                 b.err, x, r % b.g.ny,
                                 r / b.g.ny);
      }
    }
  }
}

cudaError_t launch_sweep_batch(int Q, int storage, const InstDesc *d, int n, const int4 *tiles,
                               int ntiles, int *ticket, int parity, int rows_per_tile,
                               int ctas_per_sm, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = sms * ctas_per_sm;
  if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
  KBC_DISPATCH(Q, storage, {
    k_sweep_batch<QQ, SS><<<grid, 128, 0, s>>>(d, n, tiles, ntiles, ticket, parity,
                                                rows_per_tile);
    return cudaGetLastError();
  });
}

static dim3 sweep_block(const Grid &g) {
  if (g.nx >= 128) return dim3(128, 1, 1);
  if (g.nx >= 64) return dim3(64, 2, 1);
  return dim3(32, 4, 1);
}

template <int Q, int S>
static cudaError_t sweep_t(const Grid &g, const void *fin, void *fout, const uint8_t *flags,
                           double beta_d, int bgk, int *err, cudaStream_t s, int variant) {
  using T = typename Store<S>::T;
  using C = typename Store<S>::C;
  const C beta = (C)beta_d;
  // FP64 storage: the one-node kernel only
  if constexpr (S != STORE_F64) {
    if (variant == SWEEP_ASYNC && S == STORE_F32 && (long long)g.ny * g.nz <= 65535LL * 8)
      return sweep_async_t<Q>(g, fin, fout, flags, beta, bgk, err, s);
    if (variant == SWEEP_ROWS) {
      bool used = false;
      cudaError_t e = sweep_rows_t<Q, S>(g, fin, fout, flags, beta, bgk, err, s, &used);
      if (e != cudaSuccess || used) return e;
    }
    if (variant == SWEEP_AUTO || variant == SWEEP_PAIR)
      return sweep2_t<Q, S>(g, fin, fout, flags, beta, bgk, err, s);
  }
  dim3 b = sweep_block(g);
  dim3 grid((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
  const bool narrow = (long long)Q * g.N < (1LL << 31);  // every offset fits an int
  if (flags && narrow)
    k_sweep<Q, S, true, int><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  else if (flags)
    k_sweep<Q, S, true, long long><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk,
                                                      err);
  else if (narrow)
    k_sweep<Q, S, false, int><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk, err);
  else
    k_sweep<Q, S, false, long long><<<grid, b, 0, s>>>(g, (const T *)fin, (T *)fout, flags, beta, bgk,
                                                       err);
  return cudaGetLastError();
}



cudaError_t launch_sweep(int Q, int storage, const Grid &g, const void *fin, void *fout,
                         const uint8_t *flags, double beta, int bgk, int *err, cudaStream_t s,
                         int variant) {
  KBC_DISPATCH(Q, storage,
               return (sweep_t<QQ, SS>(g, fin, fout, flags, beta, bgk, err, s, variant)));
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
                         long long count, float *__restrict__ rho32, float *__restrict__ u32) {
  using L = Lat<Q>;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const long long k = interior_to_stored(g, begin + t);
  double r = 0, ux = 0, uy = 0, uz = 0;
  if (!flags || flags[k] == NODE_FLUID) {
    // sums of the stored deviations in FP32 (exact to the storage precision),
    // rho = 1 + sum and u = j / rho in FP64
    using C = typename Store<S>::C;
    C dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const C v = Store<S>::load(f + (long long)i * g.N + k, (C)weight<L>(i));
      dr += v;
      jx += L::cx(i) * v;
      jy += L::cy(i) * v;
      jz += L::cz(i) * v;
    }
    if (rho32) {
      // FP32 outputs: rho and u = j / rho in FP32
      const float rf = 1.f + (float)dr, ir = 1.f / rf;
      rho32[t] = rf;
      u32[t] = (float)jx * ir;
      u32[ustride + t] = (float)jy * ir;
      if (L::D == 3) u32[2 * ustride + t] = (float)jz * ir;
      return;
    }
    r = 1.0 + (double)dr;
    ux = (double)jx / r;
    uy = (double)jy / r;
    uz = (double)jz / r;
  }
  if (rho32) {
    rho32[t] = 0.f;
    u32[t] = 0.f;
    u32[ustride + t] = 0.f;
    if (L::D == 3) u32[2 * ustride + t] = 0.f;
    return;
  }
  rho[t] = r;
  u[t] = ux;
  u[ustride + t] = uy;
  if (L::D == 3) u[2 * ustride + t] = uz;
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
                          long long count, cudaStream_t s, float *rho32, float *u32) {
  if (count <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    k_macros<QQ, SS><<<nblk(count, 256), 256, 0, s>>>(
        g, (const typename Store<SS>::T *)f, flags, rho, u, ustride, begin, count, rho32, u32);
    return cudaGetLastError();
  });
}

}  // namespace kbc
