// sweep_io.cuh -- the pull of one node's populations from their source nodes
// and the store of its post-collision values (shared by the single-phase and
// the multiphase sweeps).
#pragma once
#include "kbc_common.cuh"

namespace kbc {

// Pull of the Q populations of stored node (X, Y, Z) from their sources
// (X - c_i), and the store of the post-collision values at stored index k.
template <int Q, int S, typename IX>
__device__ __forceinline__ void sweep_gather(const Grid &g,
                                             const typename Store<S>::T *__restrict__ fin, int X,
                                             int Y, int Z, typename Store<S>::C (&v)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
  const int xs[3] = {nbr(X, 1, g.NX), X, nbr(X, -1, g.NX)};  // source x for cx = -1, 0, +1
  const int ys[3] = {nbr(Y, 1, g.NY), Y, nbr(Y, -1, g.NY)};
  int zs[3] = {Z, Z, Z};
  if (L::D == 3) {
    zs[0] = nbr(Z, 1, g.NZ);
    zs[2] = nbr(Z, -1, g.NZ);
  }
  const IX N = (IX)g.N;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const IX src = ((IX)zs[L::cz(i) + 1] * (IX)g.NY + (IX)ys[L::cy(i) + 1]) * (IX)g.pitch +
                   (IX)xs[L::cx(i) + 1];
    v[i] = St::load(fin + ((IX)i * N + src), (typename St::C)weight<L>(i));
  }
}

template <int Q, int S, typename IX>
__device__ __forceinline__ void sweep_scatter(const Grid &g, typename Store<S>::T *__restrict__ fout,
                                              IX k, const typename Store<S>::C (&v)[Q]) {
  using L = Lat<Q>;
  using St = Store<S>;
  const IX N = (IX)g.N;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    St::store(fout + ((IX)i * N + k), v[i], (typename St::C)(1.0 / weight<L>(i)));
}

}  // namespace kbc
