// boundary.cuh -- device data of the boundary treatment.
#pragma once
#include <stdint.h>

#include "kbc_common.cuh"

namespace kbc {

// face boundary kinds (values of the C ABI)
enum { BCK_PERIODIC = 0, BCK_WALL = 1, BCK_INLET = 2, BCK_OUTLET = 3, BCK_FREESTREAM = 4 };

// A fluid node with at least one missing population (its source x - c_i is
// solid or a ghost beyond a non-periodic face).
struct BNode {
  int64_t k;      // stored linear index
  int link0;      // first immersed link of the node in the link array (-1: none)
  int nlink;      // number of immersed links (ascending direction order)
};

// An immersed cut link: fluid node -> solid source along -c_i, crossing the
// surface at x_b - q c_i on element `elem`.
struct Link {
  int i;          // direction of the missing population
  int body;       // body of the hit element
  float q;        // wall distance fraction in (0, 1]
  float uw[3];    // wall velocity at the crossing
  int v[3];       // vertices of the hit element (2 used in 2-D)
  float vw[3];    // interpolation weights of those vertices
};

struct SurfaceDev {
  int dim, nv, ne, nb;
  const double *x;     // [nv][dim] vertex positions (lattice units)
  const double *v;     // [nv][dim] vertex velocities
  const int32_t *e;    // [ne][dim] element vertex ids
  const int32_t *eb;   // [ne] body id
  float *box;          // [6] bounding box of the vertices (lo xyz, hi xyz), or nullptr
};

struct Band {          // box of interior coordinates, inclusive lower, exclusive upper
  int x0, x1, y0, y1, z0, z1;
};

struct BoundaryParams {
  int bc[6];
  float face_u[6][3];
  const float *inlet[6];  // per face [3][face nodes] prescribed velocity or nullptr
  double beta;
  int ramp_steps;         // inlet velocity ramp (1 - cos(pi t / T)) / 2, 0 = none
  const int *step;        // device step counter (ramp clock)
};

// One lattice of a batch (all device pointers point into its own workspace).
struct InstDesc {
  Grid g;
  void *f[2];             // population buffers; step parity p reads f[(cur0 + p) & 1]
  int cur0;
  uint8_t *flags;
  double beta;
  int bgk;
  int *err;
  int narrow;             // Q N < 2^31: 32-bit population offsets in the sweep
  // boundary fill and force
  BNode *bnodes;          // face nodes, then immersed nodes
  int *nbn;               // immersed node counter (nullptr: no bodies)
  int nfixed, cap;
  Link *links;
  BoundaryParams bp;
  double *vforce, *bforce;
  int nbodies, nv;
  // geometry rebuild (moving surface)
  int coupled;
  Band band;
  SurfaceDev sd;
  int64_t *fresh;
  int *nfresh;
  int *nl;
  int lcap;
};

// Stored coordinates of the linear stored index k.
__device__ __forceinline__ void decompose(const Grid &g, long long k, int &X, int &Y, int &Z) {
  X = (int)(k % g.pitch);
  const long long r = k / g.pitch;
  Y = (int)(r % g.NY);
  Z = (int)(r / g.NY);
}

}  // namespace kbc
