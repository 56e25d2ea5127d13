// fem_beam.cuh -- device data of the GPU beam (shared with the batched launch).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kbc {

constexpr int kMaxBeamNodes = 48;

struct BeamParams {
  int nn;
  double EA, EI, rhoA, h;
  double theta, lambda, rtol, atol, dt;
  int max_it;
  double accept_tol;   // > 0: accept the initial guess when |R| <= accept_tol |F_ext|
  int solve64;         // 1: Newton matrix and solve in FP64, 0: in FP32 (inexact Newton)
  // spanwise extrusion (quasi-2-D coupling to a D3Q27 lattice periodic in z):
  // the flag polygon's vertices at z = z0 start at the coupling's first
  // vertex, those at z = z1 at v1; loads per unit span are the four vertex
  // forces of a node summed and times inv_depth
  int span, v1;
  double z0, z1, inv_depth;
};

struct BeamDev {
  const double *X;     // [nn][2]
  const int32_t *fixed;
  double *u, *v, *F0;  // [3nn] state and previous loads
  int *iters;          // last step's Newton iteration count (negative: not converged)
  const double *u_guess;  // [3nn] Newton initial guess (nullptr: the current state)
  int *stats;          // accepted / rejected guesses, Newton solves, steps
  const double *M;     // [3nn][11] consistent mass matrix, band storage (constant)
};

// A coupled beam of a batch: its state and the surface arrays of its lattice.
struct BeamBatchDesc {
  BeamParams p;
  BeamDev d;
  const double *vforce;
  double *surf_x, *surf_v;
  int v0;
};

}  // namespace kbc
