// lbm_internal.h -- launchers shared between the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kbc_common.cuh"

namespace kbc {

// Fused pull-stream + KBC collision over all interior nodes (solid nodes are
// skipped when flags != nullptr).  fin / fout: population buffers in storage
// layout [Q][NZ][NY][NX].  err: device word, bit 0 set on a bad density.
enum { SWEEP_AUTO = 0, SWEEP_DIRECT = 1, SWEEP_ROWS = 2 };
// variant: SWEEP_AUTO / SWEEP_ROWS use the row-staged bulk-copy kernel when its
// shared-memory plan fits, else the direct kernel; SWEEP_DIRECT forces the latter.
cudaError_t launch_sweep(int Q, int storage, const Grid &g, const void *fin, void *fout,
                         const uint8_t *flags, float beta, int bgk, int *err, cudaStream_t s,
                         int variant = SWEEP_AUTO);

// f = feq(rho, u) for interior nodes [begin, begin+count) of the linear
// interior index; rho[count], u[dim][ustride] (FP64, device).
cudaError_t launch_init_eq(int Q, int storage, const Grid &g, const double *rho, const double *u,
                           long long ustride, long long begin, long long count, void *f,
                           cudaStream_t s);

// One direction i of the interface layout, nodes [begin, begin+count):
// FP64 absolute populations <-> storage.
cudaError_t launch_set_pop(int Q, int storage, const Grid &g, int i, const double *src,
                           long long begin, long long count, void *f, cudaStream_t s);
cudaError_t launch_get_pop(int Q, int storage, const Grid &g, int i, double *dst,
                           long long begin, long long count, const void *f, cudaStream_t s);

// rho[count], u[dim][ustride] for interior nodes [begin, begin+count); solid
// nodes give zeros.
cudaError_t launch_macros(int Q, int storage, const Grid &g, const void *f, const uint8_t *flags,
                          double *rho, double *u, long long ustride, long long begin,
                          long long count, cudaStream_t s);

}  // namespace kbc
