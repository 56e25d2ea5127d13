// lbm_internal.h -- launchers shared between the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kbc_lbm.h"
#include "boundary.cuh"
#include "fem_beam.cuh"
#include "kbc_common.cuh"

namespace kbc {

// Dispatch a runtime (lattice, storage) pair to compile-time constants QQ, SS;
// every branch must return.  FP64 storage exists for D2Q9 only.
#define KBC_DISPATCH(Q, storage, ...)                                               \
  do {                                                                              \
    if (Q == 9) {                                                                   \
      if (storage == STORE_F32) { constexpr int QQ = 9, SS = STORE_F32; __VA_ARGS__; }     \
      if (storage == STORE_F16) { constexpr int QQ = 9, SS = STORE_F16; __VA_ARGS__; }     \
      if (storage == STORE_BF16) { constexpr int QQ = 9, SS = STORE_BF16; __VA_ARGS__; }   \
      if (storage == STORE_F16N) { constexpr int QQ = 9, SS = STORE_F16N; __VA_ARGS__; }   \
      if (storage == STORE_F64) { constexpr int QQ = 9, SS = STORE_F64; __VA_ARGS__; }     \
    } else if (Q == 27) {                                                           \
      if (storage == STORE_F32) { constexpr int QQ = 27, SS = STORE_F32; __VA_ARGS__; }    \
      if (storage == STORE_F16) { constexpr int QQ = 27, SS = STORE_F16; __VA_ARGS__; }    \
      if (storage == STORE_BF16) { constexpr int QQ = 27, SS = STORE_BF16; __VA_ARGS__; }  \
      if (storage == STORE_F16N) { constexpr int QQ = 27, SS = STORE_F16N; __VA_ARGS__; }  \
    }                                                                               \
    return cudaErrorInvalidValue;                                                   \
  } while (0)

// Fused pull-stream + KBC collision over all interior nodes (solid nodes are
// skipped when flags != nullptr).  fin / fout: population buffers in storage
// layout [Q][NZ][NY][NX].  err: device word, bit 0 set on a bad density.
enum { SWEEP_AUTO = 0, SWEEP_DIRECT = 1, SWEEP_ROWS = 2, SWEEP_ASYNC = 3, SWEEP_PAIR = 4 };
// variant: SWEEP_AUTO and SWEEP_PAIR use the two-node kernel (paired FP32
// instructions); SWEEP_DIRECT the one-node kernel; SWEEP_ROWS the
// row-staged bulk-copy kernel when its shared-memory plan fits (else the
// one-node kernel).
cudaError_t launch_sweep(int Q, int storage, const Grid &g, const void *fin, void *fout,
                         const uint8_t *flags, double beta, int bgk, int *err, cudaStream_t s,
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
// FP64 outputs rho / u, or FP32 outputs rho32 / u32 when rho32 is given.
cudaError_t launch_macros(int Q, int storage, const Grid &g, const void *f, const uint8_t *flags,
                          double *rho, double *u, long long ustride, long long begin,
                          long long count, cudaStream_t s, float *rho32 = nullptr,
                          float *u32 = nullptr);

// ---- multiphase model (periodic lattices; FP32 storage, or FP64 for D2Q9)
enum { MP_EOS_PAPER = 0, MP_EOS_IDEAL = 1 };
struct MpParams {
  double kappa;    // capillary coefficient
  double g[3];     // uniform acceleration (F gains rho g)
  double kappa_w;  // wetting strength (walls only)
  int eos;         // MP_EOS_*
  int pair;        // FP32: the two-node form of the forced sweep
  int wall;        // axis normal to the two planar walls, -1: fully periodic
};
// Rows of the wall-band scratch per wall side: the fluid velocity and the
// force of the previous step on the first three interior rows.
constexpr int kMpBandRows = 3;
// Bytes of that scratch: 2 sides x 3 rows x 6 values x the largest plane.
inline size_t mp_band_bytes(int nx, int ny, int nz, int cb) {
  const long long a = (long long)nx * ny, b = (long long)ny * nz, c = (long long)nx * nz;
  const long long m = a > b ? (a > c ? a : c) : (b > c ? b : c);
  return (size_t)cb * 2 * kMpBandRows * 6 * (size_t)m;
}
// One multiphase step fin -> fout: density pass (rho, phi), Laplacian pass
// (lap rho), forced sweep.  Populations are stored as f_i - W_i R(x), R the
// node's density of the step that wrote them: fin relative to rref, fout
// relative to the new densities rho.  rref, rho: [N] compute type; pl: [N]
// (phi, lap) pairs.
// ctl: momentum-controller state (kMpControl doubles, zero to start):
// [0..2] the correcting acceleration a_c of the current step (force rho a_c
// subtracted per node), [6..8] the momentum of the step before, [9] the
// number of sweeps with partials (0, 1, 2), [10..11] a_c as three floats;
// partial: kMpPartialDoubles per
// CTA of mp_grid, then the same per group of kMpGroupCtas CTAs
// (mp_partial_bytes).
constexpr int kMpControl = 12;
constexpr int kMpPartialDoubles = 4;
constexpr int kMpGroupCtas = 128;
// With walls (mp.wall >= 0) the step first fills the missing populations
// of the wall nodes into the ghost slots of fin (Grad), using band (scratch
// of mp_band_bytes) and the force of the previous step when have_force.
cudaError_t launch_mp_step(int Q, int storage, const Grid &g, void *fin, void *fout,
                           const void *rref, void *rho, void *pl, double *ctl, double *partial,
                           void *band, int have_force, const MpParams &mp, double beta, int bgk,
                           int *err, cudaStream_t s);
// CTA shape and count of the multiphase kernels over an nx * ny * nz lattice.
struct MpGrid {
  int bx, by;
  long long blocks;
};
inline MpGrid mp_grid(int nx, int ny, int nz) {
  MpGrid m;
  m.bx = nx >= 128 ? 128 : 32;
  m.by = nx >= 128 ? 1 : 4;
  m.blocks = (long long)((nx + m.bx - 1) / m.bx) * ((ny + m.by - 1) / m.by) * nz;
  return m;
}
inline size_t mp_partial_bytes(int nx, int ny, int nz) {
  const long long nb = mp_grid(nx, ny, nz).blocks;
  const long long ng = (nb + kMpGroupCtas - 1) / kMpGroupCtas;
  return sizeof(double) * kMpPartialDoubles * (size_t)(nb + ng);
}
// Read-out of a stored state f relative to rref for interior nodes [begin,
// begin + count): the force of the last step F[3][stride] (when F given; zero
// when !have_force; mean: the controller state ctl, whose correction of the
// last step, ctl[0..2], is subtracted), density and fluid velocity (j - F/2) / rho (FP64 rho_out
// / u, or FP32 rho32 / u32), absolute populations fabs[Q][stride] (FP64).
cudaError_t launch_mp_read(int Q, int storage, const Grid &g, const void *f, const void *rref,
                           const void *pl, const MpParams &mp, int have_force,
                           const double *mean, long long begin,
                           long long count, long long stride, double *F, double *rho_out,
                           double *u, float *rho32, float *u32, double *fabs, cudaStream_t s);
// Change the reference of a stored state to the constant Rnew (populations
// shifted when shift_populations, rref set to Rnew).
cudaError_t launch_mp_rebase(int Q, int storage, const Grid &g, void *f, void *rref, double Rnew,
                             int shift_populations, cudaStream_t s);

// ---- two-level refinement (D2Q9, FP32 or FP64 storage)
struct RefLaunch {
  Grid gc, gf;             // coarse (periodic) and fine (with its ghost layer) grids
  int storage;
  const void *fc_in;       // coarse state at t (post-collision)
  void *fc_out;            // coarse state at t + 1 (the covered cells restricted)
  void *ff[2];             // fine ping-pong buffers
  int cur_f;               // fine buffer holding the state at t (it holds t + 1 after two steps)
  const uint8_t *flags_f;  // fine node flags (ghosts skipped by the sweep)
  double beta_c, beta_f;
  int bgk, variant;
  int i0, j0;              // first covered coarse cell
  void *fields;            // refine_workspace_bytes scratch (set up by launch_refine_init)
  int *err_c, *err_f;
};
// One coarse step of the refined pair (coarse sweep, the sampling pass with
// the Grad fill of the fine boundary nodes, two fine sweeps, restriction).
cudaError_t launch_refine_step(const RefLaunch &R, cudaStream_t s);
// The coarse-cell mask of the scratch (cells the coarse sweep skips); once
// per coupling.
cudaError_t launch_refine_init(const RefLaunch &R, cudaStream_t s);
size_t refine_workspace_bytes(int storage, const Grid &gc, int nfx, int nfy);

}  // namespace kbc

namespace kbc {

cudaError_t launch_mark_ghosts(const Grid &g, uint8_t *flags, cudaStream_t s);
cudaError_t launch_face_nodes(const Grid &g, BNode *out, int *count, int cap, cudaStream_t s);
// Solid flags, fresh-node initialisation (track_fresh) and the immersed
// boundary-node / cut-link lists of the band.
cudaError_t launch_geometry(int Q, int storage, const Grid &g, const Band &bd, const SurfaceDev &sd,
                            uint8_t *flags, void *f, int64_t *fresh, int *nfresh, int fresh_cap,
                            int track_fresh, BNode *bnodes, int *nbn, int bcap, Link *links,
                            int *nl, int lcap, int *err, cudaStream_t s);
// Grad fill of the missing populations of nfixed face nodes followed by
// min(*nbn, cap - nfixed) immersed boundary nodes, and the force gather.
cudaError_t launch_grad(int Q, int storage, const Grid &g, void *f, const uint8_t *flags,
                        const BNode *bnodes, const int *nbn, int nfixed, int cap,
                        const Link *links, const BoundaryParams &bp, double *vforce,
                        double *bforce, int nbodies, cudaStream_t s);
cudaError_t launch_step_counter(int *step, cudaStream_t s);
// Immersed boundary nodes and cut links of the band for the current flags.
// Fluid stress at the immersed boundary nodes (pre-collision state of the
// step in f) and the traction forces it gives on every surface element.
cudaError_t launch_traction(int Q, int storage, const Grid &g, const void *f, const BNode *bn,
                            const int *nbn, int cap, double beta, const SurfaceDev &sd,
                            double *sigma, double *orient, double *vforce, double *bforce,
                            int nbodies, cudaStream_t s);

cudaError_t launch_build_links(int Q, const Grid &g, const Band &bd, const SurfaceDev &sd,
                               const uint8_t *flags, BNode *bnodes, int *nbn, int bcap,
                               Link *links, int *nl, int lcap, int *err, cudaStream_t s);

// batched phases (one launch each for all lattices of a batch)
cudaError_t launch_batch_pre(const InstDesc *d, int n, int max_nv3, int *ticket, cudaStream_t s);
cudaError_t launch_grad_batch(int Q, int storage, const InstDesc *d, int n, int max_cap, int parity,
                              cudaStream_t s);
cudaError_t launch_sweep_batch(int Q, int storage, const InstDesc *d, int n, const int4 *tiles,
                               int ntiles, int *ticket, int parity, int rows_per_tile,
                               int ctas_per_sm, cudaStream_t s);
cudaError_t launch_geometry_batch(int Q, int storage, const InstDesc *d, const int *idx, int n,
                                  long long max_band, int max_fresh, int parity, cudaStream_t s);

int fem_nodes(const fem_ctx *f);
// Spanwise extrusion of a coupled beam's flag (quasi-2-D coupling, D3Q27).
void fem_set_span(fem_ctx *f, int span, int v1, double z0, double z1, double inv_depth);
int fem_span(const fem_ctx *f);
cudaError_t launch_surrogate_input(fem_ctx *f, const double *vforce, int v0, float *xin,
                                   cudaStream_t s);
cudaError_t launch_surrogate_guess(fem_ctx *f, const float *yhat, cudaStream_t s);
cudaError_t launch_beam_coupled_guess(fem_ctx *f, const double *vforce, double *surf_x,
                                      double *surf_v, int v0, double accept_tol, cudaStream_t s);
lbm_status fem_set_normalisation(fem_ctx *f, const float *in_mean, const float *in_std,
                                 const float *out_mean, const float *out_std);
// Structural-step counters: surrogate guesses accepted, rejected, Newton
// solves, structural steps (since coupling or the last reset).
constexpr int kFemStats = 4;
lbm_status fem_get_stats(fem_ctx *f, int *stats);
lbm_status fem_reset_stats(fem_ctx *f);
// Surrogate network input width for an nn-node beam: three out-of-balance
// load vectors, u and v, each on the 3 nn - 3 free DOFs.
constexpr int surrogate_inputs(int nn) { return 15 * nn - 15; }
lbm_status mlp_forward_device(mlp_ctx *x, int B, cudaStream_t s, float **yhat, float **xin);
float *mlp_input_buffer(mlp_ctx *x);
int mlp_dim(const mlp_ctx *x, int l);
int mlp_layers(const mlp_ctx *x);
void fem_describe(const fem_ctx *f, BeamParams *p, BeamDev *d);
cudaError_t launch_beam_batch(const BeamBatchDesc *d, int n, int any_fp64, cudaStream_t s);
cudaError_t launch_beam_coupled(fem_ctx *f, const double *vforce, double *surf_x, double *surf_v,
                                int v0, cudaStream_t s);
cudaError_t launch_flag_surface(fem_ctx *f, double *surf_x, double *surf_v, int v0,
                                cudaStream_t s);
int shell_nodes(const fem_shell_ctx *s);
cudaError_t launch_shell_surface(fem_shell_ctx *s, double *surf_x, double *surf_v, int v0,
                                 cudaStream_t st);
cudaError_t launch_shell_coupled(fem_shell_ctx *s, const double *vforce, double *surf_x,
                                 double *surf_v, int v0, cudaStream_t st);
int shell_free_dofs(const fem_shell_ctx *s);
lbm_status shell_set_surrogate(fem_shell_ctx *s, const float *in_mean, const float *in_std,
                               const float *out_mean, const float *out_std);
lbm_status shell_get_stats(fem_shell_ctx *s, int *stats, int reset);
cudaError_t launch_shell_coupled_guess(fem_shell_ctx *s, const double *vforce, double *surf_x,
                                       double *surf_v, int v0, double accept_tol, mlp_ctx *mlp,
                                       cudaStream_t st);

}  // namespace kbc
