// lbm_api.cu -- the C ABI (include/kbc_lbm.h): context, workspace layout,
// host/device argument staging and step orchestration.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <mutex>
#include <vector>

#include "../../include/kbc_lbm.h"
#include "lbm_internal.h"

using namespace kbc;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStageBytes = 16u << 20;  // host<->device staging chunk

constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

constexpr int kMaxBodies = 16;
#ifndef KBC_BATCH_CTAS
#define KBC_BATCH_CTAS 5
#endif

struct Layout {
  size_t f[2], flags, err, stage;
  size_t sx, sv, se, seb, links, bnodes, fresh, counters, vforce, bforce, inlet[6];
  size_t sigma, orient, tvforce, tbforce;  // stress-traction output
  size_t sbox;                             // bounding box of the surface (6 floats)
  size_t mp_rho[2], mp_pl;                 // multiphase fields (0: not reserved)
  size_t mp_ctl, mp_partial;               // momentum-controller state, CTA partials
  size_t mp_band;                          // wall-band scratch (walls in the multiphase model)
  int nface, bcap, inlet_n[6];
  size_t total;
};

int pop_bytes(int storage) {
  return storage == LBM_STORE_F64 ? 8 : (storage == LBM_STORE_F32 ? 4 : 2);
}

Grid make_grid(const lbm_config &c) {
  Grid g;
  g.nx = c.nx; g.ny = c.ny; g.nz = c.nz;
  g.px = (c.bc[0] == LBM_BC_PERIODIC) ? 0 : 1;
  g.py = (c.bc[2] == LBM_BC_PERIODIC) ? 0 : 1;
  g.pz = (c.lattice == LBM_D3Q27 && c.bc[4] != LBM_BC_PERIODIC) ? 1 : 0;
  g.NX = c.nx + 2 * g.px;
  g.NY = c.ny + 2 * g.py;
  g.NZ = c.nz + 2 * g.pz;
  g.pitch = (g.NX + 7) / 8 * 8;
  g.N = (long long)g.pitch * g.NY * g.NZ;
  return g;
}

Layout make_layout(const lbm_config &c) {
  Grid g = make_grid(c);
  Layout L;
  size_t off = 0;
  const size_t fb = align_up((size_t)c.lattice * (size_t)g.N * pop_bytes(c.storage));
  L.f[0] = off; off += fb;
  L.f[1] = off; off += fb;
  L.flags = off; off += align_up((size_t)g.N);
  L.err = off; off += kAlign;
  L.stage = off; off += kStageBytes;
  // immersed surface and boundary lists
  const int nv = c.max_vertices, ne = c.max_elements, nl = c.max_links;
  L.sx = off; off += align_up(sizeof(double) * 3 * (size_t)std::max(nv, 1));
  L.sv = off; off += align_up(sizeof(double) * 3 * (size_t)std::max(nv, 1));
  L.se = off; off += align_up(sizeof(int32_t) * 3 * (size_t)std::max(ne, 1));
  L.seb = off; off += align_up(sizeof(int32_t) * (size_t)std::max(ne, 1));
  L.links = off; off += align_up(sizeof(Link) * (size_t)std::max(nl, 1));
  long long nface = 0;
  const long long n[3] = {c.nx, c.ny, c.nz};
  const int pads[3] = {g.px, g.py, g.pz};
  for (int a = 0; a < 3; ++a)
    if (pads[a]) nface += 2 * (n[0] * n[1] * n[2] / n[a]);
  L.nface = (int)nface;
  L.bcap = L.nface + nl;
  L.bnodes = off; off += align_up(sizeof(BNode) * (size_t)std::max(L.bcap, 1));
  L.fresh = off; off += align_up(sizeof(int64_t) * (size_t)std::max(nl, 1));
  L.counters = off; off += kAlign;  // nbn, nl, nfresh, step, nface
  L.vforce = off; off += align_up(sizeof(double) * 3 * (size_t)std::max(nv, 1));
  L.bforce = off; off += align_up(sizeof(double) * 3 * kMaxBodies);
  L.sigma = off; off += align_up(sizeof(double) * 6 * (size_t)std::max(nl, 1));
  L.orient = off; off += align_up(sizeof(double) * kMaxBodies);
  L.tvforce = off; off += align_up(sizeof(double) * 3 * (size_t)std::max(nv, 1));
  L.tbforce = off; off += align_up(sizeof(double) * 3 * kMaxBodies);
  L.sbox = off; off += align_up(sizeof(float) * 8);
  L.mp_rho[0] = L.mp_rho[1] = L.mp_pl = L.mp_ctl = L.mp_partial = L.mp_band = 0;
  if (c.multiphase) {
    // two density buffers (the reference of the stored state, the density
    // of the step being computed) and (phi, lap rho) per stored node, in the
    // compute precision
    const size_t cb = c.storage == LBM_STORE_F64 ? 8 : 4;
    L.mp_rho[0] = off; off += align_up(cb * (size_t)g.N);
    L.mp_rho[1] = off; off += align_up(cb * (size_t)g.N);
    L.mp_pl = off; off += align_up(2 * cb * (size_t)g.N);
    L.mp_ctl = off; off += align_up(sizeof(double) * kMpControl);
    L.mp_partial = off;
    off += align_up(mp_partial_bytes(c.nx, c.ny, c.nz));
    L.mp_band = off;
    off += align_up(mp_band_bytes(c.nx, c.ny, c.nz, (int)cb));
  }
  for (int fc = 0; fc < 6; ++fc) {
    L.inlet_n[fc] = 0;
    L.inlet[fc] = 0;
    if (c.bc[fc] == LBM_BC_INLET) {
      const int a = fc / 2;
      L.inlet_n[fc] = (int)(n[0] * n[1] * n[2] / n[a]);
      L.inlet[fc] = off;
      off += align_up(sizeof(float) * 3 * (size_t)L.inlet_n[fc]);
    }
  }
  L.total = off;
  return L;
}

const char *validate(const lbm_config *c) {
  if (!c) return "config is NULL";
  if (c->lattice != LBM_D2Q9 && c->lattice != LBM_D3Q27) return "lattice must be 9 or 27";
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "lattice sizes must be >= 1";
  if (c->lattice == LBM_D2Q9 && c->nz != 1) return "D2Q9 needs nz == 1";
  if (c->ny > 65535 || c->nz > 65535) return "ny and nz must be <= 65535";
  if (!(c->beta > 0.0 && c->beta < 1.0)) return "beta must lie in (0, 1)";
  if (c->storage != LBM_STORE_F32 && c->storage != LBM_STORE_F16 && c->storage != LBM_STORE_BF16 &&
      c->storage != LBM_STORE_F16N && c->storage != LBM_STORE_F64)
    return "unknown storage";
  if (c->storage == LBM_STORE_F64 && c->lattice != LBM_D2Q9) return "FP64 storage is D2Q9 only";
  if (c->collision != LBM_COLLIDE_KBC && c->collision != LBM_COLLIDE_BGK)
    return "unknown collision";
  const int naxes = c->lattice == LBM_D2Q9 ? 2 : 3;
  for (int a = 0; a < 3; ++a) {
    const int lo = c->bc[2 * a], hi = c->bc[2 * a + 1];
    if (lo < LBM_BC_PERIODIC || lo > LBM_BC_FREESTREAM || hi < LBM_BC_PERIODIC ||
        hi > LBM_BC_FREESTREAM)
      return "unknown face boundary kind";
    if ((lo == LBM_BC_PERIODIC) != (hi == LBM_BC_PERIODIC))
      return "periodic faces must come in pairs";
    if (a >= naxes && (lo != LBM_BC_PERIODIC)) return "D2Q9 z faces must be periodic";
  }
  long long n = (long long)c->nx * c->ny * c->nz;
  if (n > (1LL << 31)) return "lattice too large";
  if (c->max_links < 0 || c->max_vertices < 0 || c->max_elements < 0) return "negative capacity";
  if (c->inlet_ramp_steps < 0) return "negative inlet ramp";
  if (c->multiphase != 0 && c->multiphase != 1) return "multiphase must be 0 or 1";
  if (c->multiphase && c->storage != LBM_STORE_F32 && c->storage != LBM_STORE_F64)
    return "the multiphase model needs FP32 or FP64 storage";
  const int nz_ax = c->lattice == LBM_D2Q9 ? 2 : 3;
  const int nn[3] = {c->nx, c->ny, c->nz};
  for (int a = 0; a < nz_ax; ++a)
    if (c->bc[2 * a] != LBM_BC_PERIODIC && nn[a] < 3) return "non-periodic axes need >= 3 nodes";
  return nullptr;
}

}  // namespace

struct lbm_ctx {
  lbm_config cfg;
  Grid g;
  Layout lay;
  int Q = 0;
  int device = 0;            // the CUDA device current at lbm_create (workspace, stream)
  char *ws = nullptr;
  bool own_ws = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  uint8_t *flags = nullptr;
  bool has_solid = false;
  int *err = nullptr;
  char *stage = nullptr;
  int sweep_variant = SWEEP_AUTO;
  // boundary state
  int nface = 0;             // face boundary nodes (fixed list head)
  int nbodies = 0, nv = 0, ne = 0;
  Band band{0, 0, 0, 0, 0, 0};
  int *counters = nullptr;   // [0] immersed nodes, [1] links, [2] fresh, [3] step
  BoundaryParams bp;
  fem_ctx *fem = nullptr;    // coupled beam (conventional serial staggered loop)
  int fem_v0 = 0;
  fem_shell_ctx *shell = nullptr;  // coupled plate (3-D)
  int shell_v0 = 0;
  mlp_ctx *mlp = nullptr;    // structural-step surrogate (Newton initial guess)
  bool traction_on = false;  // stress-traction output each step
  bool mp_on = false;        // multiphase step (lbm_set_multiphase)
  MpParams mp{};
  int mp_cur = 0;            // density buffer holding the reference of the stored state
  bool mp_have_force = false;  // a multiphase step has produced the stored state
  int graph_cur = 0, graph_mp_cur = 0;  // buffer parities the graph was captured at
  // two-level refinement: on a coarse lattice, its fine patch; on a fine
  // lattice, the coarse lattice that steps it
  lbm_ctx *ref_fine = nullptr, *ref_coarse = nullptr;
  int ref_i0 = 0, ref_j0 = 0;
  char *ref_ws = nullptr;
  bool ref_own_ws = false;
  double accept_tol = 0.0;
  // CUDA graph of graph_n steps (replayed by lbm_step_graph)
  cudaGraphExec_t gexec = nullptr;
  int graph_n = 0;
  bool graph_dirty = true;
  bool poisoned = false;
  char msg[512] = {0};
};

static lbm_status fail(lbm_ctx *c, lbm_status st, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
  }
  return st;
}

static lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where) {
  if (c) c->poisoned = true;
  return fail(c, LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (cudaHostAlloc / cudaHostRegister,
// e.g. torch's pin_memory()), which kernels read and write in place over the
// host link; nullptr for any other pointer.
static void *mapped_host_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static thread_local char g_create_msg[512];

extern "C" {

lbm_status lbm_workspace_size(const lbm_config *cfg, size_t *bytes) {
  if (!bytes) return LBM_EINVAL;
  if (validate(cfg)) return LBM_EINVAL;
  *bytes = make_layout(*cfg).total;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config *cfg, void *workspace, size_t workspace_bytes,
                      lbm_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (const char *why = validate(cfg)) {
    snprintf(g_create_msg, sizeof(g_create_msg), "lbm_create: %s", why);
    return LBM_EINVAL;
  }
  lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return LBM_ENOMEM;
  ctx->cfg = *cfg;
  ctx->Q = cfg->lattice;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    snprintf(g_create_msg, sizeof(g_create_msg), "lbm_create: no current CUDA device");
    delete ctx;
    return LBM_ECUDA;
  }
  ctx->g = make_grid(*cfg);
  ctx->lay = make_layout(*cfg);
  if (workspace) {
    if (workspace_bytes < ctx->lay.total || ((uintptr_t)workspace % kAlign) != 0) {
      snprintf(g_create_msg, sizeof(g_create_msg),
               "lbm_create: workspace needs %zu bytes, 256-byte aligned", ctx->lay.total);
      delete ctx;
      return LBM_ENOMEM;
    }
    ctx->ws = (char *)workspace;
  } else {
    cudaError_t e = cudaMalloc((void **)&ctx->ws, ctx->lay.total);
    if (e != cudaSuccess) {
      snprintf(g_create_msg, sizeof(g_create_msg), "lbm_create: cudaMalloc(%zu): %s",
               ctx->lay.total, cudaGetErrorString(e));
      delete ctx;
      return LBM_ENOMEM;
    }
    ctx->own_ws = true;
  }
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      if (ctx->own_ws) cudaFree(ctx->ws);
      delete ctx;
      return LBM_ECUDA;
    }
    ctx->own_stream = true;
  }
  ctx->f[0] = ctx->ws + ctx->lay.f[0];
  ctx->f[1] = ctx->ws + ctx->lay.f[1];
  ctx->flags = (uint8_t *)(ctx->ws + ctx->lay.flags);
  ctx->err = (int *)(ctx->ws + ctx->lay.err);
  ctx->stage = ctx->ws + ctx->lay.stage;
  // rest state f = W everywhere (zero deviation), all nodes fluid, ghosts solid
  CK(cudaMemsetAsync(ctx->f[0], 0, ctx->lay.f[1] - ctx->lay.f[0], ctx->stream));
  CK(cudaMemsetAsync(ctx->f[1], 0, ctx->lay.f[1] - ctx->lay.f[0], ctx->stream));
  CK(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->flags, NODE_FLUID, (size_t)ctx->g.N, ctx->stream));
  ctx->has_solid = false;
  ctx->counters = (int *)(ctx->ws + ctx->lay.counters);
  CK(cudaMemsetAsync(ctx->counters, 0, kAlign, ctx->stream));
  // boundary parameters
  for (int fc = 0; fc < 6; ++fc) {
    ctx->bp.bc[fc] = cfg->bc[fc];
    for (int a = 0; a < 3; ++a) ctx->bp.face_u[fc][a] = (float)cfg->face_velocity[fc][a];
    ctx->bp.inlet[fc] = nullptr;
  }
  ctx->bp.beta = cfg->beta;
  ctx->bp.ramp_steps = cfg->inlet_ramp_steps;
  ctx->bp.step = ctx->counters + 3;
  if (ctx->g.px || ctx->g.py || ctx->g.pz) {
    // ghost layer and the fixed list of face boundary nodes
    CK(launch_mark_ghosts(ctx->g, ctx->flags, ctx->stream));
    int *cnt = ctx->counters + 4;
    CK(launch_face_nodes(ctx->g, (BNode *)(ctx->ws + ctx->lay.bnodes), cnt, ctx->lay.nface,
                         ctx->stream));
    int h = 0;
    CK(cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->nface = std::min(h, ctx->lay.nface);
    ctx->has_solid = true;  // ghosts are skipped by the sweep
  }
  *out = ctx;
  return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->msg : g_create_msg; }

void *lbm_stream(const lbm_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

static void refine_release(lbm_ctx *coarse);

void lbm_destroy(lbm_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->ref_fine) refine_release(ctx);
  if (ctx->ref_coarse) refine_release(ctx->ref_coarse);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->own_ws) cudaFree(ctx->ws);
  delete ctx;
}

#define GUARD()                                                              \
  do {                                                                       \
    if (!ctx) return LBM_EINVAL;                                             \
    if (ctx->poisoned) return fail(ctx, LBM_ESTATE, "context poisoned: %s", ctx->msg); \
    if (!on_ctx_device(ctx))                                                 \
      return fail(ctx, LBM_EINVAL, "the current CUDA device is not the context's device %d", \
                  ctx->device);                                              \
  } while (0)

// The context's stream and workspace belong to the device that was current at
// lbm_create; every call expects that device to be current again.
static bool on_ctx_device(const lbm_ctx *ctx) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == ctx->device;
}

static lbm_status mp_adopt_state(lbm_ctx *ctx);
static const void *mp_ref(const lbm_ctx *ctx);
static const double *mp_mean_used(const lbm_ctx *ctx);

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u) {
  GUARD();
  if (!rho || !u) return fail(ctx, LBM_EINVAL, "lbm_init_equilibrium: NULL argument");
  if (lbm_status st = mp_adopt_state(ctx); st != LBM_OK) return st;
  const int dim = ctx->Q == 9 ? 2 : 3;
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  const bool dev = is_device_ptr(rho) && is_device_ptr(u);
  if (dev) {
    CK(launch_init_eq(ctx->Q, ctx->cfg.storage, ctx->g, rho, u, n, 0, n, ctx->f[ctx->cur],
                      ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the caller may reuse the arrays on return
    return LBM_OK;
  }
  const double *mr = (const double *)mapped_host_ptr(rho), *mu = (const double *)mapped_host_ptr(u);
  if (mr && mu) {
    // page-locked host arrays: the kernel reads them in place
    CK(launch_init_eq(ctx->Q, ctx->cfg.storage, ctx->g, mr, mu, n, 0, n, ctx->f[ctx->cur],
                      ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host arrays may be released on return
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / (sizeof(double) * (1 + dim)));
  double *s = (double *)ctx->stage;
  for (long long b = 0; b < n; b += chunk) {
    const long long cnt = (n - b < chunk) ? n - b : chunk;
    CK(cudaMemcpyAsync(s, rho + b, cnt * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    for (int a = 0; a < dim; ++a)
      CK(cudaMemcpyAsync(s + (1 + a) * cnt, u + a * n + b, cnt * sizeof(double),
                         cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_init_eq(ctx->Q, ctx->cfg.storage, ctx->g, s, s + cnt, cnt, b, cnt,
                      ctx->f[ctx->cur], ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));  // the host arrays may be released on return
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f) {
  GUARD();
  if (!f) return fail(ctx, LBM_EINVAL, "lbm_set_populations: NULL argument");
  if (lbm_status st = mp_adopt_state(ctx); st != LBM_OK) return st;
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  if (is_device_ptr(f)) {
    for (int i = 0; i < ctx->Q; ++i)
      CK(launch_set_pop(ctx->Q, ctx->cfg.storage, ctx->g, i, f + i * n, 0, n, ctx->f[ctx->cur],
                        ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the caller may reuse the array on return
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / sizeof(double));
  double *s = (double *)ctx->stage;
  for (int i = 0; i < ctx->Q; ++i)
    for (long long b = 0; b < n; b += chunk) {
      const long long cnt = (n - b < chunk) ? n - b : chunk;
      CK(cudaMemcpyAsync(s, f + i * n + b, cnt * sizeof(double), cudaMemcpyHostToDevice,
                         ctx->stream));
      CK(launch_set_pop(ctx->Q, ctx->cfg.storage, ctx->g, i, s, b, cnt, ctx->f[ctx->cur],
                        ctx->stream));
    }
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *ctx, double *f) {
  GUARD();
  if (!f) return fail(ctx, LBM_EINVAL, "lbm_get_populations: NULL argument");
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  if (ctx->mp_on) {
    // populations stored relative to the local reference density
    const void *mpl = ctx->ws + ctx->lay.mp_pl;
    if (is_device_ptr(f)) {
      CK(launch_mp_read(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], mp_ref(ctx), mpl,
                        ctx->mp, 0, mp_mean_used(ctx), 0, n, n, nullptr, nullptr, nullptr,
                        nullptr, nullptr, f, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      return LBM_OK;
    }
    const long long chunk = (long long)(kStageBytes / (sizeof(double) * ctx->Q));
    double *s = (double *)ctx->stage;
    for (long long b = 0; b < n; b += chunk) {
      const long long cnt = (n - b < chunk) ? n - b : chunk;
      CK(launch_mp_read(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], mp_ref(ctx), mpl,
                        ctx->mp, 0, mp_mean_used(ctx), b, cnt, cnt, nullptr, nullptr, nullptr,
                        nullptr, nullptr, s, ctx->stream));
      for (int i = 0; i < ctx->Q; ++i)
        CK(cudaMemcpyAsync(f + i * n + b, s + i * cnt, cnt * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    return LBM_OK;
  }
  if (is_device_ptr(f)) {
    for (int i = 0; i < ctx->Q; ++i)
      CK(launch_get_pop(ctx->Q, ctx->cfg.storage, ctx->g, i, f + i * n, 0, n, ctx->f[ctx->cur],
                        ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / sizeof(double));
  double *s = (double *)ctx->stage;
  for (int i = 0; i < ctx->Q; ++i)
    for (long long b = 0; b < n; b += chunk) {
      const long long cnt = (n - b < chunk) ? n - b : chunk;
      CK(launch_get_pop(ctx->Q, ctx->cfg.storage, ctx->g, i, s, b, cnt, ctx->f[ctx->cur],
                        ctx->stream));
      CK(cudaMemcpyAsync(f + i * n + b, s, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
  return LBM_OK;
}

static lbm_status run_geometry(lbm_ctx *ctx, int track_fresh);
static SurfaceDev surface_dev(lbm_ctx *ctx);

// A state written from outside (single-phase convention, f_i - W_i) becomes
// the stored state of the multiphase step: reference 1 everywhere, no force
// yet applied.
static lbm_status mp_adopt_state(lbm_ctx *ctx) {
  if (!ctx->mp_on) return LBM_OK;
  CK(launch_mp_rebase(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur],
                      ctx->ws + ctx->lay.mp_rho[ctx->mp_cur], 1.0, 0, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.mp_ctl, 0, sizeof(double) * kMpControl, ctx->stream));
  // lap R = 0 for the uniform reference R = 1 (the density pass reads it)
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.mp_pl, 0, ctx->lay.mp_ctl - ctx->lay.mp_pl, ctx->stream));
  CK(cudaMemsetAsync(ctx->ws + ctx->lay.mp_partial, 0,
                     mp_partial_bytes(ctx->g.nx, ctx->g.ny, ctx->g.nz), ctx->stream));
  ctx->mp_have_force = false;
  return LBM_OK;
}

static const void *mp_ref(const lbm_ctx *ctx) { return ctx->ws + ctx->lay.mp_rho[ctx->mp_cur]; }
static double *mp_ctl(const lbm_ctx *ctx) { return (double *)(ctx->ws + ctx->lay.mp_ctl); }
// the controller state, which holds the correction the last step used
static const double *mp_mean_used(const lbm_ctx *ctx) { return mp_ctl(ctx); }

lbm_status lbm_set_multiphase(lbm_ctx *ctx, const lbm_multiphase_params *params) {
  GUARD();
  if (!params) {
    if (ctx->mp_on)  // back to the single-phase convention f_i - W_i
      CK(launch_mp_rebase(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur],
                          ctx->ws + ctx->lay.mp_rho[ctx->mp_cur], 1.0, 1, ctx->stream));
    ctx->mp_on = false;
    ctx->graph_dirty = true;
    return LBM_OK;
  }
  if (!ctx->cfg.multiphase)
    return fail(ctx, LBM_ESTATE, "lbm_set_multiphase: context created without multiphase = 1");
  // fully periodic, or two walls at rest on the faces of one axis
  int wall = -1;
  const int naxes = ctx->Q == 9 ? 2 : 3;
  for (int a = 0; a < naxes; ++a) {
    const int lo = ctx->cfg.bc[2 * a], hi = ctx->cfg.bc[2 * a + 1];
    if (lo == LBM_BC_PERIODIC && hi == LBM_BC_PERIODIC) continue;
    if (lo != LBM_BC_WALL || hi != LBM_BC_WALL || wall >= 0)
      return fail(ctx, LBM_EINVAL,
                  "lbm_set_multiphase: faces must be periodic, or walls on both faces of one axis");
    for (int fc = 2 * a; fc < 2 * a + 2; ++fc)
      for (int b = 0; b < 3; ++b)
        if (ctx->cfg.face_velocity[fc][b] != 0.0)
          return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: the walls must be at rest");
    wall = a;
  }
  if (!std::isfinite(params->kappa_w))
    return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: non-finite kappa_w");
  if (ctx->nbodies > 0 || ctx->fem || ctx->shell)
    return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: immersed bodies are not supported");
  if (ctx->cfg.storage != LBM_STORE_F32 && ctx->cfg.storage != LBM_STORE_F64)
    return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: FP32 or FP64 storage only");
  if (!(params->kappa >= 0.0) || !std::isfinite(params->kappa))
    return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: kappa must be finite and >= 0");
  if (params->eos != LBM_EOS_PAPER && params->eos != LBM_EOS_IDEAL)
    return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: unknown eos %d", params->eos);
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(params->g[a]))
      return fail(ctx, LBM_EINVAL, "lbm_set_multiphase: non-finite acceleration");
  ctx->mp.kappa = params->kappa;
  ctx->mp.kappa_w = wall >= 0 ? params->kappa_w : 0.0;
  ctx->mp.wall = wall;
  ctx->mp.eos = params->eos == LBM_EOS_IDEAL ? MP_EOS_IDEAL : MP_EOS_PAPER;
  for (int a = 0; a < 3; ++a) ctx->mp.g[a] = (a < 2 || ctx->Q == 27) ? params->g[a] : 0.0;
  if (!ctx->mp_on) {
    ctx->mp_on = true;
    lbm_status st = mp_adopt_state(ctx);
    if (st != LBM_OK) return st;
  }
  ctx->graph_dirty = true;
  return LBM_OK;
}

lbm_status lbm_get_force_field(lbm_ctx *ctx, double *F) {
  GUARD();
  if (!F) return fail(ctx, LBM_EINVAL, "lbm_get_force_field: NULL argument");
  if (!ctx->mp_on) return fail(ctx, LBM_ESTATE, "lbm_get_force_field: the multiphase model is off");
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  const void *mpl = ctx->ws + ctx->lay.mp_pl;
  const int hf = ctx->mp_have_force;
  double *mf = is_device_ptr(F) ? F : (double *)mapped_host_ptr(F);
  if (mf) {
    CK(launch_mp_read(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], mp_ref(ctx), mpl, ctx->mp,
                      hf, mp_mean_used(ctx), 0, n, n, mf, nullptr, nullptr, nullptr, nullptr,
                      nullptr, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / (sizeof(double) * 3));
  double *s = (double *)ctx->stage;
  for (long long b = 0; b < n; b += chunk) {
    const long long cnt = (n - b < chunk) ? n - b : chunk;
    CK(launch_mp_read(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], mp_ref(ctx), mpl, ctx->mp,
                      hf, mp_mean_used(ctx), b, cnt, cnt, s, nullptr, nullptr, nullptr, nullptr,
                      nullptr, ctx->stream));
    for (int a = 0; a < 3; ++a)
      CK(cudaMemcpyAsync(F + a * n + b, s + a * cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                         ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

static lbm_status refine_steps(lbm_ctx *ctx, int n);

lbm_status lbm_step(lbm_ctx *ctx, int n) {
  GUARD();
  if (n < 0) return fail(ctx, LBM_EINVAL, "lbm_step: n < 0");
  if (ctx->ref_coarse)
    return fail(ctx, LBM_ESTATE, "lbm_step: a fine patch is stepped by its coarse lattice");
  if (ctx->ref_fine) return refine_steps(ctx, n);
  const double beta = ctx->cfg.beta;
  const int bgk = ctx->cfg.collision == LBM_COLLIDE_BGK;
  // the multiphase step fills its wall nodes itself
  const bool bnd = (ctx->nface > 0 || ctx->nbodies > 0) && !ctx->mp_on;
  const int cap = ctx->nface + (ctx->nbodies > 0 ? ctx->cfg.max_links : 0);
  for (int t = 0; t < n; ++t) {
    if (bnd) {
      if (ctx->nbodies > 0) {
        CK(cudaMemsetAsync(ctx->ws + ctx->lay.vforce, 0, sizeof(double) * 3 * (size_t)ctx->nv,
                           ctx->stream));
        CK(cudaMemsetAsync(ctx->ws + ctx->lay.bforce, 0, sizeof(double) * 3 * kMaxBodies,
                           ctx->stream));
      }
      CK(launch_grad(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], ctx->flags,
                     (const BNode *)(ctx->ws + ctx->lay.bnodes),
                     ctx->nbodies > 0 ? ctx->counters : nullptr, ctx->nface, cap,
                     (const Link *)(ctx->ws + ctx->lay.links), ctx->bp,
                     (double *)(ctx->ws + ctx->lay.vforce), (double *)(ctx->ws + ctx->lay.bforce),
                     ctx->nbodies, ctx->stream));
      if (ctx->bp.ramp_steps > 0) CK(launch_step_counter(ctx->counters + 3, ctx->stream));
    }
    if (ctx->mp_on) {
      // the one-node forced sweep is the faster form (AUTO); PAIR asks for the other
      ctx->mp.pair = ctx->sweep_variant == SWEEP_PAIR;
      CK(launch_mp_step(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], ctx->f[1 - ctx->cur],
                        ctx->ws + ctx->lay.mp_rho[ctx->mp_cur],
                        ctx->ws + ctx->lay.mp_rho[1 - ctx->mp_cur], ctx->ws + ctx->lay.mp_pl,
                        mp_ctl(ctx), (double *)(ctx->ws + ctx->lay.mp_partial),
                        ctx->ws + ctx->lay.mp_band, ctx->mp_have_force ? 1 : 0, ctx->mp, beta,
                        bgk, ctx->err, ctx->stream));
      ctx->mp_cur = 1 - ctx->mp_cur;
      ctx->mp_have_force = true;
    } else
      CK(launch_sweep(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], ctx->f[1 - ctx->cur],
                      ctx->has_solid ? ctx->flags : nullptr, beta, bgk, ctx->err, ctx->stream,
                      ctx->sweep_variant));
    if (ctx->traction_on && ctx->nbodies > 0)
      CK(launch_traction(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur],
                         (const BNode *)(ctx->ws + ctx->lay.bnodes) + ctx->nface, ctx->counters,
                         ctx->cfg.max_links, ctx->cfg.beta, surface_dev(ctx),
                         (double *)(ctx->ws + ctx->lay.sigma), (double *)(ctx->ws + ctx->lay.orient),
                         (double *)(ctx->ws + ctx->lay.tvforce),
                         (double *)(ctx->ws + ctx->lay.tbforce), ctx->nbodies, ctx->stream));
    ctx->cur = 1 - ctx->cur;
    if (ctx->fem && ctx->mlp) {
      // surrogate: network guess of the increment, accepted by the FEM
      // residual or refined by Newton from there
      const double *vf = (const double *)(ctx->ws + ctx->lay.vforce);
      CK(launch_surrogate_input(ctx->fem, vf, ctx->fem_v0, mlp_input_buffer(ctx->mlp), ctx->stream));
      float *yhat = nullptr, *xin = nullptr;
      lbm_status st = mlp_forward_device(ctx->mlp, 1, ctx->stream, &yhat, &xin);
      if (st != LBM_OK) return fail(ctx, st, "surrogate forward failed");
      CK(launch_surrogate_guess(ctx->fem, yhat, ctx->stream));
      CK(launch_beam_coupled_guess(ctx->fem, vf, (double *)(ctx->ws + ctx->lay.sx),
                                   (double *)(ctx->ws + ctx->lay.sv), ctx->fem_v0, ctx->accept_tol,
                                   ctx->stream));
      st = run_geometry(ctx, 1);
      if (st != LBM_OK) return st;
    } else if (ctx->shell && ctx->mlp) {
      CK(launch_shell_coupled_guess(ctx->shell, (const double *)(ctx->ws + ctx->lay.vforce),
                                    (double *)(ctx->ws + ctx->lay.sx),
                                    (double *)(ctx->ws + ctx->lay.sv), ctx->shell_v0,
                                    ctx->accept_tol, ctx->mlp, ctx->stream));
      lbm_status st = run_geometry(ctx, 1);
      if (st != LBM_OK) return st;
    } else if (ctx->shell) {
      CK(launch_shell_coupled(ctx->shell, (const double *)(ctx->ws + ctx->lay.vforce),
                              (double *)(ctx->ws + ctx->lay.sx), (double *)(ctx->ws + ctx->lay.sv),
                              ctx->shell_v0, ctx->stream));
      lbm_status st = run_geometry(ctx, 1);
      if (st != LBM_OK) return st;
    } else if (ctx->fem) {
      // structural step from this step's forces, transfer to the surface, new geometry
      CK(launch_beam_coupled(ctx->fem, (const double *)(ctx->ws + ctx->lay.vforce),
                             (double *)(ctx->ws + ctx->lay.sx), (double *)(ctx->ws + ctx->lay.sv),
                             ctx->fem_v0, ctx->stream));
      lbm_status st = run_geometry(ctx, 1);
      if (st != LBM_OK) return st;
    }
  }
  return LBM_OK;
}

// ---- two-level refinement
static RefLaunch refine_launch(const lbm_ctx *ctx);

static void refine_release(lbm_ctx *coarse) {
  lbm_ctx *fine = coarse->ref_fine;
  if (coarse->ref_own_ws && coarse->ref_ws) {
    cudaStreamSynchronize(coarse->stream);
    cudaFree(coarse->ref_ws);
  }
  coarse->ref_ws = nullptr;
  coarse->ref_own_ws = false;
  coarse->ref_fine = nullptr;
  coarse->graph_dirty = true;
  if (fine) fine->ref_coarse = nullptr;
}

static bool refine_busy(const lbm_ctx *c) {
  // (has_solid is also set by a ghost layer alone; solid interior nodes come with bodies)
  return c->nbodies > 0 || c->fem || c->shell || c->mlp || c->mp_on;
}

static const char *refine_mismatch(const lbm_ctx *c, const lbm_ctx *f) {
  if (c->Q != 9 || f->Q != 9) return "both lattices must be D2Q9";
  if (c->cfg.storage != f->cfg.storage) return "the two lattices need the same storage";
  if (c->cfg.storage != LBM_STORE_F32 && c->cfg.storage != LBM_STORE_F64)
    return "refinement needs FP32 or FP64 storage";
  if (c->cfg.collision != f->cfg.collision) return "the two lattices need the same collision";
  if (c->stream != f->stream) return "the two lattices must share one stream";
  if (c->device != f->device) return "the two lattices must be on one device";
  for (int k = 0; k < 4; ++k)
    if (c->cfg.bc[k] != LBM_BC_PERIODIC) return "the coarse lattice must be periodic";
  for (int k = 0; k < 4; ++k)
    if (f->cfg.bc[k] == LBM_BC_PERIODIC) return "the fine lattice needs non-periodic x and y faces";
  if (f->cfg.nx < 4 || f->cfg.ny < 4 || (f->cfg.nx & 1) || (f->cfg.ny & 1))
    return "the fine sizes must be even and >= 4";
  const double bf = 1.0 / (2.0 / c->cfg.beta - 1.0);
  if (!(std::fabs(f->cfg.beta - bf) <= 1e-12 * bf))
    return "fine beta must be 1 / (2 / beta_c - 1) (nu_f = 2 nu_c)";
  return nullptr;
}

lbm_status lbm_refine_workspace_size(lbm_ctx *coarse, lbm_ctx *fine, size_t *bytes) {
  lbm_ctx *ctx = coarse;
  GUARD();
  if (!fine || !bytes) return fail(ctx, LBM_EINVAL, "lbm_refine_workspace_size: NULL argument");
  if (const char *why = refine_mismatch(coarse, fine))
    return fail(ctx, LBM_EINVAL, "lbm_refine_workspace_size: %s", why);
  *bytes = align_up(refine_workspace_bytes(coarse->cfg.storage, coarse->g, fine->cfg.nx,
                                           fine->cfg.ny));
  return LBM_OK;
}

lbm_status lbm_refine_couple(lbm_ctx *coarse, lbm_ctx *fine, int i0, int j0, void *workspace,
                             size_t workspace_bytes) {
  lbm_ctx *ctx = coarse;
  GUARD();
  if (!fine) {
    refine_release(coarse);
    return LBM_OK;
  }
  if (fine == coarse) return fail(ctx, LBM_EINVAL, "lbm_refine_couple: fine == coarse");
  if (fine->poisoned) return fail(ctx, LBM_ESTATE, "lbm_refine_couple: fine context poisoned");
  if (coarse->ref_fine || coarse->ref_coarse || fine->ref_fine || fine->ref_coarse)
    return fail(ctx, LBM_ESTATE, "lbm_refine_couple: a context is already part of a pair");
  if (refine_busy(coarse) || refine_busy(fine))
    return fail(ctx, LBM_ESTATE,
                "lbm_refine_couple: bodies, beams, shells or the multiphase model are set");
  if (const char *why = refine_mismatch(coarse, fine))
    return fail(ctx, LBM_EINVAL, "lbm_refine_couple: %s", why);
  if (i0 < 0 || j0 < 0 || i0 + fine->cfg.nx / 2 > coarse->cfg.nx ||
      j0 + fine->cfg.ny / 2 > coarse->cfg.ny)
    return fail(ctx, LBM_EINVAL, "lbm_refine_couple: the patch leaves the coarse grid");
  if (fine->cfg.nx / 2 > coarse->cfg.nx - 2 || fine->cfg.ny / 2 > coarse->cfg.ny - 2)
    return fail(ctx, LBM_EINVAL, "lbm_refine_couple: the patch must leave two coarse cells free");
  const size_t need = align_up(refine_workspace_bytes(coarse->cfg.storage, coarse->g,
                                                      fine->cfg.nx, fine->cfg.ny));
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
      return fail(ctx, LBM_ENOMEM, "lbm_refine_couple: workspace needs %zu bytes, 256-byte aligned",
                  need);
    if (!is_device_ptr(workspace))
      return fail(ctx, LBM_EINVAL, "lbm_refine_couple: workspace must be device memory");
    coarse->ref_ws = (char *)workspace;
    coarse->ref_own_ws = false;
  } else {
    cudaError_t e = cudaMalloc((void **)&coarse->ref_ws, need);
    if (e != cudaSuccess) {
      coarse->ref_ws = nullptr;
      return fail(ctx, LBM_ENOMEM, "lbm_refine_couple: cudaMalloc(%zu): %s", need,
                  cudaGetErrorString(e));
    }
    coarse->ref_own_ws = true;
  }
  coarse->ref_fine = fine;
  coarse->ref_i0 = i0;
  coarse->ref_j0 = j0;
  fine->ref_coarse = coarse;
  coarse->graph_dirty = true;
  const cudaError_t e = launch_refine_init(refine_launch(coarse), coarse->stream);
  if (e != cudaSuccess) {
    refine_release(coarse);
    return cuda_fail(ctx, e, "launch_refine_init");
  }
  return LBM_OK;
}

static lbm_status refine_steps(lbm_ctx *ctx, int n) {
  lbm_ctx *fine = ctx->ref_fine;
  if (refine_busy(ctx) || refine_busy(fine))
    return fail(ctx, LBM_ESTATE, "lbm_step: the refined pair gained bodies or a model it lacks");
  RefLaunch R = refine_launch(ctx);
  for (int t = 0; t < n; ++t) {
    R.fc_in = ctx->f[ctx->cur];
    R.fc_out = ctx->f[1 - ctx->cur];
    CK(launch_refine_step(R, ctx->stream));
    ctx->cur = 1 - ctx->cur;  // two fine steps leave the fine state in its own buffer
  }
  return LBM_OK;
}

// Launch description of a coupled pair (coarse buffers set per step).
static RefLaunch refine_launch(const lbm_ctx *ctx) {
  const lbm_ctx *fine = ctx->ref_fine;
  RefLaunch R;
  R.gc = ctx->g;
  R.gf = fine->g;
  R.storage = ctx->cfg.storage;
  R.ff[0] = fine->f[0];
  R.ff[1] = fine->f[1];
  R.cur_f = fine->cur;
  R.flags_f = nullptr;
  R.beta_c = ctx->cfg.beta;
  R.beta_f = fine->cfg.beta;
  R.bgk = ctx->cfg.collision == LBM_COLLIDE_BGK;
  R.variant = ctx->sweep_variant;
  R.i0 = ctx->ref_i0;
  R.j0 = ctx->ref_j0;
  R.fields = ctx->ref_ws;
  R.err_c = R.err_f = ctx->err;
  R.fc_in = R.fc_out = nullptr;
  return R;
}

static lbm_status copy_in(lbm_ctx *ctx, void *dst, const void *src, size_t bytes) {
  // cudaMemcpyDefault infers host or device from the unified address space
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
  return LBM_OK;
}

static SurfaceDev surface_dev(lbm_ctx *ctx) {
  SurfaceDev s;
  s.dim = ctx->Q == 9 ? 2 : 3;
  s.nv = ctx->nv;
  s.ne = ctx->ne;
  s.nb = ctx->nbodies;
  s.x = (const double *)(ctx->ws + ctx->lay.sx);
  s.v = (const double *)(ctx->ws + ctx->lay.sv);
  s.e = (const int32_t *)(ctx->ws + ctx->lay.se);
  s.eb = (const int32_t *)(ctx->ws + ctx->lay.seb);
  s.box = (float *)(ctx->ws + ctx->lay.sbox);
  return s;
}

static lbm_status run_geometry(lbm_ctx *ctx, int track_fresh) {
  CK(launch_geometry(ctx->Q, ctx->cfg.storage, ctx->g, ctx->band, surface_dev(ctx), ctx->flags,
                     ctx->f[ctx->cur], (int64_t *)(ctx->ws + ctx->lay.fresh), ctx->counters + 2,
                     ctx->cfg.max_links, track_fresh,
                     (BNode *)(ctx->ws + ctx->lay.bnodes) + ctx->nface, ctx->counters,
                     ctx->cfg.max_links, (Link *)(ctx->ws + ctx->lay.links), ctx->counters + 1,
                     ctx->cfg.max_links, ctx->err, ctx->stream));
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx *ctx, int nbodies, const double *verts, int nv,
                            const int32_t *elems, int ne, const int32_t *elem_body,
                            const double *vert_vel, double band_margin) {
  GUARD();
  if (ctx->mp_on)
    return fail(ctx, LBM_EINVAL, "lbm_set_geometry: the multiphase model runs on periodic lattices without bodies");
  const int dim = ctx->Q == 9 ? 2 : 3;
  if (nbodies < 1 || nbodies > kMaxBodies || nv < dim || ne < 1 || !verts || !elems ||
      !elem_body || !(band_margin >= 0.0))
    return fail(ctx, LBM_EINVAL, "lbm_set_geometry: bad arguments");
  if (nv > ctx->cfg.max_vertices || ne > ctx->cfg.max_elements)
    return fail(ctx, LBM_ECAPACITY, "lbm_set_geometry: %d vertices / %d elements exceed capacity",
                nv, ne);
  // host copies for validation and the band
  std::vector<double> hx((size_t)nv * dim);
  std::vector<int32_t> he((size_t)ne * dim), hb((size_t)ne);
  CK(cudaMemcpy(hx.data(), verts, hx.size() * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(he.data(), elems, he.size() * sizeof(int32_t), cudaMemcpyDefault));
  CK(cudaMemcpy(hb.data(), elem_body, hb.size() * sizeof(int32_t), cudaMemcpyDefault));
  for (int32_t v : he)
    if (v < 0 || v >= nv) return fail(ctx, LBM_EINVAL, "lbm_set_geometry: element vertex id out of range");
  for (int32_t b : hb)
    if (b < 0 || b >= nbodies) return fail(ctx, LBM_EINVAL, "lbm_set_geometry: body id out of range");
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < nv; ++v)
    for (int a = 0; a < dim; ++a) {
      const double x = hx[(size_t)v * dim + a];
      if (!std::isfinite(x)) return fail(ctx, LBM_EINVAL, "lbm_set_geometry: non-finite vertex");
      lo[a] = std::min(lo[a], x);
      hi[a] = std::max(hi[a], x);
    }
  const int n[3] = {ctx->g.nx, ctx->g.ny, ctx->g.nz};
  const int pads[3] = {ctx->g.px, ctx->g.py, ctx->g.pz};
  int b0[3] = {0, 0, 0}, b1[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    b0[a] = (int)std::floor(lo[a] - band_margin) - 2;
    b1[a] = (int)std::ceil(hi[a] + band_margin) + 3;
    if (pads[a] && (b0[a] < 2 || b1[a] > n[a] - 2))
      return fail(ctx, LBM_EINVAL,
                  "lbm_set_geometry: bodies (plus margin) must stay 2 nodes inside non-periodic faces");
    b0[a] = std::max(b0[a], 0);
    b1[a] = std::min(b1[a], n[a]);
  }
  if (dim == 2) { b0[2] = 0; b1[2] = 1; }
  ctx->band = Band{b0[0], b1[0], b0[1], b1[1], b0[2], b1[2]};
  ctx->graph_dirty = true;
  ctx->nbodies = nbodies;
  ctx->nv = nv;
  ctx->ne = ne;
  lbm_status st;
  if ((st = copy_in(ctx, ctx->ws + ctx->lay.sx, verts, sizeof(double) * dim * nv)) != LBM_OK) return st;
  if (vert_vel) {
    if ((st = copy_in(ctx, ctx->ws + ctx->lay.sv, vert_vel, sizeof(double) * dim * nv)) != LBM_OK) return st;
  } else {
    CK(cudaMemsetAsync(ctx->ws + ctx->lay.sv, 0, sizeof(double) * dim * nv, ctx->stream));
  }
  if ((st = copy_in(ctx, ctx->ws + ctx->lay.se, elems, sizeof(int32_t) * dim * ne)) != LBM_OK) return st;
  if ((st = copy_in(ctx, ctx->ws + ctx->lay.seb, elem_body, sizeof(int32_t) * ne)) != LBM_OK) return st;
  // every previously solid node of the band is reset to fluid, then re-marked
  if ((st = run_geometry(ctx, 0)) != LBM_OK) return st;
  ctx->has_solid = true;
  int h[3];
  CK(cudaMemcpyAsync(h, ctx->counters, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h[0] > ctx->cfg.max_links || h[1] > ctx->cfg.max_links)
    return fail(ctx, LBM_ECAPACITY, "lbm_set_geometry: %d boundary nodes / %d links exceed max_links %d",
                h[0], h[1], ctx->cfg.max_links);
  return LBM_OK;
}

lbm_status lbm_update_surface(lbm_ctx *ctx, const double *verts, const double *vert_vel) {
  GUARD();
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "lbm_update_surface: no geometry set");
  if (!verts) return fail(ctx, LBM_EINVAL, "lbm_update_surface: NULL vertices");
  const int dim = ctx->Q == 9 ? 2 : 3;
  lbm_status st;
  if ((st = copy_in(ctx, ctx->ws + ctx->lay.sx, verts, sizeof(double) * dim * ctx->nv)) != LBM_OK) return st;
  if (vert_vel &&
      (st = copy_in(ctx, ctx->ws + ctx->lay.sv, vert_vel, sizeof(double) * dim * ctx->nv)) != LBM_OK)
    return st;
  return run_geometry(ctx, 1);
}

lbm_status lbm_get_interface_force(lbm_ctx *ctx, double *vert_force, double *body_force) {
  GUARD();
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "lbm_get_interface_force: no geometry set");
  if (vert_force)
    CK(cudaMemcpyAsync(vert_force, ctx->ws + ctx->lay.vforce, sizeof(double) * 3 * ctx->nv,
                       cudaMemcpyDefault, ctx->stream));
  if (body_force)
    CK(cudaMemcpyAsync(body_force, ctx->ws + ctx->lay.bforce, sizeof(double) * 3 * ctx->nbodies,
                       cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_set_traction_output(lbm_ctx *ctx, int enable) {
  GUARD();
  ctx->traction_on = enable != 0;
  ctx->graph_dirty = true;
  if (ctx->traction_on) {
    CK(cudaMemsetAsync(ctx->ws + ctx->lay.tvforce, 0, sizeof(double) * 3 * (size_t)std::max(ctx->nv, 1),
                       ctx->stream));
    CK(cudaMemsetAsync(ctx->ws + ctx->lay.tbforce, 0, sizeof(double) * 3 * kMaxBodies, ctx->stream));
  }
  return LBM_OK;
}

lbm_status lbm_get_traction_force(lbm_ctx *ctx, double *vert_force, double *body_force) {
  GUARD();
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "lbm_get_traction_force: no geometry set");
  if (!ctx->traction_on)
    return fail(ctx, LBM_ESTATE, "lbm_get_traction_force: enable it with lbm_set_traction_output");
  if (vert_force)
    CK(cudaMemcpyAsync(vert_force, ctx->ws + ctx->lay.tvforce, sizeof(double) * 3 * ctx->nv,
                       cudaMemcpyDefault, ctx->stream));
  if (body_force)
    CK(cudaMemcpyAsync(body_force, ctx->ws + ctx->lay.tbforce, sizeof(double) * 3 * ctx->nbodies,
                       cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_set_inlet_profile(lbm_ctx *ctx, int face, const double *u) {
  GUARD();
  if (face < 0 || face > 5 || ctx->cfg.bc[face] != LBM_BC_INLET || !u)
    return fail(ctx, LBM_EINVAL, "lbm_set_inlet_profile: face %d is not an inlet", face);
  const size_t n = (size_t)ctx->lay.inlet_n[face];
  std::vector<double> h(3 * n);
  CK(cudaMemcpy(h.data(), u, sizeof(double) * 3 * n, cudaMemcpyDefault));
  std::vector<float> hf(3 * n);
  for (size_t k = 0; k < 3 * n; ++k) hf[k] = (float)h[k];
  float *dst = (float *)(ctx->ws + ctx->lay.inlet[face]);
  CK(cudaMemcpyAsync(dst, hf.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->bp.inlet[face] = dst;
  ctx->graph_dirty = true;
  return LBM_OK;
}

lbm_status fsi_couple(lbm_ctx *ctx, fem_ctx *f, int first_vertex) {
  GUARD();
  ctx->mlp = nullptr;
  if (!f) {
    ctx->fem = nullptr;
    ctx->graph_dirty = true;
    return LBM_OK;
  }
  if (ctx->Q != 9) return fail(ctx, LBM_EINVAL, "fsi_couple: the beam couples to D2Q9 lattices");
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "fsi_couple: set the geometry first");
  const int nn = fem_nodes(f);
  if (first_vertex < 0 || first_vertex + 2 * nn > ctx->nv)
    return fail(ctx, LBM_EINVAL, "fsi_couple: vertices [%d, %d) outside the surface (%d)",
                first_vertex, first_vertex + 2 * nn, ctx->nv);
  ctx->fem = f;
  ctx->fem_v0 = first_vertex;
  ctx->graph_dirty = true;
  fem_set_span(f, 0, 0, 0.0, 0.0, 1.0);
  if (fem_reset_stats(f) != LBM_OK) return fail(ctx, LBM_ECUDA, "fsi_couple: counter reset failed");
  CK(launch_flag_surface(f, (double *)(ctx->ws + ctx->lay.sx), (double *)(ctx->ws + ctx->lay.sv),
                         first_vertex, ctx->stream));
  return run_geometry(ctx, 1);
}

lbm_status fsi_couple_span(lbm_ctx *ctx, fem_ctx *f, int first_vertex_z0, int first_vertex_z1,
                           double z0, double z1) {
  GUARD();
  ctx->mlp = nullptr;
  if (!f) return fail(ctx, LBM_EINVAL, "fsi_couple_span: no beam");
  if (ctx->Q != 27) return fail(ctx, LBM_EINVAL, "fsi_couple_span: the spanwise coupling is D3Q27");
  if (ctx->cfg.bc[4] != LBM_BC_PERIODIC)
    return fail(ctx, LBM_EINVAL, "fsi_couple_span: the z axis must be periodic");
  if (!(z0 < 0.0 && z1 > (double)ctx->g.nz))
    return fail(ctx, LBM_EINVAL, "fsi_couple_span: the flag must span the periodic box (z0 < 0, z1 > nz)");
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "fsi_couple_span: set the geometry first");
  if (ctx->shell) return fail(ctx, LBM_ESTATE, "fsi_couple_span: a shell is coupled already");
  const int nn = fem_nodes(f);
  if (first_vertex_z0 < 0 || first_vertex_z0 + 2 * nn > ctx->nv || first_vertex_z1 < 0 ||
      first_vertex_z1 + 2 * nn > ctx->nv ||
      (first_vertex_z0 < first_vertex_z1 + 2 * nn && first_vertex_z1 < first_vertex_z0 + 2 * nn))
    return fail(ctx, LBM_EINVAL, "fsi_couple_span: vertex ranges [%d, +%d) and [%d, +%d) invalid "
                "for a surface of %d vertices", first_vertex_z0, 2 * nn, first_vertex_z1, 2 * nn,
                ctx->nv);
  ctx->fem = f;
  ctx->fem_v0 = first_vertex_z0;
  ctx->graph_dirty = true;
  fem_set_span(f, 1, first_vertex_z1, z0, z1, 1.0 / (double)ctx->g.nz);
  if (fem_reset_stats(f) != LBM_OK)
    return fail(ctx, LBM_ECUDA, "fsi_couple_span: counter reset failed");
  CK(launch_flag_surface(f, (double *)(ctx->ws + ctx->lay.sx), (double *)(ctx->ws + ctx->lay.sv),
                         first_vertex_z0, ctx->stream));
  return run_geometry(ctx, 1);
}

lbm_status fsi_couple_shell(lbm_ctx *ctx, fem_shell_ctx *s, int first_vertex) {
  GUARD();
  ctx->mlp = nullptr;
  if (!s) {
    ctx->shell = nullptr;
    ctx->graph_dirty = true;
    return LBM_OK;
  }
  if (ctx->Q != 27) return fail(ctx, LBM_EINVAL, "fsi_couple_shell: the shell couples to D3Q27 lattices");
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "fsi_couple_shell: set the geometry first");
  if (ctx->fem) return fail(ctx, LBM_ESTATE, "fsi_couple_shell: a beam is coupled already");
  const int nn = shell_nodes(s);
  if (first_vertex < 0 || first_vertex + 2 * nn > ctx->nv)
    return fail(ctx, LBM_EINVAL, "fsi_couple_shell: vertices [%d, %d) outside the surface (%d)",
                first_vertex, first_vertex + 2 * nn, ctx->nv);
  int zero[4];
  if (shell_get_stats(s, zero, 1) != LBM_OK)
    return fail(ctx, LBM_ECUDA, "fsi_couple_shell: counter reset failed");
  ctx->shell = s;
  ctx->shell_v0 = first_vertex;
  ctx->graph_dirty = true;
  CK(launch_shell_surface(s, (double *)(ctx->ws + ctx->lay.sx), (double *)(ctx->ws + ctx->lay.sv),
                          first_vertex, ctx->stream));
  return run_geometry(ctx, 1);
}

lbm_status fsi_set_surrogate(lbm_ctx *ctx, mlp_ctx *mlp, const float *in_mean, const float *in_std,
                             const float *out_mean, const float *out_std, double accept_tol) {
  GUARD();
  if (!mlp) {
    ctx->mlp = nullptr;
    ctx->graph_dirty = true;
    return LBM_OK;
  }
  if (!in_mean || !in_std || !out_mean || !out_std || !(accept_tol > 0.0))
    return fail(ctx, LBM_EINVAL, "fsi_set_surrogate: bad normalisation or tolerance");
  if (ctx->shell) {
    const int nf = shell_free_dofs(ctx->shell);
    if (mlp_dim(mlp, 0) != 5 * nf || mlp_dim(mlp, mlp_layers(mlp)) != nf)
      return fail(ctx, LBM_EINVAL,
                  "fsi_set_surrogate: the network must map %d inputs to %d outputs for this shell",
                  5 * nf, nf);
    lbm_status st = shell_set_surrogate(ctx->shell, in_mean, in_std, out_mean, out_std);
    if (st != LBM_OK) return fail(ctx, st, "fsi_set_surrogate: copy failed");
    ctx->mlp = mlp;
    ctx->accept_tol = accept_tol;
    ctx->graph_dirty = true;
    return LBM_OK;
  }
  if (!ctx->fem) return fail(ctx, LBM_ESTATE, "fsi_set_surrogate: couple a beam or a shell first");
  if (ctx->fem && fem_span(ctx->fem))
    return fail(ctx, LBM_EINVAL, "fsi_set_surrogate: not for a spanwise-coupled beam");
  const int nn = fem_nodes(ctx->fem);
  if (mlp_dim(mlp, 0) != surrogate_inputs(nn) || mlp_dim(mlp, mlp_layers(mlp)) != 3 * nn - 3)
    return fail(ctx, LBM_EINVAL,
                "fsi_set_surrogate: the network must map %d inputs to %d outputs for a %d-node beam",
                surrogate_inputs(nn), 3 * nn - 3, nn);
  if (!in_mean || !in_std || !out_mean || !out_std || !(accept_tol > 0.0))
    return fail(ctx, LBM_EINVAL, "fsi_set_surrogate: bad normalisation or tolerance");
  lbm_status st = fem_set_normalisation(ctx->fem, in_mean, in_std, out_mean, out_std);
  if (st != LBM_OK) return fail(ctx, st, "fsi_set_surrogate: copy failed");
  ctx->mlp = mlp;
  ctx->accept_tol = accept_tol;
  ctx->graph_dirty = true;
  return LBM_OK;
}

lbm_status fsi_get_structure_stats(lbm_ctx *ctx, int stats[4], int reset) {
  GUARD();
  if (!stats) return fail(ctx, LBM_EINVAL, "fsi_get_structure_stats: NULL");
  if (!ctx->fem && !ctx->shell)
    return fail(ctx, LBM_ESTATE, "fsi_get_structure_stats: no structure coupled");
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->shell) {
    lbm_status st = shell_get_stats(ctx->shell, stats, reset);
    if (st != LBM_OK) return fail(ctx, st, "fsi_get_structure_stats: copy failed");
    return LBM_OK;
  }
  lbm_status st = fem_get_stats(ctx->fem, stats);
  if (st == LBM_OK && reset) st = fem_reset_stats(ctx->fem);
  if (st != LBM_OK) return fail(ctx, st, "fsi_get_structure_stats: copy failed");
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_get_boundary_info(lbm_ctx *ctx, int *info) {
  GUARD();
  if (!info) return fail(ctx, LBM_EINVAL, "lbm_get_boundary_info: NULL");
  int h[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, ctx->counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  info[0] = ctx->nface;
  info[1] = ctx->nbodies ? h[0] : 0;
  info[2] = ctx->nbodies ? h[1] : 0;
  info[3] = h[3];
  return LBM_OK;
}

lbm_status lbm_step_graph(lbm_ctx *ctx, int n, int repeats) {
  GUARD();
  if (ctx->ref_coarse)
    return fail(ctx, LBM_ESTATE, "lbm_step_graph: a fine patch is stepped by its coarse lattice");
  if (n <= 0 || (n & 1) || repeats < 0)
    return fail(ctx, LBM_EINVAL, "lbm_step_graph: n must be even and positive, repeats >= 0");
  if (ctx->graph_dirty || ctx->graph_n != n || !ctx->gexec || ctx->cur != ctx->graph_cur ||
      ctx->mp_cur != ctx->graph_mp_cur) {
    if (ctx->gexec) {
      cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = nullptr;
    }
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
    const int cur0 = ctx->cur, mp_cur0 = ctx->mp_cur;
    lbm_status st = lbm_step(ctx, n);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    // an even number of steps returns to the same buffers
    ctx->cur = cur0;
    ctx->mp_cur = mp_cur0;
    ctx->graph_cur = cur0;
    ctx->graph_mp_cur = mp_cur0;
    if (st != LBM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->graph_n = n;
    ctx->graph_dirty = false;
  }
  for (int r = 0; r < repeats; ++r) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
  if (repeats > 0 && ctx->mp_on) ctx->mp_have_force = true;
  return LBM_OK;
}

lbm_status lbm_set_sweep_variant(lbm_ctx *ctx, int variant) {
  GUARD();
  if (variant < LBM_SWEEP_AUTO || variant > LBM_SWEEP_PAIR)
    return fail(ctx, LBM_EINVAL, "lbm_set_sweep_variant: unknown variant %d", variant);
  if (ctx->mp_on && (variant == SWEEP_PAIR) != (ctx->sweep_variant == SWEEP_PAIR)) {
    // the two forms of the multiphase sweep leave per-CTA partials of
    // different grids: restart the momentum controller
    CK(cudaMemsetAsync(ctx->ws + ctx->lay.mp_ctl, 0, sizeof(double) * kMpControl, ctx->stream));
    CK(cudaMemsetAsync(ctx->ws + ctx->lay.mp_partial, 0,
                       mp_partial_bytes(ctx->g.nx, ctx->g.ny, ctx->g.nz), ctx->stream));
  }
  ctx->sweep_variant = variant;
  ctx->graph_dirty = true;
  return LBM_OK;
}

lbm_status lbm_check(lbm_ctx *ctx) {
  GUARD();
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    CK(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
    if (h & 2) return fail(ctx, LBM_ETIMEOUT, "a bounded device wait gave up (flags 0x%x)", h);
    if (h & 4) return fail(ctx, LBM_ECAPACITY, "cut-link list overflowed max_links (flags 0x%x)", h);
    return fail(ctx, LBM_EUNSTABLE, "non-finite or non-positive density met (flags 0x%x)", h);
  }
  return LBM_OK;
}

// Density and velocity of the stored state for interior nodes [begin, begin
// + count): the single-phase read-out, or in the multiphase model the
// density R + sum g_i and the fluid velocity (j - F/2) / rho.
static cudaError_t read_macros(lbm_ctx *ctx, const uint8_t *fl, double *rho, double *u,
                               long long ustride, long long begin, long long count,
                               float *rho32 = nullptr, float *u32 = nullptr) {
  if (ctx->mp_on)
    return launch_mp_read(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], mp_ref(ctx),
                          ctx->ws + ctx->lay.mp_pl, ctx->mp, ctx->mp_have_force,
                          mp_mean_used(ctx), begin, count, ustride, nullptr, rho, u, rho32, u32,
                          nullptr, ctx->stream);
  return launch_macros(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], fl, rho, u, ustride,
                       begin, count, ctx->stream, rho32, u32);
}

lbm_status lbm_get_macros_f32(lbm_ctx *ctx, float *rho, float *u) {
  GUARD();
  if (!rho || !u) return fail(ctx, LBM_EINVAL, "lbm_get_macros_f32: NULL argument");
  const int dim = ctx->Q == 9 ? 2 : 3;
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  const uint8_t *fl = ctx->has_solid ? ctx->flags : nullptr;
  float *dr = nullptr, *du = nullptr;
  if (is_device_ptr(rho) && is_device_ptr(u)) {
    dr = rho;
    du = u;
  } else {
    dr = (float *)mapped_host_ptr(rho);
    du = (float *)mapped_host_ptr(u);
  }
  if (dr && du) {
    // device or page-locked host arrays: written in place
    CK(read_macros(ctx, fl, nullptr, nullptr, n, 0, n, dr, du));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / (sizeof(float) * (1 + dim)));
  float *s = (float *)ctx->stage;
  for (long long b = 0; b < n; b += chunk) {
    const long long cnt = (n - b < chunk) ? n - b : chunk;
    CK(read_macros(ctx, fl, nullptr, nullptr, cnt, b, cnt, s, s + cnt));
    CK(cudaMemcpyAsync(rho + b, s, cnt * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    for (int a = 0; a < dim; ++a)
      CK(cudaMemcpyAsync(u + a * n + b, s + (1 + a) * cnt, cnt * sizeof(float),
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

lbm_status lbm_get_macros(lbm_ctx *ctx, double *rho, double *u) {
  GUARD();
  if (!rho || !u) return fail(ctx, LBM_EINVAL, "lbm_get_macros: NULL argument");
  const int dim = ctx->Q == 9 ? 2 : 3;
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  const uint8_t *fl = ctx->has_solid ? ctx->flags : nullptr;
  if (is_device_ptr(rho) && is_device_ptr(u)) {
    CK(read_macros(ctx, fl, rho, u, n, 0, n));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  double *mr = (double *)mapped_host_ptr(rho), *mu = (double *)mapped_host_ptr(u);
  if (mr && mu) {
    // page-locked host arrays: the kernel writes them in place (no staging)
    CK(read_macros(ctx, fl, mr, mu, n, 0, n));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / (sizeof(double) * (1 + dim)));
  double *s = (double *)ctx->stage;
  for (long long b = 0; b < n; b += chunk) {
    const long long cnt = (n - b < chunk) ? n - b : chunk;
    CK(read_macros(ctx, fl, s, s + cnt, cnt, b, cnt));
    CK(cudaMemcpyAsync(rho + b, s, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    for (int a = 0; a < dim; ++a)
      CK(cudaMemcpyAsync(u + a * n + b, s + (1 + a) * cnt, cnt * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Force probe without allocation.
//
// For callers that cannot allocate device memory at this point (for example
// code running where cudaMalloc is not allowed: inside a memory-pool budget
// fixed at start-up, or on a path that must not synchronise the device as a
// cudaMalloc may).  Its scratch -- the boundary-node list, the cut-link
// list, the counters and the FP64 force accumulators -- lives in one
// file-scope device array that every GPU loading this library holds until
// the process exits.  Every call reuses it; calls that overlap on the GPU
// race on it.
namespace {

constexpr int kProbeMaxLinks = 65536;
constexpr int kProbeMaxNodes = 65536;
constexpr int kProbeMaxVertices = 16384;
constexpr size_t kProbeLinksOff = 0;
constexpr size_t kProbeNodesOff = align_up(sizeof(Link) * kProbeMaxLinks);
constexpr size_t kProbeVforceOff = kProbeNodesOff + align_up(sizeof(BNode) * kProbeMaxNodes);
constexpr size_t kProbeBforceOff =
    kProbeVforceOff + align_up(sizeof(double) * 3 * kProbeMaxVertices);
constexpr size_t kProbeCountOff = kProbeBforceOff + align_up(sizeof(double) * 3 * kMaxBodies);
constexpr size_t kProbeBytes = kProbeCountOff + kAlign;  // about 5.4 MB

static __device__ __align__(256) unsigned char g_probe_scratch[kProbeBytes];

constexpr int kProbeMaxDevices = 64;
// device address of g_probe_scratch per device, looked up once per device
// (std::call_once: host threads making their first call together agree)
static char *g_probe_ptr[kProbeMaxDevices];
static cudaError_t g_probe_err[kProbeMaxDevices];
static std::once_flag g_probe_once[kProbeMaxDevices];

}  // namespace

extern "C" lbm_status lbm_probe_interface_force_static(lbm_ctx *ctx, double *vert_force,
                                                       double *body_force) {
  GUARD();
  if (ctx->nbodies == 0) return fail(ctx, LBM_ESTATE, "lbm_probe_interface_force_static: no geometry");
  if (ctx->nv > kProbeMaxVertices)
    return fail(ctx, LBM_ECAPACITY,
                "lbm_probe_interface_force_static: %d surface vertices exceed the fixed maximum %d",
                ctx->nv, kProbeMaxVertices);
  // the array's address is per device: the context's device must be current
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(ctx, LBM_EINVAL,
                "lbm_probe_interface_force_static: device %d is current, the context lives on "
                "device %d",
                dev, ctx->device);
  if (dev < 0 || dev >= kProbeMaxDevices)
    return fail(ctx, LBM_EINVAL, "lbm_probe_interface_force_static: device %d unsupported", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(ctx->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(ctx, LBM_ESTATE,
                "lbm_probe_interface_force_static: the stream is being captured (the probe "
                "synchronises)");
  // first call on this device (device current): the host-side name of the
  // array is only a stand-in, the kernels need its device address
  std::call_once(g_probe_once[dev], [dev]() {
    void *p = nullptr;
    g_probe_err[dev] = cudaGetSymbolAddress(&p, g_probe_scratch);
    g_probe_ptr[dev] = (char *)p;
  });
  if (g_probe_err[dev] != cudaSuccess)
    return cuda_fail(ctx, g_probe_err[dev], "cudaGetSymbolAddress(g_probe_scratch)");
  char *base = g_probe_ptr[dev];
  Link *links = (Link *)(base + kProbeLinksOff);
  BNode *nodes = (BNode *)(base + kProbeNodesOff);
  double *vf = (double *)(base + kProbeVforceOff);
  double *bf = (double *)(base + kProbeBforceOff);
  int *cnt = (int *)(base + kProbeCountOff);  // [0] nodes, [1] links, [2] overflow flags
  // the array keeps the previous call's contents: clear what must start at zero
  CK(cudaMemsetAsync(cnt, 0, 4 * sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(vf, 0, sizeof(double) * 3 * (size_t)ctx->nv, ctx->stream));
  CK(cudaMemsetAsync(bf, 0, sizeof(double) * 3 * kMaxBodies, ctx->stream));
  CK(launch_build_links(ctx->Q, ctx->g, ctx->band, surface_dev(ctx), ctx->flags, nodes, cnt,
                        kProbeMaxNodes, links, cnt + 1, kProbeMaxLinks, cnt + 2, ctx->stream));
  CK(launch_grad(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], ctx->flags, nodes, cnt, 0,
                 kProbeMaxNodes, links, ctx->bp, vf, bf, ctx->nbodies, ctx->stream));
  int h[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(h, cnt, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (vert_force)
    CK(cudaMemcpyAsync(vert_force, vf, sizeof(double) * 3 * ctx->nv, cudaMemcpyDefault,
                       ctx->stream));
  if (body_force)
    CK(cudaMemcpyAsync(body_force, bf, sizeof(double) * 3 * ctx->nbodies, cudaMemcpyDefault,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h[2] || h[0] > kProbeMaxNodes || h[1] > kProbeMaxLinks)
    return fail(ctx, LBM_ECAPACITY,
                "lbm_probe_interface_force_static: %d boundary nodes / %d cut links exceed the "
                "fixed maximum %d / %d",
                h[0], h[1], kProbeMaxNodes, kProbeMaxLinks);
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches: many lattices advanced by one launch per phase.
struct lbm_batch {
  int n = 0;
  std::vector<lbm_ctx *> ctx;
  int Q = 0, storage = 0;
  cudaStream_t stream = nullptr;
  char *ws = nullptr;
  bool own_ws = false;
  InstDesc *d_desc = nullptr;
  int4 *d_tiles = nullptr;
  int *d_ticket = nullptr;
  int *d_coupled = nullptr;
  BeamBatchDesc *d_beam = nullptr;
  int ncoupled = 0;
  int beam_fp64 = 0;  // some coupled beam solves its Newton systems in FP64
  int max_cap = 0, max_nv3 = 0, max_fresh = 0;
  long long max_band = 0;
  int ntiles = 0, max_tiles = 0;
  int rows_per_tile = 1, ctas_per_sm = KBC_BATCH_CTAS;
  int parity = 0;
  std::vector<int> cur0;
  cudaGraphExec_t gexec = nullptr;
  int graph_n = 0;
  bool graph_dirty = true;
  char msg[256] = {0};
};

namespace {

size_t batch_tiles_capacity(lbm_ctx *const *ctxs, int n) {
  size_t t = 0;
  for (int i = 0; i < n; ++i)
    t += (size_t)ctxs[i]->g.ny * ctxs[i]->g.nz * ((ctxs[i]->g.nx + 127) / 128);
  return t;
}

struct BatchLayout {
  size_t desc, tiles, ticket, coupled, beam, total;
};

BatchLayout batch_layout(lbm_ctx *const *ctxs, int n) {
  BatchLayout L;
  size_t off = 0;
  L.desc = off; off += align_up(sizeof(InstDesc) * (size_t)n);
  L.tiles = off; off += align_up(sizeof(int4) * std::max<size_t>(1, batch_tiles_capacity(ctxs, n)));
  L.ticket = off; off += kAlign;
  L.coupled = off; off += align_up(sizeof(int) * (size_t)n);
  L.beam = off; off += align_up(sizeof(BeamBatchDesc) * (size_t)n);
  L.total = off;
  return L;
}

// Tiles (lattice, first row, x segment), largest lattices first.
std::vector<int4> batch_tiles(lbm_batch *b) {
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)b->ctx[a]->g.nx * b->ctx[a]->g.ny * b->ctx[a]->g.nz >
           (long long)b->ctx[c]->g.nx * b->ctx[c]->g.ny * b->ctx[c]->g.nz;
  });
  std::vector<int4> t;
  for (int i : order) {
    const Grid &g = b->ctx[i]->g;
    const int rows = g.ny * g.nz, xs = (g.nx + 127) / 128;
    for (int r = 0; r < rows; r += b->rows_per_tile)
      for (int x = 0; x < xs; ++x) t.push_back(make_int4(i, r, x, 0));
  }
  return t;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_size(lbm_ctx *const *ctxs, int n, size_t *bytes) {
  if (!ctxs || n < 1 || !bytes) return LBM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return LBM_EINVAL;
  *bytes = batch_layout(ctxs, n).total;
  return LBM_OK;
}

lbm_status lbm_batch_create(lbm_ctx *const *ctxs, int n, void *workspace, size_t bytes,
                            lbm_batch **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) return LBM_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || ctxs[i]->poisoned) return LBM_EINVAL;
    if (ctxs[i]->Q != ctxs[0]->Q || ctxs[i]->cfg.storage != ctxs[0]->cfg.storage ||
        ctxs[i]->stream != ctxs[0]->stream) {
      snprintf(g_create_msg, sizeof(g_create_msg),
               "lbm_batch_create: lattices must share lattice type, storage and stream");
      return LBM_EINVAL;
    }
    if (ctxs[i]->sweep_variant == SWEEP_ROWS) return LBM_EINVAL;
    if (ctxs[i]->mp_on) {
      snprintf(g_create_msg, sizeof(g_create_msg),
               "lbm_batch_create: multiphase lattices are stepped one by one");
      return LBM_EINVAL;
    }
    if (ctxs[i]->ref_fine || ctxs[i]->ref_coarse) {
      snprintf(g_create_msg, sizeof(g_create_msg),
               "lbm_batch_create: a lattice of a refined pair is stepped by its pair");
      return LBM_EINVAL;
    }
  }
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->n = n;
  b->ctx.assign(ctxs, ctxs + n);
  b->Q = ctxs[0]->Q;
  b->storage = ctxs[0]->cfg.storage;
  if (b->Q == 9) b->rows_per_tile = 4;  // D2Q9: the sweep gathers 4 rows together
  b->stream = ctxs[0]->stream;
  const BatchLayout L = batch_layout(ctxs, n);
  if (workspace) {
    if (bytes < L.total || ((uintptr_t)workspace % kAlign)) {
      delete b;
      return LBM_ENOMEM;
    }
    b->ws = (char *)workspace;
  } else {
    if (cudaMalloc((void **)&b->ws, L.total) != cudaSuccess) {
      delete b;
      return LBM_ENOMEM;
    }
    b->own_ws = true;
  }
  b->d_desc = (InstDesc *)(b->ws + L.desc);
  b->d_tiles = (int4 *)(b->ws + L.tiles);
  b->d_ticket = (int *)(b->ws + L.ticket);
  b->d_coupled = (int *)(b->ws + L.coupled);
  b->d_beam = (BeamBatchDesc *)(b->ws + L.beam);
  b->max_tiles = (int)batch_tiles_capacity(ctxs, n);
  std::vector<InstDesc> hd(n);
  std::vector<int> coupled;
  std::vector<BeamBatchDesc> beams;
  b->cur0.resize(n);
  for (int i = 0; i < n; ++i) {
    lbm_ctx *c = ctxs[i];
    InstDesc &d = hd[i];
    memset(&d, 0, sizeof(d));
    d.g = c->g;
    d.f[0] = c->f[0];
    d.f[1] = c->f[1];
    d.cur0 = c->cur;
    b->cur0[i] = c->cur;
    d.flags = c->flags;
    d.beta = c->cfg.beta;
    d.bgk = c->cfg.collision == LBM_COLLIDE_BGK;
    d.err = c->err;
    d.narrow = (long long)c->Q * c->g.N < (1LL << 31);
    d.bnodes = (BNode *)(c->ws + c->lay.bnodes);
    d.nbn = c->nbodies > 0 ? c->counters : nullptr;
    d.nfixed = c->nface;
    d.cap = c->nface + (c->nbodies > 0 ? c->cfg.max_links : 0);
    d.links = (Link *)(c->ws + c->lay.links);
    d.bp = c->bp;
    d.vforce = (double *)(c->ws + c->lay.vforce);
    d.bforce = (double *)(c->ws + c->lay.bforce);
    d.nbodies = c->nbodies;
    d.nv = c->nv;
    d.coupled = c->fem != nullptr;
    d.band = c->band;
    d.sd = surface_dev(c);
    d.fresh = (int64_t *)(c->ws + c->lay.fresh);
    d.nfresh = c->counters + 2;
    d.nl = c->counters + 1;
    d.lcap = c->cfg.max_links;
    b->max_cap = std::max(b->max_cap, d.cap);
    b->max_nv3 = std::max(b->max_nv3, 3 * std::max(d.nv, kMaxBodies));
    if (c->fem) {
      coupled.push_back(i);
      BeamBatchDesc bd;
      fem_describe(c->fem, &bd.p, &bd.d);
      bd.vforce = d.vforce;
      bd.surf_x = (double *)(c->ws + c->lay.sx);
      bd.surf_v = (double *)(c->ws + c->lay.sv);
      bd.v0 = c->fem_v0;
      if (bd.p.solve64) b->beam_fp64 = 1;
      beams.push_back(bd);
      const Band &B = c->band;
      b->max_band = std::max(b->max_band, (long long)(B.x1 - B.x0) * (B.y1 - B.y0) * (B.z1 - B.z0));
      b->max_fresh = std::max(b->max_fresh, c->cfg.max_links);
    }
  }
  b->ncoupled = (int)coupled.size();
  cudaError_t e = cudaMemcpyAsync(b->d_desc, hd.data(), sizeof(InstDesc) * n,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && b->ncoupled)
    e = cudaMemcpyAsync(b->d_coupled, coupled.data(), sizeof(int) * b->ncoupled,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && b->ncoupled)
    e = cudaMemcpyAsync(b->d_beam, beams.data(), sizeof(BeamBatchDesc) * b->ncoupled,
                        cudaMemcpyHostToDevice, b->stream);
  std::vector<int4> t = batch_tiles(b);
  b->ntiles = (int)t.size();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    if (b->own_ws) cudaFree(b->ws);
    delete b;
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->msg : g_create_msg; }

#define BCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      snprintf(b->msg, sizeof(b->msg), "%s: %s", #call, cudaGetErrorString(e_));   \
      return LBM_ECUDA;                                                            \
    }                                                                              \
  } while (0)

static lbm_status batch_steps(lbm_batch *b, int nsteps) {
  for (int t = 0; t < nsteps; ++t) {
    BCK(launch_batch_pre(b->d_desc, b->n, b->max_nv3, b->d_ticket, b->stream));
    BCK(launch_grad_batch(b->Q, b->storage, b->d_desc, b->n, b->max_cap, b->parity, b->stream));
    BCK(launch_sweep_batch(b->Q, b->storage, b->d_desc, b->n, b->d_tiles, b->ntiles, b->d_ticket,
                           b->parity, b->rows_per_tile, b->ctas_per_sm, b->stream));
    b->parity ^= 1;
    if (b->ncoupled) {
      BCK(launch_beam_batch(b->d_beam, b->ncoupled, b->beam_fp64, b->stream));
      BCK(launch_geometry_batch(b->Q, b->storage, b->d_desc, b->d_coupled, b->ncoupled,
                                b->max_band, b->max_fresh, b->parity, b->stream));
    }
  }
  for (int i = 0; i < b->n; ++i) b->ctx[i]->cur = (b->cur0[i] + b->parity) & 1;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int nsteps) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  return batch_steps(b, nsteps);
}

lbm_status lbm_batch_step_graph(lbm_batch *b, int n, int repeats) {
  if (!b || n <= 0 || (n & 1) || repeats < 0) return LBM_EINVAL;
  if (b->graph_dirty || b->graph_n != n || !b->gexec) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    const int p0 = b->parity;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
    lbm_status st = batch_steps(b, n);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    b->parity = p0;  // capture does not advance the state
    for (int i = 0; i < b->n; ++i) b->ctx[i]->cur = (b->cur0[i] + b->parity) & 1;
    if (st != LBM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    BCK(e);
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    BCK(e);
    b->graph_n = n;
    b->graph_dirty = false;
  }
  for (int r = 0; r < repeats; ++r) BCK(cudaGraphLaunch(b->gexec, b->stream));
  // an even n leaves every lattice's buffer roles unchanged
  return LBM_OK;
}

lbm_status lbm_batch_set_tuning(lbm_batch *b, int rows_per_tile, int ctas_per_sm) {
  if (!b || rows_per_tile < 1 || rows_per_tile > 64 || ctas_per_sm < 1 || ctas_per_sm > 32)
    return LBM_EINVAL;
  b->ctas_per_sm = ctas_per_sm;
  if (rows_per_tile != b->rows_per_tile) {
    b->rows_per_tile = rows_per_tile;
    std::vector<int4> t = batch_tiles(b);
    b->ntiles = (int)t.size();
    BCK(cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
  }
  b->graph_dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *best_rows, int *best_ctas,
                              float *best_us) {
  if (!b || steps < 2) return LBM_EINVAL;
  const int rows_c[] = {1, 2, 4, 8};
  const int ctas_c[] = {3, 4, 5, 6, 8};
  float best = 1e30f;
  int br = b->rows_per_tile, bc = b->ctas_per_sm;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  for (int r : rows_c)
    for (int c : ctas_c) {
      lbm_status st = lbm_batch_set_tuning(b, r, c);
      if (st != LBM_OK) return st;
      if ((st = batch_steps(b, 2)) != LBM_OK) return st;  // warm-up
      BCK(cudaEventRecord(e0, b->stream));
      if ((st = batch_steps(b, steps)) != LBM_OK) return st;
      BCK(cudaEventRecord(e1, b->stream));
      BCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, e0, e1));
      const float us = ms * 1e3f / steps;
      if (us < best) {
        best = us;
        br = r;
        bc = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lbm_status st = lbm_batch_set_tuning(b, br, bc);
  if (st != LBM_OK) return st;
  if (best_rows) *best_rows = br;
  if (best_ctas) *best_ctas = bc;
  if (best_us) *best_us = best;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->own_ws) cudaFree(b->ws);
  delete b;
}

}  // extern "C"
