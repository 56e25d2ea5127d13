// lbm_api.cu -- the C ABI (include/kbc_lbm.h): context, workspace layout,
// host/device argument staging and step orchestration.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/kbc_lbm.h"
#include "lbm_internal.h"

using namespace kbc;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStageBytes = 16u << 20;  // host<->device staging chunk

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t f[2], flags, err, stage, total;
};

int pop_bytes(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

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
  if (c->storage < LBM_STORE_F32 || c->storage > LBM_STORE_BF16) return "unknown storage";
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
  return nullptr;
}

}  // namespace

struct lbm_ctx {
  lbm_config cfg;
  Grid g;
  Layout lay;
  int Q = 0;
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
  *out = ctx;
  return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->msg : g_create_msg; }

void *lbm_stream(const lbm_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

void lbm_destroy(lbm_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->own_ws) cudaFree(ctx->ws);
  delete ctx;
}

#define GUARD()                                                              \
  do {                                                                       \
    if (!ctx) return LBM_EINVAL;                                             \
    if (ctx->poisoned) return fail(ctx, LBM_ESTATE, "context poisoned: %s", ctx->msg); \
  } while (0)

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u) {
  GUARD();
  if (!rho || !u) return fail(ctx, LBM_EINVAL, "lbm_init_equilibrium: NULL argument");
  const int dim = ctx->Q == 9 ? 2 : 3;
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  const bool dev = is_device_ptr(rho) && is_device_ptr(u);
  if (dev) {
    CK(launch_init_eq(ctx->Q, ctx->cfg.storage, ctx->g, rho, u, n, 0, n, ctx->f[ctx->cur],
                      ctx->stream));
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
  const long long n = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
  if (is_device_ptr(f)) {
    for (int i = 0; i < ctx->Q; ++i)
      CK(launch_set_pop(ctx->Q, ctx->cfg.storage, ctx->g, i, f + i * n, 0, n, ctx->f[ctx->cur],
                        ctx->stream));
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

lbm_status lbm_step(lbm_ctx *ctx, int n) {
  GUARD();
  if (n < 0) return fail(ctx, LBM_EINVAL, "lbm_step: n < 0");
  const float beta = (float)ctx->cfg.beta;
  const int bgk = ctx->cfg.collision == LBM_COLLIDE_BGK;
  for (int t = 0; t < n; ++t) {
    CK(launch_sweep(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], ctx->f[1 - ctx->cur],
                    ctx->has_solid || ctx->g.px || ctx->g.py || ctx->g.pz ? ctx->flags : nullptr,
                    beta, bgk, ctx->err, ctx->stream, ctx->sweep_variant));
    ctx->cur = 1 - ctx->cur;
  }
  return LBM_OK;
}

lbm_status lbm_set_sweep_variant(lbm_ctx *ctx, int variant) {
  GUARD();
  if (variant < LBM_SWEEP_AUTO || variant > LBM_SWEEP_ROWS)
    return fail(ctx, LBM_EINVAL, "lbm_set_sweep_variant: unknown variant %d", variant);
  ctx->sweep_variant = variant;
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
    return fail(ctx, LBM_EUNSTABLE, "non-finite or non-positive density met (flags 0x%x)", h);
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
    CK(launch_macros(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], fl, rho, u, n, 0, n,
                     ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
  }
  const long long chunk = (long long)(kStageBytes / (sizeof(double) * (1 + dim)));
  double *s = (double *)ctx->stage;
  for (long long b = 0; b < n; b += chunk) {
    const long long cnt = (n - b < chunk) ? n - b : chunk;
    CK(launch_macros(ctx->Q, ctx->cfg.storage, ctx->g, ctx->f[ctx->cur], fl, s, s + cnt, cnt, b,
                     cnt, ctx->stream));
    CK(cudaMemcpyAsync(rho + b, s, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    for (int a = 0; a < dim; ++a)
      CK(cudaMemcpyAsync(u + a * n + b, s + (1 + a) * cnt, cnt * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

}  // extern "C"
