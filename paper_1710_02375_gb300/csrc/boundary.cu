// boundary.cu -- Grad's-approximation boundary fill, cut-link geometry and
// the momentum-exchange force gather (arXiv 1710.02375, section "Fluid
// boundary conditions", Eq. (grad); section "Solid boundary conditions").
//
// Readings of the target values (the paper defers them to earlier work):
//   missing set M(x_b): directions i whose source x_b - c_i is solid or a
//     ghost beyond a non-periodic face;
//   immersed link i: crossing at x_b - q_i c_i (nearest, q in (0,1]) with the
//     wall velocity interpolated on the hit element; a wall face: q = 1/2 and
//     the face velocity;
//   open node (a missing link crosses an inlet/outlet/free-stream face, first
//     such face in the order -x,+x,-y,+y,-z,+z): inlet u_t = prescribed,
//     rho_t = rho(x_n); outlet u_t = u(x_n), rho_t = 1; free stream
//     u_t = face velocity, rho_t = 1, grad u = 0 (x_n: next node inward);
//   wall node: u_t = mean over M of (u_w + q u(x_b + c_i)) / (1 + q) (u_w
//     alone if x_b + c_i is not fluid); rho_t = moving-wall bounce-back density
//     sum_known f_i + sum_M [f'_opp(i)(x_b) + 6 W_i c_i.u_w];
//   grad u: central differences of the previous-step velocity, one-sided
//     second order through x_b at walls (first order with one fluid node);
//   f*_i = W_i [rho + 3 rho c_i.u + 9/2 (rho u u + Pi_neq):(c_i c_i - I/3)],
//     Pi_neq = -rho/(6 beta) (grad u + grad u^T), for every missing i;
//   force on the surface per immersed link: -c_i (f'_opp(i)(x_b) + f*_i - 2 W_i)
//     (relative to the rest state, i.e. without the uniform ambient pressure,
//     which cancels on a closed body but loads one attached to another),
//     accumulated in FP64 per vertex (interpolation weights) and per body.
// The previous-step velocity of a node is the first moment of its stored
// post-collision populations (collisions conserve it).
//
// Layout: the fill writes f*_i straight into the solid (or ghost) slot
// A[i][x_b - c_i] of the source buffer, which the fused sweep then pulls
// unchanged; no boundary branch is needed in the sweep itself.
#include <type_traits>

#include "boundary.cuh"
#include "lbm_internal.h"

namespace kbc {

// ---------------------------------------------------------------- helpers

// Stored coordinate S + c on one axis; -1 if it leaves the interior of a
// padded (non-periodic) axis.
__device__ __forceinline__ int step_axis(int S, int c, int NS, int pad) {
  int s = S + c;
  if (pad) return (s < pad || s >= NS - pad) ? -1 : s;
  while (s < 0) s += NS;
  while (s >= NS) s -= NS;
  return s;
}

// Knuth's TwoSum: s + e == a + b exactly in round-to-nearest FP32 (the
// additions are kept in this order: no fast-math, no contraction here).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// Sum of stored FP32 values in the caller's precision.  FP64: cascaded
// TwoSum with the rounding errors gathered in a second FP32 word (Ogita,
// Rump and Oishi's Sum2); hi + lo is the sum to within about (n 2^-24)^2 of
// the sum of magnitudes -- FP64 summation accuracy for a handful of terms --
// with every add on the FP32 pipes (FP64 instructions are scarce on this
// part and the boundary pass is bound by them).  FP32: a plain running sum.
template <typename R>
struct PopSum {
  float s = 0.f;
  __device__ __forceinline__ void add(float x) { s += x; }
  __device__ __forceinline__ void sub(float x) { s -= x; }
  __device__ __forceinline__ float value() const { return s; }
};
template <>
struct PopSum<double> {
  float hi = 0.f, lo = 0.f;
  double d = 0.0;  // FP64 stored values (F64 storage) are summed in FP64
  __device__ __forceinline__ void add(float x) {
    float t, e;
    two_sum(hi, x, t, e);
    hi = t;
    lo += e;
  }
  __device__ __forceinline__ void add(double x) { d += x; }
  __device__ __forceinline__ void sub(float x) { add(-x); }
  __device__ __forceinline__ void sub(double x) { d -= x; }
  __device__ __forceinline__ double value() const { return ((double)hi + (double)lo) + d; }
};

// (nh + nl) / (dh + dl) for unevaluated FP32 pairs, as a double: the FP32
// quotient q1, its exact remainder nh - q1 dh (one fused multiply-add), the
// correction q2 from the remainder and the low parts; q1 + q2 carries about
// 44 bits.
__device__ __forceinline__ double df_div(float nh, float nl, float dh, float dl) {
  const float q1 = __fdiv_rn(nh, dh);
  float r = fmaf(-q1, dh, nh);
  r = (r + nl) - q1 * dl;
  const float q2 = __fdiv_rn(r, dh);
  return (double)q1 + (double)q2;
}

// Per-direction constants for directions known only at run time (the same
// values as weight<L>, read from constant memory instead of recomputed in
// FP64): W_i, W_i and 1 / W_i in FP32.
template <int Q>
struct DirTab {
  double w[Q];
  float wf[Q], iwf[Q];
  constexpr DirTab() : w(), wf(), iwf() {
    for (int i = 0; i < Q; ++i) {
      w[i] = weight<Lat<Q>>(i);
      wf[i] = (float)w[i];
      iwf[i] = (float)(1.0 / w[i]);
    }
  }
};
__constant__ DirTab<9> c_dir9 = DirTab<9>();
__constant__ DirTab<27> c_dir27 = DirTab<27>();
template <int Q>
__device__ __forceinline__ const DirTab<Q> &dir_tab() {
  if constexpr (Q == 9) return c_dir9;
  else return c_dir27;
}

// Deviation moments of a node.  D2Q9 in FP64 (the boundary path): the
// stored values summed with PopSum<double>.  Otherwise FP32 sums returned in
// the caller's type (27 FP64 adds per neighbour would dominate the 3-D
// boundary pass).  Directions with a zero component skip that moment.
template <int Q, int S, typename R = float>
__device__ void dev_moments(const Grid &g, const typename Store<S>::T *f, long long k, R &drho,
                            R (&j)[3]) {
  using L = Lat<Q>;
  using A = typename std::conditional<Q == 9 && std::is_same<R, double>::value, double, float>::type;
  PopSum<A> dr, jx, jy, jz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const auto v = Store<S>::load(f + (long long)i * g.N + k, (typename Store<S>::C)weight<L>(i));
    dr.add(v);
    if (L::cx(i) > 0) jx.add(v);
    if (L::cx(i) < 0) jx.sub(v);
    if (L::cy(i) > 0) jy.add(v);
    if (L::cy(i) < 0) jy.sub(v);
    if (L::cz(i) > 0) jz.add(v);
    if (L::cz(i) < 0) jz.sub(v);
  }
  drho = (R)dr.value();
  j[0] = (R)jx.value();
  j[1] = (R)jy.value();
  j[2] = L::D == 3 ? (R)jz.value() : (R)0;
}

// Velocity (and density) of a node; in FP64 one reciprocal of rho instead of
// a division per component.
template <int Q, int S, typename R = float>
__device__ void dev_velocity(const Grid &g, const typename Store<S>::T *f, long long k, R (&u)[3],
                             R *rho = nullptr) {
  if constexpr (std::is_same<typename Store<S>::C, double>::value) {
    // FP64 storage: FP64 sums and one FP64 reciprocal of rho
    using L = Lat<Q>;
    double dr = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = Store<S>::load(f + (long long)i * g.N + k, weight<L>(i));
      dr += v;
      if (L::cx(i)) j[0] += L::cx(i) * v;
      if (L::cy(i)) j[1] += L::cy(i) * v;
      if (L::cz(i)) j[2] += L::cz(i) * v;
    }
    const double r = 1.0 + dr, ir = 1.0 / r;
    for (int a = 0; a < 3; ++a) u[a] = (R)(j[a] * ir);
    if (rho) *rho = (R)r;
    return;
  } else if constexpr (Q == 9 && std::is_same<R, double>::value) {
    // D2Q9 in FP64: the moments stay unevaluated FP32 pairs (hi + lo) and
    // rho = 1 + drho and u = j / rho are formed in double-float arithmetic
    // on the FP32 pipes (about 44 bits), with one conversion pair per
    // result instead of FP64 sums and an FP64 division
    using L = Lat<Q>;
    PopSum<double> dr, jx, jy;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float v = Store<S>::load(f + (long long)i * g.N + k, (float)weight<L>(i));
      dr.add(v);
      if (L::cx(i) > 0) jx.add(v);
      if (L::cx(i) < 0) jx.sub(v);
      if (L::cy(i) > 0) jy.add(v);
      if (L::cy(i) < 0) jy.sub(v);
    }
    float rh, rl;
    two_sum(1.0f, dr.hi, rh, rl);
    rl += dr.lo;
    u[0] = df_div(jx.hi, jx.lo, rh, rl);
    u[1] = df_div(jy.hi, jy.lo, rh, rl);
    u[2] = 0.0;
    if (rho) *rho = (double)rh + (double)rl;
    return;
  }
  if constexpr (Q == 27 && std::is_same<R, double>::value) {
    // D3Q27 in FP64: FP32 moment sums (as in dev_moments), then rho and the
    // quotients in double-float arithmetic (as above) instead of an FP64
    // division
    float drf, jf[3];
    dev_moments<Q, S, float>(g, f, k, drf, jf);
    float rh, rl;
    two_sum(1.0f, drf, rh, rl);
    for (int a = 0; a < 3; ++a) u[a] = df_div(jf[a], 0.0f, rh, rl);
    if (rho) *rho = (double)rh + (double)rl;
    return;
  }
  R dr, j[3];
  dev_moments<Q, S, R>(g, f, k, dr, j);
  const R r = (R)1 + dr;
  if constexpr (std::is_same<R, double>::value) {
    const R ir = (R)1 / r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] * ir;
  } else {
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
  }
  if (rho) *rho = r;
}

// ---------------------------------------------------------------- ghosts / faces
__global__ void k_mark_ghosts(Grid g, uint8_t *flags) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.N) return;
  int X, Y, Z;
  decompose(g, k, X, Y, Z);
  const bool ghost = X >= g.NX || (g.px && (X == 0 || X == g.NX - 1)) ||
                     (g.py && (Y == 0 || Y == g.NY - 1)) || (g.pz && (Z == 0 || Z == g.NZ - 1));
  flags[k] = ghost ? NODE_GHOST : NODE_FLUID;
}

// Interior nodes that touch a non-periodic face.
__global__ void k_face_nodes(Grid g, BNode *out, int *count, int cap) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)g.nx * g.ny * g.nz;
  if (t >= n) return;
  const int x = (int)(t % g.nx), y = (int)((t / g.nx) % g.ny), z = (int)(t / ((long long)g.nx * g.ny));
  const bool face = (g.px && (x == 0 || x == g.nx - 1)) || (g.py && (y == 0 || y == g.ny - 1)) ||
                    (g.pz && (z == 0 || z == g.nz - 1));
  if (!face) return;
  const int slot = atomicAdd(count, 1);
  if (slot < cap) out[slot] = BNode{sidx(g, x + g.px, y + g.py, z + g.pz), -1, 0};
}

// ---------------------------------------------------------------- geometry (FP64)
__constant__ double c_ray2[2] = {0.8191520442889918, 0.5735764363510461};
__constant__ double c_ray3[3] = {0.6245004513516506, 0.4806291366599437, 0.6155950585117604};

// Crossing of the ray p + t d (t > 0) with segment a-b at parameter s in
// [0, 1), decided without division: t = tn/den > 0 and s = sn/den in [0, 1).
__device__ bool seg_ray_cross(const double *p, const double *d, const double *a, const double *b) {
  const double ex = b[0] - a[0], ey = b[1] - a[1];
  const double den = d[0] * (-ey) - d[1] * (-ex);
  if (fabs(den) < 1e-300) return false;
  const double rx = a[0] - p[0], ry = a[1] - p[1];
  const double tn = rx * (-ey) - ry * (-ex);
  const double sn = d[0] * ry - d[1] * rx;
  if (den > 0.0) return tn > 0.0 && sn >= 0.0 && sn < den;
  return tn < 0.0 && sn <= 0.0 && sn > den;
}

// Moller-Trumbore; barycentrics (1-u-v, u, v) at distance t along d.
__device__ bool tri_ray(const double *p, const double *d, const double *a, const double *b,
                        const double *c, double &t, double &u, double &v) {
  const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double pv[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2],
                        d[0] * e2[1] - d[1] * e2[0]};
  const double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
  if (fabs(det) < 1e-300) return false;
  const double inv = 1.0 / det;
  const double tv[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
  const double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2],
                        tv[0] * e1[1] - tv[1] * e1[0]};
  v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
  t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
  return true;
}

// Within tol of triangle (a, b, c): distance to its plane <= tol |n| and the
// in-plane barycentrics in [0, 1].
__device__ bool on_triangle(const double *p, const double *a, const double *b, const double *c,
                            double tol) {
  const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  const double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
  const double nn = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
  if (nn == 0.0 || fabs(nr[0] * w[0] + nr[1] * w[1] + nr[2] * w[2]) > tol * nn) return false;
  const double d11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  const double d12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
  const double d22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  const double dw1 = w[0] * e1[0] + w[1] * e1[1] + w[2] * e1[2];
  const double dw2 = w[0] * e2[0] + w[1] * e2[1] + w[2] * e2[2];
  const double den = d11 * d22 - d12 * d12;
  const double u = (d22 * dw1 - d12 * dw2) / den, v = (d11 * dw2 - d12 * dw1) / den;
  return u >= 0.0 && v >= 0.0 && u + v <= 1.0;
}

// Within 1e-12 of an element: a node exactly on a face is solid (the parity
// test alone would depend on the ray direction there).
__device__ bool on_surface(const SurfaceDev &s, const double *p) {
  const double tol = 1e-12;
  for (int k = 0; k < s.ne; ++k) {
    if (s.dim == 2) {
      const double *a = s.x + 2 * s.e[2 * k], *b = s.x + 2 * s.e[2 * k + 1];
      const double ex = b[0] - a[0], ey = b[1] - a[1];
      const double px = p[0] - a[0], py = p[1] - a[1];
      const double len2 = ex * ex + ey * ey;
      const double cr = ex * py - ey * px, dt = ex * px + ey * py;
      // a zero-length element has no surface
      if (len2 > 0.0 && fabs(cr) <= tol * sqrt(len2) && dt >= 0.0 && dt <= len2) return true;
    } else {
      if (on_triangle(p, s.x + 3 * s.e[3 * k], s.x + 3 * s.e[3 * k + 1], s.x + 3 * s.e[3 * k + 2],
                      tol))
        return true;
    }
  }
  return false;
}

__device__ bool inside_any(const SurfaceDev &s, const double *p) {
  if (on_surface(s, p)) return true;
  // crossing parity per body; a node is solid inside any body
  for (int b = 0; b < s.nb; ++b) {
    int cnt = 0;
    for (int k = 0; k < s.ne; ++k) {
      if (s.eb[k] != b) continue;
      if (s.dim == 2) {
        const double *a = s.x + 2 * s.e[2 * k], *c = s.x + 2 * s.e[2 * k + 1];
        // the ray runs towards +x and +y: an element entirely behind the node
        // in either coordinate cannot cross it (exact test, no rounding)
        if ((a[0] < p[0] && c[0] < p[0]) || (a[1] < p[1] && c[1] < p[1])) continue;
        cnt += seg_ray_cross(p, c_ray2, a, c);
      } else {
        const double *a = s.x + 3 * s.e[3 * k], *c = s.x + 3 * s.e[3 * k + 1],
                     *e = s.x + 3 * s.e[3 * k + 2];
        if ((a[0] < p[0] && c[0] < p[0] && e[0] < p[0]) ||
            (a[1] < p[1] && c[1] < p[1] && e[1] < p[1]) ||
            (a[2] < p[2] && c[2] < p[2] && e[2] < p[2]))
          continue;
        double t, u, v;
        if (tri_ray(p, c_ray3, s.x + 3 * s.e[3 * k], s.x + 3 * s.e[3 * k + 1],
                    s.x + 3 * s.e[3 * k + 2], t, u, v) &&
            t > 0.0 && u >= 0.0 && v >= 0.0 && u + v < 1.0)
          cnt++;
      }
    }
    if (cnt & 1) return true;
  }
  return false;
}

// ---- FP32 filters over staged 2-D elements.  Every decision above is taken
// in FP64; these filters only skip elements whose FP64 test cannot pass,
// judged in FP32 with a margin T far above the FP32 rounding of the
// endpoints and of the products (about 4e-7 of the coordinates), so the
// filtered and unfiltered paths give identical flags and links.
constexpr int kStageSeg = 1024;

struct SegStage {
  union {
    float4 seg[kStageSeg];        // 2-D: (ax, ay, bx, by) rounded to FP32
    float tri[kStageSeg][9];      // 3-D: (a, b, c) rounded to FP32
  };
  unsigned char body[kStageSeg];
  float wbox[8][6];  // per-warp bounding boxes of the staged vertices (lo xyz, hi xyz)
};

// Stage the elements of the surface (all threads of the CTA, at most 256;
// the caller synchronises).  Returns false when the surface is too large.
__device__ bool stage_segments(const SurfaceDev &s, SegStage &st) {
  if (s.ne > kStageSeg) return false;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int k = threadIdx.x; k < s.ne; k += blockDim.x) {
    if (s.dim == 2) {
      const double *a = s.x + 2 * s.e[2 * k], *b = s.x + 2 * s.e[2 * k + 1];
      st.seg[k] = make_float4((float)a[0], (float)a[1], (float)b[0], (float)b[1]);
      for (int q = 0; q < 2; ++q) {
        lo[q] = fminf(lo[q], fminf((float)a[q], (float)b[q]));
        hi[q] = fmaxf(hi[q], fmaxf((float)a[q], (float)b[q]));
      }
      lo[2] = hi[2] = 0.5f;
    } else {
      for (int m = 0; m < 3; ++m) {
        const double *v = s.x + 3 * s.e[3 * k + m];
        for (int q = 0; q < 3; ++q) {
          const float c = (float)v[q];
          st.tri[k][3 * m + q] = c;
          lo[q] = fminf(lo[q], c);
          hi[q] = fmaxf(hi[q], c);
        }
      }
    }
    st.body[k] = (unsigned char)s.eb[k];
  }
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  if ((threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < 8)
    for (int q = 0; q < 3; ++q) {
      st.wbox[threadIdx.x >> 5][q] = lo[q];
      st.wbox[threadIdx.x >> 5][3 + q] = hi[q];
    }
  return true;
}

// Whether node p lies outside the staged surface's bounding box by a margin
// far above the FP32 rounding of the vertices: then it is neither inside a
// body nor on the surface.
__device__ __forceinline__ bool outside_staged_box(const SegStage &st, const double *p, int dim) {
  const int nw = min((int)(blockDim.x >> 5), 8);
  for (int q = 0; q < dim; ++q) {
    float lo = 3e38f, hi = -3e38f;
    for (int w = 0; w < nw; ++w) {
      lo = fminf(lo, st.wbox[w][q]);
      hi = fmaxf(hi, st.wbox[w][3 + q]);
    }
    const float pq = (float)p[q];
    if (pq < lo - 1e-5f * (1.f + fabsf(pq) + fabsf(lo)) ||
        pq > hi + 1e-5f * (1.f + fabsf(pq) + fabsf(hi)))
      return true;
  }
  return false;
}

__device__ __forceinline__ float seg_margin(const float4 &q, float px, float py) {
  return 4e-6f * (1.f + fabsf(px) + fabsf(py) + fabsf(q.x) + fabsf(q.y) + fabsf(q.z) + fabsf(q.w));
}

// inside_any for a 2-D surface through the staged filters.
// Segment k of the staged 2-D surface against node p: whether p lies on
// it (FP64 test behind an FP32 filter) and whether the parity ray from p
// crosses it.
__device__ __forceinline__ void seg_test(const SurfaceDev &s, const SegStage &st, int k,
                                         const double *p, float px, float py, float dx, float dy,
                                         bool &on, bool &cross) {
  const double tol = 1e-12;
  on = false;
  cross = false;
  const float4 q = st.seg[k];
  const float T = seg_margin(q, px, py);
  const float xlo = fminf(q.x, q.z), xhi = fmaxf(q.x, q.z);
  const float ylo = fminf(q.y, q.w), yhi = fmaxf(q.y, q.w);
  const bool near = px >= xlo - T && px <= xhi + T && py >= ylo - T && py <= yhi + T;
  if (near) {  // on-surface test (as in on_surface)
    const double *a = s.x + 2 * s.e[2 * k], *b = s.x + 2 * s.e[2 * k + 1];
    const double ex = b[0] - a[0], ey = b[1] - a[1];
    const double qx = p[0] - a[0], qy = p[1] - a[1];
    const double len2 = ex * ex + ey * ey;
    const double cr = ex * qy - ey * qx, dt = ex * qx + ey * qy;
    if (len2 > 0.0 && fabs(cr) <= tol * sqrt(len2) && dt >= 0.0 && dt <= len2) {
      on = true;
      return;
    }
  }
  if (xhi < px - T || yhi < py - T) return;  // behind the node in x or y
  const float sa = dx * (q.y - py) - dy * (q.x - px);
  const float sb = dx * (q.w - py) - dy * (q.z - px);
  if ((sa > T && sb > T) || (sa < -T && sb < -T)) return;  // off the ray's line
  const double *a = s.x + 2 * s.e[2 * k], *b = s.x + 2 * s.e[2 * k + 1];
  if ((a[0] < p[0] && b[0] < p[0]) || (a[1] < p[1] && b[1] < p[1])) return;
  cross = seg_ray_cross(p, c_ray2, a, b);
}

__device__ bool inside_any_staged(const SurfaceDev &s, const SegStage &st, const double *p) {
  const float px = (float)p[0], py = (float)p[1];
  const float dx = (float)c_ray2[0], dy = (float)c_ray2[1];
  unsigned par = 0;
  for (int k = 0; k < s.ne; ++k) {
    bool on, cross;
    seg_test(s, st, k, p, px, py, dx, dy, on, cross);
    if (on) return true;
    if (cross) par ^= 1u << st.body[k];
  }
  return par != 0;
}

// Triple product d . ((A - p) x (B - p)) in FP32 and a bound far above its
// rounding error (the Pluecker side of the ray's line against edge A-B).
__device__ __forceinline__ float edge_side(const float *A, const float *B, const float *p,
                                           const float *d, float mag, float &bound) {
  const float a0 = A[0] - p[0], a1 = A[1] - p[1], a2 = A[2] - p[2];
  const float b0 = B[0] - p[0], b1 = B[1] - p[1], b2 = B[2] - p[2];
  const float S = fabsf(a0) + fabsf(a1) + fabsf(a2) + fabsf(b0) + fabsf(b1) + fabsf(b2);
  bound = 2e-6f * (mag + S) * (1.f + S);
  return d[0] * (a1 * b2 - a2 * b1) + d[1] * (a2 * b0 - a0 * b2) + d[2] * (a0 * b1 - a1 * b0);
}

// inside_any for a 3-D surface through the staged filters: a triangle is
// skipped when the node is off its bounding box (on-surface test), when it
// lies behind the node on an axis, or when two of its edges put the ray's
// line on strictly opposite sides (the line misses it).
// Triangle k of the staged 3-D surface against node p (as seg_test).
__device__ __forceinline__ void tri_test(const SurfaceDev &s, const SegStage &st, int k,
                                         const double *p, const float *pf, const float *d,
                                         bool &on, bool &cross) {
  on = false;
  cross = false;
  const float *t = st.tri[k];
  float mag = 1.f + fabsf(pf[0]) + fabsf(pf[1]) + fabsf(pf[2]);
  for (int q = 0; q < 9; ++q) mag += fabsf(t[q]);
  const float T = 4e-6f * mag;
  bool near = true, behind = false;
  for (int q = 0; q < 3; ++q) {
    const float lo = fminf(fminf(t[q], t[3 + q]), t[6 + q]);
    const float hi = fmaxf(fmaxf(t[q], t[3 + q]), t[6 + q]);
    near = near && pf[q] >= lo - T && pf[q] <= hi + T;
    behind = behind || hi < pf[q] - T;
  }
  const double *a = s.x + 3 * s.e[3 * k], *b = s.x + 3 * s.e[3 * k + 1], *c = s.x + 3 * s.e[3 * k + 2];
  if (near && on_triangle(p, a, b, c, 1e-12)) {
    on = true;
    return;
  }
  if (behind) return;
  float b0, b1, b2;
  const float s0 = edge_side(t, t + 3, pf, d, mag, b0);
  const float s1 = edge_side(t + 3, t + 6, pf, d, mag, b1);
  const float s2 = edge_side(t + 6, t, pf, d, mag, b2);
  const bool pos = s0 > b0 || s1 > b1 || s2 > b2, neg = s0 < -b0 || s1 < -b1 || s2 < -b2;
  if (pos && neg) return;
  if ((a[0] < p[0] && b[0] < p[0] && c[0] < p[0]) || (a[1] < p[1] && b[1] < p[1] && c[1] < p[1]) ||
      (a[2] < p[2] && b[2] < p[2] && c[2] < p[2]))
    return;
  double tt, u, v;
  cross = tri_ray(p, c_ray3, a, b, c, tt, u, v) && tt > 0.0 && u >= 0.0 && v >= 0.0 && u + v < 1.0;
}

__device__ bool inside_any_staged3(const SurfaceDev &s, const SegStage &st, const double *p) {
  const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
  const float d[3] = {(float)c_ray3[0], (float)c_ray3[1], (float)c_ray3[2]};
  unsigned par = 0;
  for (int k = 0; k < s.ne; ++k) {
    bool on, cross;
    tri_test(s, st, k, p, pf, d, on, cross);
    if (on) return true;
    if (cross) par ^= 1u << st.body[k];
  }
  return par != 0;
}

// Whether band node p is inside a body or on the surface, with the warp's
// lanes splitting the staged elements (on-surface: any lane; parity: XOR of
// the lanes' per-body crossing masks).  All lanes call it with the same p.
__device__ bool inside_any_warp(const SurfaceDev &s, const SegStage &st, const double *p,
                                int lane) {
  bool on_any = false;
  unsigned par = 0;
  if (s.dim == 2) {
    const float px = (float)p[0], py = (float)p[1];
    const float dx = (float)c_ray2[0], dy = (float)c_ray2[1];
    for (int k = lane; k < s.ne; k += 32) {
      bool on, cross;
      seg_test(s, st, k, p, px, py, dx, dy, on, cross);
      on_any = on_any || on;
      if (!on && cross) par ^= 1u << st.body[k];
    }
  } else {
    const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
    const float d[3] = {(float)c_ray3[0], (float)c_ray3[1], (float)c_ray3[2]};
    for (int k = lane; k < s.ne; k += 32) {
      bool on, cross;
      tri_test(s, st, k, p, pf, d, on, cross);
      on_any = on_any || on;
      if (!on && cross) par ^= 1u << st.body[k];
    }
  }
  if (__any_sync(0xffffffffu, on_any)) return true;
  return __reduce_xor_sync(0xffffffffu, par) != 0;
}

// ---- cut links.  The link from x_b along -c_i has the box [lo, hi] (with
// the crossing tolerance); link_may_hit is the exact FP32 prefilter of an
// element against it, link_crossing the FP64 test (parameter sp in
// (eps, 1 + eps] along the link, barycentric weights bw), link_finish fills
// the Link from the nearest crossing.
__device__ __forceinline__ void link_box(const double *xb, const double *d, double *lo, double *hi) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = fmin(xb[a], xb[a] + d[a]) - 1e-6;
    hi[a] = fmax(xb[a], xb[a] + d[a]) + 1e-6;
  }
}

__device__ __forceinline__ bool link_may_hit(const SurfaceDev &s, const SegStage *st, int k,
                                             const double *lo, const double *hi) {
  if (!st) return true;
  if (s.dim == 2) {
    const float4 q = st->seg[k];
    const float flo0 = (float)lo[0], fhi0 = (float)hi[0], flo1 = (float)lo[1], fhi1 = (float)hi[1];
    const float T = seg_margin(q, flo0, flo1);
    return !(fmaxf(q.x, q.z) < flo0 - T || fminf(q.x, q.z) > fhi0 + T ||
             fmaxf(q.y, q.w) < flo1 - T || fminf(q.y, q.w) > fhi1 + T);
  }
  const float *t = st->tri[k];
  float mag = 1.f + fabsf((float)lo[0]) + fabsf((float)lo[1]) + fabsf((float)lo[2]);
  for (int q = 0; q < 9; ++q) mag += fabsf(t[q]);
  const float T = 4e-6f * mag;
  for (int q = 0; q < 3; ++q)
    if (fmaxf(fmaxf(t[q], t[3 + q]), t[6 + q]) < (float)lo[q] - T ||
        fminf(fminf(t[q], t[3 + q]), t[6 + q]) > (float)hi[q] + T)
      return false;
  return true;
}

__device__ bool link_crossing(const SurfaceDev &s, const double *xb, const double *d,
                              const double *lo, const double *hi, int k, double &sp, double *bw) {
  const double eps = 1e-9;
  if (s.dim == 2) {
    const double *a = s.x + 2 * s.e[2 * k], *b = s.x + 2 * s.e[2 * k + 1];
    if (fmax(a[0], b[0]) < lo[0] || fmin(a[0], b[0]) > hi[0] || fmax(a[1], b[1]) < lo[1] ||
        fmin(a[1], b[1]) > hi[1])
      return false;
    const double ex = b[0] - a[0], ey = b[1] - a[1];
    const double den = d[0] * (-ey) - d[1] * (-ex);
    if (fabs(den) < 1e-300) return false;
    const double rx = a[0] - xb[0], ry = a[1] - xb[1];
    sp = (rx * (-ey) - ry * (-ex)) / den;
    const double t = (d[0] * ry - d[1] * rx) / den;
    if (!(sp > eps && sp <= 1.0 + eps && t >= -eps && t <= 1.0 + eps)) return false;
    const double tt = t < 0 ? 0 : (t > 1 ? 1 : t);
    bw[0] = 1.0 - tt; bw[1] = tt; bw[2] = 0.0;
    return true;
  }
  const double *a = s.x + 3 * s.e[3 * k], *b = s.x + 3 * s.e[3 * k + 1], *c = s.x + 3 * s.e[3 * k + 2];
  bool out = false;
  for (int q = 0; q < 3; ++q)
    out |= fmax(fmax(a[q], b[q]), c[q]) < lo[q] || fmin(fmin(a[q], b[q]), c[q]) > hi[q];
  if (out) return false;
  double u, v;
  if (!tri_ray(xb, d, a, b, c, sp, u, v)) return false;
  if (!(sp > eps && sp <= 1.0 + eps && u >= -eps && v >= -eps && u + v <= 1.0 + eps)) return false;
  bw[0] = 1.0 - u - v; bw[1] = u; bw[2] = v;
  return true;
}

__device__ void link_finish(const SurfaceDev &s, int best, double bs, const double *bw, Link &L) {
  L.uw[0] = L.uw[1] = L.uw[2] = 0.f;
  L.v[0] = L.v[1] = L.v[2] = 0;
  L.vw[0] = L.vw[1] = L.vw[2] = 0.f;
  if (best < 0) {  // no crossing found: a wall half-way at rest, no force
    L.q = 0.5f;
    L.body = -1;
    return;
  }
  L.q = (float)(bs > 1.0 ? 1.0 : bs);
  L.body = s.eb[best];
  double uw[3] = {0, 0, 0};
  for (int m = 0; m < s.dim; ++m) {
    const int vid = s.e[s.dim * best + m];
    L.v[m] = vid;
    L.vw[m] = (float)bw[m];
    for (int a = 0; a < s.dim; ++a) uw[a] += bw[m] * s.v[s.dim * vid + a];
  }
  for (int a = 0; a < 3; ++a) L.uw[a] = (float)uw[a];
}

// Bounding box of the surface vertices (one CTA), rounded to FP32.
__device__ __forceinline__ void surface_box_body(const SurfaceDev &s) {
  __shared__ float red[6][8];
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int v = threadIdx.x; v < s.nv; v += blockDim.x)
    for (int q = 0; q < s.dim; ++q) {
      const float c = (float)s.x[s.dim * v + q];
      lo[q] = fminf(lo[q], c);
      hi[q] = fmaxf(hi[q], c);
    }
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) {
      red[q][w] = lo[q];
      red[3 + q][w] = hi[q];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const bool is_lo = threadIdx.x < 3;
    float v = is_lo ? 3e38f : -3e38f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
      v = is_lo ? fminf(v, red[threadIdx.x][k]) : fmaxf(v, red[threadIdx.x][k]);
    s.box[threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256) k_surface_box(SurfaceDev s) { surface_box_body(s); }

// Whether node p lies outside box by a margin far above the FP32 rounding of
// the box: then it is neither inside a body nor on the surface.
__device__ __forceinline__ bool outside_box(const float *box, const double *p, int dim) {
  for (int q = 0; q < dim; ++q) {
    const float pq = (float)p[q], lo = box[q], hi = box[3 + q];
    if (pq < lo - 1e-5f * (1.f + fabsf(pq) + fabsf(lo)) || pq > hi + 1e-5f * (1.f + fabsf(pq) + fabsf(hi)))
      return true;
  }
  return false;
}

// New solid flags inside the band; nodes that turn fluid are listed as fresh.
// Flag update of band node t (shared by the node pass and the deferred
// warp pass): solid or fluid, and a solid -> fluid change recorded as fresh.
__device__ __forceinline__ void set_solid_flag(uint8_t *flags, long long k, bool in, int64_t *fresh,
                                               int *nfresh, int cap, int track_fresh) {
  const uint8_t now = in ? NODE_SOLID : NODE_FLUID;
  const uint8_t before = flags[k];
  if (before == NODE_GHOST) return;
  if (track_fresh && before == NODE_SOLID && now == NODE_FLUID) {
    const int slot = atomicAdd(nfresh, 1);
    if (slot < cap) fresh[slot] = k;
  }
  flags[k] = now;
}

__device__ __forceinline__ void band_node(const Band &bd, long long t, int &x, int &y, int &z) {
  const int bx = bd.x1 - bd.x0, by = bd.y1 - bd.y0;
  x = bd.x0 + (int)(t % bx);
  y = bd.y0 + (int)((t / bx) % by);
  z = bd.z0 + (int)(t / ((long long)bx * by));
}

// Solid flags of the band.  Nodes inside the staged surface's box, where
// every element has to be tested, are deferred to the warp pass
// (solid_near_body) through near_list / near_cnt when a list is given and
// has room; the rest are decided here.
__device__ __forceinline__ void solid_flags_body(long long t, const Grid &g, const Band &bd,
                                                 const SurfaceDev &s, uint8_t *flags,
                                                 int64_t *fresh, int *nfresh, int cap,
                                                 int track_fresh, int *near_list = nullptr,
                                                 int *near_cnt = nullptr, int near_cap = 0) {
  __shared__ SegStage st;
  const int bx = bd.x1 - bd.x0, by = bd.y1 - bd.y0, bz = bd.z1 - bd.z0;
  const long long nbnd = (long long)bx * by * bz;
  if ((long long)(t - threadIdx.x) >= nbnd) return;  // whole CTA past the band
  const bool live = t < nbnd;
  const long long tt = live ? t : nbnd - 1;
  const int x = bd.x0 + (int)(tt % bx), y = bd.y0 + (int)((tt / bx) % by),
            z = bd.z0 + (int)(tt / ((long long)bx * by));
  const double p[3] = {x + 0.5, y + 0.5, z + 0.5};  // cell-centred node position
  const long long k = sidx(g, x + g.px, y + g.py, z + g.pz);
  // a CTA whose nodes all lie outside the surface's box needs no element tests
  const bool far = s.box && outside_box(s.box, p, s.dim);
  const bool all_far = s.box ? __syncthreads_and(far) != 0 : false;
  bool staged = false;
  if (!all_far) {
    staged = stage_segments(s, st);
    __syncthreads();
  }
  if (!live) return;
  bool in;
  if (far) {
    in = false;
  } else if (staged) {
    if (outside_staged_box(st, p, s.dim)) {
      in = false;
    } else {
      if (near_list) {
        const int slot = atomicAdd(near_cnt, 1);
        if (slot < near_cap) {
          near_list[slot] = (int)tt;
          return;
        }
      }
      in = s.dim == 2 ? inside_any_staged(s, st, p) : inside_any_staged3(s, st, p);
    }
  } else {
    in = inside_any(s, p);
  }
  set_solid_flag(flags, k, in, fresh, nfresh, cap, track_fresh);
}

// Deferred band nodes, one warp each (warp w of nw takes list entries w,
// w + nw, ...): the lanes split the surface elements.
__device__ __forceinline__ void solid_near_body(const Grid &g, const Band &bd, const SurfaceDev &s,
                                                uint8_t *flags, int64_t *fresh, int *nfresh,
                                                int cap, int track_fresh, const int *near_list,
                                                const int *near_cnt, int near_cap, int w, int nw) {
  __shared__ SegStage st;
  int n = *near_cnt;
  if (n > near_cap) n = near_cap;
  if ((int)(blockIdx.x * (blockDim.x >> 5)) >= n) return;  // whole CTA idle
  if (!stage_segments(s, st)) return;  // nodes are only deferred when staging fits
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int j = w; j < n; j += nw) {
    int x, y, z;
    band_node(bd, near_list[j], x, y, z);
    const double p[3] = {x + 0.5, y + 0.5, z + 0.5};
    const bool in = inside_any_warp(s, st, p, lane);
    if (lane == 0)
      set_solid_flag(flags, sidx(g, x + g.px, y + g.py, z + g.pz), in, fresh, nfresh, cap,
                     track_fresh);
  }
}

__global__ void k_solid_flags(Grid g, Band bd, SurfaceDev s, uint8_t *flags, int64_t *fresh,
                              int *nfresh, int cap, int track_fresh, int *near_list,
                              int *near_cnt, int near_cap) {
  solid_flags_body(blockIdx.x * (long long)blockDim.x + threadIdx.x, g, bd, s, flags, fresh,
                   nfresh, cap, track_fresh, near_list, near_cnt, near_cap);
}

__global__ void __launch_bounds__(128)
    k_solid_near(Grid g, Band bd, SurfaceDev s, uint8_t *flags, int64_t *fresh, int *nfresh,
                 int cap, int track_fresh, const int *near_list, const int *near_cnt,
                 int near_cap) {
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  solid_near_body(g, bd, s, flags, fresh, nfresh, cap, track_fresh, near_list, near_cnt, near_cap,
                  w, nw);
}

// Immersed boundary nodes of the band: slots in the node list and ranges in
// the link list (the links themselves: link_fill_body).
template <int Q>
__device__ __forceinline__ void build_links_body(long long t, const Grid &g, const Band &bd,
                                                 const SurfaceDev &s, const uint8_t *flags,
                                                 BNode *bnodes, int *nbn, int bcap, Link *links,
                                                 int *nl, int lcap, int *err) {
  using L = Lat<Q>;
  const int bx = bd.x1 - bd.x0, by = bd.y1 - bd.y0, bz = bd.z1 - bd.z0;
  const long long nbnd = (long long)bx * by * bz;
  if (t >= nbnd) return;
  const int x = bd.x0 + (int)(t % bx), y = bd.y0 + (int)((t / bx) % by),
            z = bd.z0 + (int)(t / ((long long)bx * by));
  const int X = x + g.px, Y = y + g.py, Z = z + g.pz;
  const long long k = sidx(g, X, Y, Z);
  if (flags[k] != NODE_FLUID) return;
  uint32_t mask = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int Xs = nbr(X, -L::cx(i), g.NX), Ys = nbr(Y, -L::cy(i), g.NY),
              Zs = (L::D == 3) ? nbr(Z, -L::cz(i), g.NZ) : Z;
    if (flags[sidx(g, Xs, Ys, Zs)] == NODE_SOLID) mask |= 1u << i;
  }
  if (!mask) return;
  const int n = __popc(mask);
  const int l0 = atomicAdd(nl, n);
  const int slot = atomicAdd(nbn, 1);
  if (slot >= bcap) {
    atomicOr(err, 4);  // capacity overflow: the node is left out
    return;
  }
  if (l0 + n > lcap) {
    // no room for its links: keep the node (walls half-way at rest, no force)
    atomicOr(err, 4);
    bnodes[slot] = BNode{k, -1, 0};
    return;
  }
  bnodes[slot] = BNode{k, l0, n};  // its links follow in link_fill_body
}

// Cut links of the listed boundary nodes: one warp per node (grid-stride
// over the list).  The lanes prefilter the surface elements of all the
// node's links in FP32 and compact the candidates (link, element); the FP64
// crossing tests then run one candidate per lane, and each link keeps its
// nearest crossing (ties: the lower element index, as in the serial scan).
constexpr int kLinkCand = 64;

struct LinkScratch {
  short cm[kLinkCand], ck[kLinkCand];
  double csp[kLinkCand];
  double bsp[27];
  int bk[27];
  int dir[27];
};

__device__ __forceinline__ void link_dir(int Q, int i, double *d) {
  if (Q == 9) {
    d[0] = -(double)(i % 3 - 1); d[1] = -(double)(i / 3 - 1); d[2] = 0.0;
  } else {
    d[0] = -(double)(i % 3 - 1); d[1] = -(double)((i / 3) % 3 - 1); d[2] = -(double)(i / 9 - 1);
  }
}

template <int Q>
__device__ __forceinline__ void link_flush(const SurfaceDev &s, const double *xb, LinkScratch &S,
                                           int count, int nm, int lane) {
  __syncwarp();
  for (int j = lane; j < count; j += 32) {
    double d[3], lo[3], hi[3], sp, w[3];
    link_dir(Q, S.dir[S.cm[j]], d);
    link_box(xb, d, lo, hi);
    S.csp[j] = link_crossing(s, xb, d, lo, hi, S.ck[j], sp, w) ? sp : 4.0;
  }
  __syncwarp();
  if (lane < nm) {
    for (int j = 0; j < count; ++j) {
      if (S.cm[j] != lane || S.csp[j] > 3.0) continue;
      const double sp = S.csp[j];
      const int k = S.ck[j];
      if (sp < S.bsp[lane] || (sp == S.bsp[lane] && k < S.bk[lane])) {
        S.bsp[lane] = sp;
        S.bk[lane] = k;
      }
    }
  }
  __syncwarp();
}

template <int Q>
__device__ __forceinline__ void link_fill_body(const Grid &g, const SurfaceDev &s,
                                               const uint8_t *flags, const BNode *bnodes,
                                               const int *nbn, int bcap, Link *links, int warp0,
                                               int nwarps) {
  using L = Lat<Q>;
  __shared__ SegStage st;
  __shared__ LinkScratch scratch[4];
  const bool staged = stage_segments(s, st);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  LinkScratch &S = scratch[(threadIdx.x >> 5) & 3];
  const int n = *nbn < bcap ? *nbn : bcap;
  for (int w = warp0; w < n; w += nwarps) {
    const BNode b = bnodes[w];
    if (b.nlink <= 0) continue;
    int X, Y, Z;
    decompose(g, b.k, X, Y, Z);
    const double xb[3] = {X - g.px + 0.5, Y - g.py + 0.5, Z - g.pz + 0.5};
    // the node's missing directions, in direction order
    bool solid = false;
    if (lane < Q) {
      const int Xs = nbr(X, -L::cx(lane), g.NX), Ys = nbr(Y, -L::cy(lane), g.NY),
                Zs = (L::D == 3) ? nbr(Z, -L::cz(lane), g.NZ) : Z;
      solid = flags[sidx(g, Xs, Ys, Zs)] == NODE_SOLID;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, solid);
    const int nm = __popc(mask);
    if (solid) {
      const int m = __popc(mask & ((1u << lane) - 1u));
      S.dir[m] = lane;
      S.bsp[m] = 2.0;
      S.bk[m] = -1;
    }
    __syncwarp();
    if (!staged) {
      // large surfaces: the lanes split the elements of each link in turn
      for (int m = 0; m < nm; ++m) {
        double d[3], lo[3], hi[3];
        link_dir(Q, S.dir[m], d);
        link_box(xb, d, lo, hi);
        double bs = 2.0;
        int best = -1;
        for (int k = lane; k < s.ne; k += 32) {
          double sp, wv[3];
          if (link_crossing(s, xb, d, lo, hi, k, sp, wv) && sp < bs) {
            bs = sp;
            best = k;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double obs = __shfl_xor_sync(0xffffffffu, bs, o);
          const int ob = __shfl_xor_sync(0xffffffffu, best, o);
          if (ob >= 0 && (best < 0 || obs < bs || (obs == bs && ob < best))) {
            bs = obs;
            best = ob;
          }
        }
        if (lane == 0) {
          S.bsp[m] = bs;
          S.bk[m] = best;
        }
        __syncwarp();
      }
    } else {
      int count = 0;
      for (int m = 0; m < nm; ++m) {
        double d[3], lo[3], hi[3];
        link_dir(Q, S.dir[m], d);
        link_box(xb, d, lo, hi);
        for (int k0 = 0; k0 < s.ne; k0 += 32) {
          const int k = k0 + lane;
          const bool pass = k < s.ne && link_may_hit(s, &st, k, lo, hi);
          const unsigned pm = __ballot_sync(0xffffffffu, pass);
          if (pass) {
            const int pos = count + __popc(pm & ((1u << lane) - 1u));
            S.cm[pos] = (short)m;
            S.ck[pos] = (short)k;
          }
          count += __popc(pm);
          if (count > kLinkCand - 32) {
            link_flush<Q>(s, xb, S, count, nm, lane);
            count = 0;
          }
        }
      }
      link_flush<Q>(s, xb, S, count, nm, lane);
    }
    if (lane < nm) {
      Link lk;
      lk.i = S.dir[lane];
      double d[3], lo[3], hi[3], sp = 2.0, bw[3] = {0, 0, 0};
      const int best = S.bk[lane];
      if (best >= 0) {
        link_dir(Q, S.dir[lane], d);
        link_box(xb, d, lo, hi);
        link_crossing(s, xb, d, lo, hi, best, sp, bw);
      }
      link_finish(s, best, sp, bw, lk);
      links[b.link0 + lane] = lk;
    }
    __syncwarp();
  }
}

template <int Q>
__global__ void __launch_bounds__(128) k_link_fill(Grid g, SurfaceDev s, const uint8_t *flags,
                                                   const BNode *bnodes, const int *nbn, int bcap,
                                                   Link *links) {
  link_fill_body<Q>(g, s, flags, bnodes, nbn, bcap, links,
                    (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
                    (int)((gridDim.x * blockDim.x) >> 5));
}

template <int Q>
__global__ void k_build_links(Grid g, Band bd, SurfaceDev s, const uint8_t *flags, BNode *bnodes,
                              int *nbn, int bcap, Link *links, int *nl, int lcap, int *err) {
  build_links_body<Q>(blockIdx.x * (long long)blockDim.x + threadIdx.x, g, bd, s, flags, bnodes,
                      nbn, bcap, links, nl, lcap, err);
}

// Fresh nodes (solid -> fluid): f = feq(mean rho of fluid non-fresh neighbours,
// velocity of the nearest surface vertex).
template <int Q, int S>
__device__ __forceinline__ void fresh_init_body(int t, const Grid &g, typename Store<S>::T *f,
                                                const uint8_t *flags, const int64_t *fresh,
                                                const int *nfresh, int cap, const SurfaceDev &s) {
  using L = Lat<Q>;
  const int nf = *nfresh < cap ? *nfresh : cap;
  if (t >= nf) return;
  const long long k = fresh[t];
  int X, Y, Z;
  decompose(g, k, X, Y, Z);
  double rsum = 0.0;
  int rn = 0;
  for (int i = 0; i < Q; ++i) {
    if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
    const int Xn = step_axis(X, L::cx(i), g.NX, g.px), Yn = step_axis(Y, L::cy(i), g.NY, g.py);
    const int Zn = (L::D == 3) ? step_axis(Z, L::cz(i), g.NZ, g.pz) : Z;
    if (Xn < 0 || Yn < 0 || Zn < 0) continue;
    const long long kn = sidx(g, Xn, Yn, Zn);
    if (flags[kn] != NODE_FLUID) continue;
    bool is_fresh = false;
    for (int m = 0; m < nf; ++m)
      if (fresh[m] == kn) { is_fresh = true; break; }
    if (is_fresh) continue;
    float dr, j[3];
    dev_moments<Q, S>(g, f, kn, dr, j);
    rsum += 1.0 + (double)dr;
    rn++;
  }
  const double rho = rn ? rsum / rn : 1.0;
  const double p[3] = {X - g.px + 0.5, Y - g.py + 0.5, Z - g.pz + 0.5};
  int best = 0;
  double bd = 1e300;
  for (int v = 0; v < s.nv; ++v) {
    double d2 = 0;
    for (int a = 0; a < s.dim; ++a) {
      const double dd = s.x[s.dim * v + a] - p[a];
      d2 += dd * dd;
    }
    if (d2 < bd) { bd = d2; best = v; }
  }
  double u[3] = {0, 0, 0};
  for (int a = 0; a < s.dim; ++a) u[a] = s.v[s.dim * best + a];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double p_eq = rho;
    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
    for (int a = 0; a < L::D; ++a) {
      const double Sa = sqrt(1.0 + 3.0 * u[a] * u[a]);
      double fa = w1d(c[a]) * (2.0 - Sa);
      if (c[a] == 1) fa *= (2.0 * u[a] + Sa) / (1.0 - u[a]);
      if (c[a] == -1) fa *= (Sa - 2.0 * u[a]) / (1.0 + u[a]);
      p_eq *= fa;
    }
    const double w = weight<L>(i);
    f[(long long)i * g.N + k] = Store<S>::encode(p_eq - w, w);
  }
}

template <int Q, int S>
__global__ void k_fresh_init(Grid g, typename Store<S>::T *f, const uint8_t *flags,
                             const int64_t *fresh, const int *nfresh, int cap, SurfaceDev s) {
  fresh_init_body<Q, S>(blockIdx.x * blockDim.x + threadIdx.x, g, f, flags, fresh, nfresh, cap, s);
}

// ---------------------------------------------------------------- Grad fill + force
// Per-body force totals of a warp: reduction per body id, one atomic per warp
// and body (all lanes call it).
__device__ __forceinline__ void body_reduce(int nbodies, int my_body, const double (&Fd)[3],
                                            double *bforce) {
  for (int b = 0; b < nbodies; ++b) {
    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = (my_body == b) ? Fd[a] : 0.0;
    const unsigned any = __ballot_sync(0xffffffffu, my_body == b);
    if (!any) continue;
    for (int off = 16; off > 0; off >>= 1)
      for (int a = 0; a < 3; ++a) v[a] += __shfl_down_sync(0xffffffffu, v[a], off);
    if ((threadIdx.x & 31) == 0)
      for (int a = 0; a < 3; ++a) atomicAdd(&bforce[3 * b + a], v[a]);
  }
}

template <int Q, int S, typename R>
__device__ __forceinline__ void grad_body(int tb, const Grid &g, typename Store<S>::T *f,
                                          const uint8_t *__restrict__ flags,
                                          const BNode *__restrict__ bnodes,
                                          const int *__restrict__ nbn, int nfixed, int cap,
                                          int first, int last, const Link *__restrict__ links,
                                          const BoundaryParams &bp, double *vforce,
                                          double *bforce, int nbodies) {
  using L = Lat<Q>;
  using St = Store<S>;
  constexpr int D = L::D;
  // threads [0, nfixed) take the face nodes, the rest the immersed nodes
  const int t = tb + first;
  int dyn = nbn ? *nbn : 0;
  if (dyn > cap - nfixed) dyn = cap - nfixed;
  const int count = last < 0 ? nfixed + dyn : last;
  const bool active = t < count;
  int my_body = -1;
  double Fd[3] = {0, 0, 0};
  if (active) {
    const BNode bn = bnodes[t];
    const long long k = bn.k;
    int X, Y, Z;
    decompose(g, k, X, Y, Z);
    long long src[Q];
    int face_of[Q];
    uint32_t miss = 0, solid_miss = 0;
    typename St::C gk[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int Xs = nbr(X, -L::cx(i), g.NX), Ys = nbr(Y, -L::cy(i), g.NY),
                Zs = (L::D == 3) ? nbr(Z, -L::cz(i), g.NZ) : Z;
      src[i] = sidx(g, Xs, Ys, Zs);
      const uint8_t fl = flags[src[i]];
      face_of[i] = -1;
      gk[i] = 0;
      if (fl == NODE_FLUID) {
        gk[i] = St::load(f + (long long)i * g.N + src[i], (typename St::C)weight<L>(i));
      } else {
        miss |= 1u << i;
        if (fl == NODE_SOLID) solid_miss |= 1u << i;
        if (fl == NODE_GHOST) {
          if (g.px && (Xs == 0 || Xs == g.NX - 1)) face_of[i] = Xs == 0 ? 0 : 1;
          else if (g.py && (Ys == 0 || Ys == g.NY - 1)) face_of[i] = Ys == 0 ? 2 : 3;
          else face_of[i] = Zs == 0 ? 4 : 5;
        }
      }
    }
    // a face node next to an immersed body would also be in the immersed
    // list, whose entry carries its cut links: that entry alone fills such a
    // node, since the face and immersed sets run in the same launch
    // (lbm_set_geometry keeps bodies two nodes inside non-periodic faces, so
    // this is a guard)
    if (t < nfixed && solid_miss) miss = 0;
    if (miss) {
      const int nmiss = __popc(miss);
      int open_face = -1;
      for (int fc = 0; fc < 6 && open_face < 0; ++fc)
        for (int i = 0; i < Q; ++i)
          if (((miss >> i) & 1u) && face_of[i] == fc &&
              (bp.bc[fc] == BCK_INLET || bp.bc[fc] == BCK_OUTLET ||
               bp.bc[fc] == BCK_FREESTREAM)) {
            open_face = fc;
            break;
          }
      R rho_t, ut[3] = {0, 0, 0};
      bool zero_grad = false;
      if (open_face >= 0) {
        const int ax = open_face / 2;
        int Xn = X, Yn = Y, Zn = Z;
        const int dir = (open_face % 2 == 0) ? 1 : -1;
        if (ax == 0) Xn = step_axis(X, dir, g.NX, g.px);
        if (ax == 1) Yn = step_axis(Y, dir, g.NY, g.py);
        if (ax == 2) Zn = step_axis(Z, dir, g.NZ, g.pz);
        long long kn = k;
        if (Xn >= 0 && Yn >= 0 && Zn >= 0 && flags[sidx(g, Xn, Yn, Zn)] == NODE_FLUID)
          kn = sidx(g, Xn, Yn, Zn);
        R u0[3], r0;
        dev_velocity<Q, S, R>(g, f, kn, u0, &r0);
        if (bp.bc[open_face] == BCK_INLET) {
          R scale = 1;
          if (bp.ramp_steps > 0 && bp.step) {
            const int st = *bp.step;
            if (st < bp.ramp_steps) scale = (R)0.5 * ((R)1 - cospi((double)st / bp.ramp_steps));
          }
          const float *prof = bp.inlet[open_face];
          const int x = X - g.px, y = Y - g.py, z = Z - g.pz;
          long long fidx, fn;
          if (ax == 0) { fidx = (long long)z * g.ny + y; fn = (long long)g.ny * g.nz; }
          else if (ax == 1) { fidx = (long long)z * g.nx + x; fn = (long long)g.nx * g.nz; }
          else { fidx = (long long)y * g.nx + x; fn = (long long)g.nx * g.ny; }
          for (int a = 0; a < D; ++a)
            ut[a] = scale * (R)(prof ? prof[a * fn + fidx] : bp.face_u[open_face][a]);
          rho_t = r0;
        } else if (bp.bc[open_face] == BCK_OUTLET) {
          for (int a = 0; a < D; ++a) ut[a] = u0[a];
          rho_t = 1;
        } else {
          for (int a = 0; a < D; ++a) ut[a] = bp.face_u[open_face][a];
          rho_t = 1;
          zero_grad = true;
        }
      } else {
        // known populations and the missing ones' opposites: PopSum; the
        // wall-velocity terms 6 W_i c_i.u_w: a separate sum in R
        PopSum<R> pops;
        R wterm = 0;
        for (int i = 0; i < Q; ++i) {
          if (!((miss >> i) & 1u)) {
            pops.add(gk[i]);
            continue;
          }
          R q = 0.5, uw[3] = {0, 0, 0};
          if (face_of[i] >= 0) {
            for (int a = 0; a < 3; ++a) uw[a] = bp.face_u[face_of[i]][a];
          } else {
            // immersed links of the node are stored in ascending direction order
            for (int l = 0; l < bn.nlink; ++l) {
              const Link &lk = links[bn.link0 + l];
              if (lk.i == i) {
                q = lk.q;
                for (int a = 0; a < 3; ++a) uw[a] = lk.uw[a];
                break;
              }
            }
          }
          const double wi = dir_tab<Q>().w[i];
          R cuw = L::cx(i) * uw[0] + L::cy(i) * uw[1];
          if (D == 3) cuw += L::cz(i) * uw[2];
          pops.add(St::load(f + (long long)(Q - 1 - i) * g.N + k,
                            (typename St::C)dir_tab<Q>().w[i]));
          wterm += (R)(6.0 * wi) * cuw;
          const int Xn = step_axis(X, L::cx(i), g.NX, g.px), Yn = step_axis(Y, L::cy(i), g.NY, g.py);
          const int Zn = (L::D == 3) ? step_axis(Z, L::cz(i), g.NZ, g.pz) : Z;
          R ui[3] = {uw[0], uw[1], uw[2]};
          if (Xn >= 0 && Yn >= 0 && Zn >= 0 && flags[sidx(g, Xn, Yn, Zn)] == NODE_FLUID) {
            R un[3];
            dev_velocity<Q, S, R>(g, f, sidx(g, Xn, Yn, Zn), un);
            const R iq = (R)1 / ((R)1 + q);
            for (int a = 0; a < D; ++a) ui[a] = (uw[a] + q * un[a]) * iq;
          }
          for (int a = 0; a < D; ++a) ut[a] += ui[a];
        }
        const R inm = (R)1 / (R)nmiss;
        for (int a = 0; a < D; ++a) ut[a] *= inm;
        rho_t = (R)1 + ((R)pops.value() + wterm);
      }
      // ---- velocity gradient G[a][b] = d u_a / d x_b (previous step)
      R G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      if (!zero_grad) {
        R u0[3];
        dev_velocity<Q, S, R>(g, f, k, u0);
        for (int b = 0; b < D; ++b) {
          int P1[3] = {X, Y, Z}, M1[3] = {X, Y, Z}, P2[3] = {X, Y, Z}, M2[3] = {X, Y, Z};
          const int NS = b == 0 ? g.NX : (b == 1 ? g.NY : g.NZ);
          const int pad = b == 0 ? g.px : (b == 1 ? g.py : g.pz);
          const int Sb = b == 0 ? X : (b == 1 ? Y : Z);
          P1[b] = step_axis(Sb, 1, NS, pad);
          M1[b] = step_axis(Sb, -1, NS, pad);
          P2[b] = step_axis(Sb, 2, NS, pad);
          M2[b] = step_axis(Sb, -2, NS, pad);
          auto fluid = [&](const int *P) {
            return P[b] >= 0 && flags[sidx(g, P[0], P[1], P[2])] == NODE_FLUID;
          };
          auto vel = [&](const int *P, R (&u)[3]) {
            dev_velocity<Q, S, R>(g, f, sidx(g, P[0], P[1], P[2]), u);
          };
          const bool fp = fluid(P1), fm = fluid(M1);
          R a1[3], a2[3];
          if (fp && fm) {
            vel(P1, a1);
            vel(M1, a2);
            for (int a = 0; a < D; ++a) G[a][b] = (R)0.5 * (a1[a] - a2[a]);
          } else if (fp) {
            vel(P1, a1);
            if (fluid(P2)) {
              vel(P2, a2);
              for (int a = 0; a < D; ++a) G[a][b] = (R)0.5 * ((R)-3 * u0[a] + (R)4 * a1[a] - a2[a]);
            } else {
              for (int a = 0; a < D; ++a) G[a][b] = a1[a] - u0[a];
            }
          } else if (fm) {
            vel(M1, a1);
            if (fluid(M2)) {
              vel(M2, a2);
              for (int a = 0; a < D; ++a) G[a][b] = (R)0.5 * ((R)3 * u0[a] - (R)4 * a1[a] + a2[a]);
            } else {
              for (int a = 0; a < D; ++a) G[a][b] = u0[a] - a1[a];
            }
          }
        }
      }
      // ---- Grad's approximation, Eq. (grad)
      // A = rho u u + Pi_neq on the lattice's axes; c.A.c and c.u per
      // direction with the components fixed at compile time (zero
      // components skipped, unit ones added or subtracted)
      R A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      const R cneq = -rho_t / ((R)6 * (R)bp.beta);
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) A[a][b] = rho_t * ut[a] * ut[b] + cneq * (G[a][b] + G[b][a]);
      R trA = A[0][0] + A[1][1];
      if (D == 3) trA += A[2][2];
      const R tr3 = trA * (R)(1.0 / 3.0);
      const R A01 = A[0][1] + A[1][0], A02 = A[0][2] + A[2][0], A12 = A[1][2] + A[2][1];
      const R r3 = (R)3 * rho_t, rm1 = rho_t - (R)1;
      int l = 0;
      // D2Q9: unrolled, the components fold at compile time; D3Q27: one
      // loop body (27 copies would crowd the instruction cache), the
      // branches on c_i are uniform across the warp
#pragma unroll(Q == 9 ? 9 : 1)
      for (int i = 0; i < Q; ++i) {
        if (!((miss >> i) & 1u)) continue;
        const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
        R cAc = 0, cu = 0;
        for (int a = 0; a < D; ++a) {
          if (c[a] != 0) cAc += A[a][a];
          if (c[a] > 0) cu += ut[a];
          if (c[a] < 0) cu -= ut[a];
        }
        if (c[0] * c[1] > 0) cAc += A01;
        if (c[0] * c[1] < 0) cAc -= A01;
        if (D == 3) {
          if (c[0] * c[2] > 0) cAc += A02;
          if (c[0] * c[2] < 0) cAc -= A02;
          if (c[1] * c[2] > 0) cAc += A12;
          if (c[1] * c[2] < 0) cAc -= A12;
        }
        const DirTab<Q> &dt = dir_tab<Q>();
        const R gstar = (R)dt.w[i] * (rm1 + r3 * cu + (R)4.5 * (cAc - tr3));
        using C = typename St::C;
        St::store(f + (long long)i * g.N + src[i], (C)gstar, (C)dt.iwf[i]);
        if (face_of[i] < 0) {
          // momentum exchange on the immersed surface, FP64 accumulation
          while (l < bn.nlink && links[bn.link0 + l].i != i) ++l;
          if (l < bn.nlink) {
            const Link &lk = links[bn.link0 + l];
            if (lk.body >= 0) {
              const double gop =
                  (double)St::load(f + (long long)(Q - 1 - i) * g.N + k, (C)dt.w[i]);
              // gauge form: the rest state f = W (ambient pressure) is taken out
              const double fsum = gop + (double)(C)gstar;
              for (int a = 0; a < D; ++a) {
                if (c[a] == 0) continue;
                const double Fa = c[a] > 0 ? -fsum : fsum;
                for (int m = 0; m < D; ++m)
                  atomicAdd(&vforce[3 * lk.v[m] + a], (double)lk.vw[m] * Fa);
                if (lk.body == my_body || my_body < 0) {
                  my_body = lk.body;
                  Fd[a] += Fa;
                } else {
                  atomicAdd(&bforce[3 * lk.body + a], Fa);
                }
              }
            }
          }
        }
      }
    }
  }
  body_reduce(nbodies, my_body, Fd, bforce);
}

template <int Q, int S, typename R>
__global__ void __launch_bounds__(128)
    k_grad(Grid g, typename Store<S>::T *f, const uint8_t *__restrict__ flags,
           const BNode *__restrict__ bnodes, const int *__restrict__ nbn, int nfixed, int cap,
           int first, int last, const Link *__restrict__ links, BoundaryParams bp, double *vforce,
           double *bforce, int nbodies) {
  grad_body<Q, S, R>(blockIdx.x * blockDim.x + threadIdx.x, g, f, flags, bnodes, nbn, nfixed, cap,
                     first, last, links, bp, vforce, bforce, nbodies);
}

// ---- the same fill with one warp per boundary node (FP64), for single
// lattices, where a few hundred to a few thousand nodes would otherwise run
// their chains of neighbour velocities one after another on few warps: lane
// i gathers direction i and computes the velocity of the neighbour x_b + c_i
// when it is needed (lanes 0..5 then the second neighbours of one-sided
// gradients), lane 0 assembles the targets and the stress exactly as
// grad_body does (same operations in the same order, velocities from the
// lanes), and lane i forms, stores and gathers the force of its missing
// direction.  Every value written equals grad_body's; only the order of the
// FP64 force atomics differs.
template <int Q, typename C>
struct GradWarpSh {
  double vel[Q + 6][3];  // [i < Q]: node x_b + c_i; [Q + 2b (+1)]: x_b + 2 e_b (- 2 e_b)
  double rho[Q];
  C gk[Q], gop[Q];       // known populations; f_opp(i)(x_b) of missing i
  float q[Q], uw[Q][3];  // link fraction and wall velocity of missing i
  double ut[3], Ad[3], A01, A02, A12, tr3, r3, rm1;
};

template <int Q>
__device__ __forceinline__ int dir_index(int cx, int cy, int cz) {
  return Q == 9 ? (cy + 1) * 3 + (cx + 1) : (cz + 1) * 9 + (cy + 1) * 3 + (cx + 1);
}

template <int Q, int S>
__device__ __forceinline__ void grad_warp_node(int t, const Grid &g, typename Store<S>::T *f,
                                               const uint8_t *__restrict__ flags,
                                               const BNode *__restrict__ bnodes, int nfixed,
                                               const Link *__restrict__ links,
                                               const BoundaryParams &bp, double *vforce,
                                               double *bforce,
                                               GradWarpSh<Q, typename Store<S>::C> &W, int lane,
                                               int &my_body, double (&Fd)[3]) {
  using L = Lat<Q>;
  using St = Store<S>;
  using R = double;
  constexpr int D = L::D;
  constexpr unsigned FULL = 0xffffffffu;
  const int rest = (Q - 1) / 2;
  const BNode bn = bnodes[t];
  const long long k = bn.k;
  int X, Y, Z;
  decompose(g, k, X, Y, Z);
  // ---- gather: lane i takes direction i
  const bool dl = lane < Q;
  const int i = dl ? lane : 0;
  const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
  long long src = 0;
  int face = -1;
  uint8_t fl = NODE_FLUID;
  if (dl) {
    const int Xs = nbr(X, -cx, g.NX), Ys = nbr(Y, -cy, g.NY), Zs = (D == 3) ? nbr(Z, -cz, g.NZ) : Z;
    src = sidx(g, Xs, Ys, Zs);
    fl = flags[src];
    if (fl == NODE_FLUID) {
      W.gk[i] = St::load(f + (long long)i * g.N + src, (typename St::C)dir_tab<Q>().w[i]);
    } else if (fl == NODE_GHOST) {
      if (g.px && (Xs == 0 || Xs == g.NX - 1)) face = Xs == 0 ? 0 : 1;
      else if (g.py && (Ys == 0 || Ys == g.NY - 1)) face = Ys == 0 ? 2 : 3;
      else face = Zs == 0 ? 4 : 5;
    }
  }
  uint32_t miss = __ballot_sync(FULL, dl && fl != NODE_FLUID);
  const uint32_t solid_miss = __ballot_sync(FULL, dl && fl == NODE_SOLID);
  if (t < nfixed && solid_miss) miss = 0;  // as in grad_body
  if (!miss) return;
  const bool mi = dl && ((miss >> i) & 1u);
  // ---- open face: the first face (in face order) crossed by a missing link
  int open_face = -1;
  for (int fc = 0; fc < 6; ++fc) {
    const bool open = bp.bc[fc] == BCK_INLET || bp.bc[fc] == BCK_OUTLET || bp.bc[fc] == BCK_FREESTREAM;
    if (open && __any_sync(FULL, mi && face == fc)) {
      open_face = fc;
      break;
    }
  }
  const bool zero_grad = open_face >= 0 && bp.bc[open_face] == BCK_FREESTREAM;
  int kn_dir = rest;
  if (open_face >= 0) {
    const int ax = open_face / 2, dir = (open_face % 2 == 0) ? 1 : -1;
    int Xn = X, Yn = Y, Zn = Z;
    if (ax == 0) Xn = step_axis(X, dir, g.NX, g.px);
    if (ax == 1) Yn = step_axis(Y, dir, g.NY, g.py);
    if (ax == 2) Zn = step_axis(Z, dir, g.NZ, g.pz);
    if (Xn >= 0 && Yn >= 0 && Zn >= 0 && flags[sidx(g, Xn, Yn, Zn)] == NODE_FLUID)
      kn_dir = dir_index<Q>(ax == 0 ? dir : 0, ax == 1 ? dir : 0, ax == 2 ? dir : 0);
  }
  // ---- neighbour velocities, lane i: x_b + c_i
  bool nfluid = false;
  int Xn = X, Yn = Y, Zn = Z;
  if (dl) {
    Xn = step_axis(X, cx, g.NX, g.px);
    Yn = step_axis(Y, cy, g.NY, g.py);
    Zn = (D == 3) ? step_axis(Z, cz, g.NZ, g.pz) : Z;
    nfluid = Xn >= 0 && Yn >= 0 && Zn >= 0 && flags[sidx(g, Xn, Yn, Zn)] == NODE_FLUID;
  }
  const uint32_t fmask = __ballot_sync(FULL, dl && nfluid);
  bool need = false;
  if (dl) {
    const int nnz = (cx != 0) + (cy != 0) + (cz != 0);
    need = open_face >= 0 ? i == kn_dir : (mi && nfluid);
    if (!zero_grad && (i == rest || (nnz == 1 && nfluid))) need = true;
  }
  if (need) {
    R u[3], r;
    dev_velocity<Q, S, R>(g, f, sidx(g, Xn, Yn, Zn), u, &r);
    W.vel[i][0] = u[0];
    W.vel[i][1] = u[1];
    W.vel[i][2] = u[2];
    W.rho[i] = r;
  }
  // second neighbours of one-sided gradients: lane j < 2 D, axis j / 2
  uint32_t f2mask = 0;
  if (!zero_grad) {
    bool f2 = false;
    if (lane < 2 * D) {
      const int b = lane / 2, sgn = (lane % 2 == 0) ? 1 : -1;
      const int ip = dir_index<Q>(b == 0, b == 1, b == 2), im = dir_index<Q>(-(b == 0), -(b == 1), -(b == 2));
      const bool fp = (fmask >> ip) & 1u, fm = (fmask >> im) & 1u;
      if (sgn > 0 ? (fp && !fm) : (fm && !fp)) {
        int P[3] = {X, Y, Z};
        const int NS = b == 0 ? g.NX : (b == 1 ? g.NY : g.NZ);
        const int pad = b == 0 ? g.px : (b == 1 ? g.py : g.pz);
        P[b] = step_axis(P[b], 2 * sgn, NS, pad);
        if (P[b] >= 0 && flags[sidx(g, P[0], P[1], P[2])] == NODE_FLUID) {
          f2 = true;
          R u[3];
          dev_velocity<Q, S, R>(g, f, sidx(g, P[0], P[1], P[2]), u);
          W.vel[Q + lane][0] = u[0];
          W.vel[Q + lane][1] = u[1];
          W.vel[Q + lane][2] = u[2];
        }
      }
    }
    f2mask = __ballot_sync(FULL, f2);
  }
  // link data of the missing directions
  if (mi) {
    float q = 0.5f, uw[3] = {0.f, 0.f, 0.f};
    if (face >= 0) {
      for (int a = 0; a < 3; ++a) uw[a] = bp.face_u[face][a];
    } else {
      for (int l = 0; l < bn.nlink; ++l) {
        const Link &lk = links[bn.link0 + l];
        if (lk.i == i) {
          q = lk.q;
          for (int a = 0; a < 3; ++a) uw[a] = lk.uw[a];
          break;
        }
      }
    }
    W.q[i] = q;
    for (int a = 0; a < 3; ++a) W.uw[i][a] = uw[a];
    W.gop[i] = St::load(f + (long long)(Q - 1 - i) * g.N + k, (typename St::C)dir_tab<Q>().w[i]);
  }
  __syncwarp();
  // ---- targets and stress on lane 0 (grad_body's arithmetic)
  if (lane == 0) {
    const int nmiss = __popc(miss);
    R rho_t, ut[3] = {0, 0, 0};
    if (open_face >= 0) {
      const int ax = open_face / 2;
      const R u0[3] = {W.vel[kn_dir][0], W.vel[kn_dir][1], W.vel[kn_dir][2]};
      const R r0 = W.rho[kn_dir];
      if (bp.bc[open_face] == BCK_INLET) {
        R scale = 1;
        if (bp.ramp_steps > 0 && bp.step) {
          const int st = *bp.step;
          if (st < bp.ramp_steps) scale = (R)0.5 * ((R)1 - cospi((double)st / bp.ramp_steps));
        }
        const float *prof = bp.inlet[open_face];
        const int x = X - g.px, y = Y - g.py, z = Z - g.pz;
        long long fidx, fn;
        if (ax == 0) { fidx = (long long)z * g.ny + y; fn = (long long)g.ny * g.nz; }
        else if (ax == 1) { fidx = (long long)z * g.nx + x; fn = (long long)g.nx * g.nz; }
        else { fidx = (long long)y * g.nx + x; fn = (long long)g.nx * g.ny; }
        for (int a = 0; a < D; ++a)
          ut[a] = scale * (R)(prof ? prof[a * fn + fidx] : bp.face_u[open_face][a]);
        rho_t = r0;
      } else if (bp.bc[open_face] == BCK_OUTLET) {
        for (int a = 0; a < D; ++a) ut[a] = u0[a];
        rho_t = 1;
      } else {
        for (int a = 0; a < D; ++a) ut[a] = bp.face_u[open_face][a];
        rho_t = 1;
      }
    } else {
      PopSum<R> pops;
      R wterm = 0;
      for (int j = 0; j < Q; ++j) {
        if (!((miss >> j) & 1u)) {
          pops.add(W.gk[j]);
          continue;
        }
        const R q = W.q[j];
        const R uw[3] = {W.uw[j][0], W.uw[j][1], W.uw[j][2]};
        const double wi = dir_tab<Q>().w[j];
        R cuw = L::cx(j) * uw[0] + L::cy(j) * uw[1];
        if (D == 3) cuw += L::cz(j) * uw[2];
        pops.add(W.gop[j]);
        wterm += (R)(6.0 * wi) * cuw;
        R ui[3] = {uw[0], uw[1], uw[2]};
        if ((fmask >> j) & 1u) {
          const R iq = (R)1 / ((R)1 + q);
          for (int a = 0; a < D; ++a) ui[a] = (uw[a] + q * W.vel[j][a]) * iq;
        }
        for (int a = 0; a < D; ++a) ut[a] += ui[a];
      }
      const R inm = (R)1 / (R)nmiss;
      for (int a = 0; a < D; ++a) ut[a] *= inm;
      rho_t = (R)1 + ((R)pops.value() + wterm);
    }
    R G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (!zero_grad) {
      const R u0[3] = {W.vel[rest][0], W.vel[rest][1], W.vel[rest][2]};
      for (int b = 0; b < D; ++b) {
        const int ip = dir_index<Q>(b == 0, b == 1, b == 2), im = dir_index<Q>(-(b == 0), -(b == 1), -(b == 2));
        const bool fp = (fmask >> ip) & 1u, fm = (fmask >> im) & 1u;
        if (fp && fm) {
          for (int a = 0; a < D; ++a) G[a][b] = (R)0.5 * (W.vel[ip][a] - W.vel[im][a]);
        } else if (fp) {
          if ((f2mask >> (2 * b)) & 1u) {
            for (int a = 0; a < D; ++a)
              G[a][b] = (R)0.5 * ((R)-3 * u0[a] + (R)4 * W.vel[ip][a] - W.vel[Q + 2 * b][a]);
          } else {
            for (int a = 0; a < D; ++a) G[a][b] = W.vel[ip][a] - u0[a];
          }
        } else if (fm) {
          if ((f2mask >> (2 * b + 1)) & 1u) {
            for (int a = 0; a < D; ++a)
              G[a][b] = (R)0.5 * ((R)3 * u0[a] - (R)4 * W.vel[im][a] + W.vel[Q + 2 * b + 1][a]);
          } else {
            for (int a = 0; a < D; ++a) G[a][b] = u0[a] - W.vel[im][a];
          }
        }
      }
    }
    R A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const R cneq = -rho_t / ((R)6 * (R)bp.beta);
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) A[a][b] = rho_t * ut[a] * ut[b] + cneq * (G[a][b] + G[b][a]);
    R trA = A[0][0] + A[1][1];
    if (D == 3) trA += A[2][2];
    W.tr3 = trA * (R)(1.0 / 3.0);
    W.A01 = A[0][1] + A[1][0];
    W.A02 = A[0][2] + A[2][0];
    W.A12 = A[1][2] + A[2][1];
    W.r3 = (R)3 * rho_t;
    W.rm1 = rho_t - (R)1;
    for (int a = 0; a < 3; ++a) {
      W.Ad[a] = A[a][a];
      W.ut[a] = ut[a];
    }
  }
  __syncwarp();
  // ---- lane i: f*_i of its missing direction, its store and its force
  if (mi) {
    const int c[3] = {cx, cy, cz};
    R cAc = 0, cu = 0;
    for (int a = 0; a < D; ++a) {
      if (c[a] != 0) cAc += W.Ad[a];
      if (c[a] > 0) cu += W.ut[a];
      if (c[a] < 0) cu -= W.ut[a];
    }
    if (c[0] * c[1] > 0) cAc += W.A01;
    if (c[0] * c[1] < 0) cAc -= W.A01;
    if (D == 3) {
      if (c[0] * c[2] > 0) cAc += W.A02;
      if (c[0] * c[2] < 0) cAc -= W.A02;
      if (c[1] * c[2] > 0) cAc += W.A12;
      if (c[1] * c[2] < 0) cAc -= W.A12;
    }
    const DirTab<Q> &dt = dir_tab<Q>();
    const R gstar = (R)dt.w[i] * (W.rm1 + W.r3 * cu + (R)4.5 * (cAc - W.tr3));
    using C = typename St::C;
    St::store(f + (long long)i * g.N + src, (C)gstar, (C)dt.iwf[i]);
    if (face < 0) {
      int l = 0;
      while (l < bn.nlink && links[bn.link0 + l].i != i) ++l;
      if (l < bn.nlink) {
        const Link &lk = links[bn.link0 + l];
        if (lk.body >= 0) {
          const double fsum = (double)W.gop[i] + (double)(C)gstar;
          for (int a = 0; a < D; ++a) {
            if (c[a] == 0) continue;
            const double Fa = c[a] > 0 ? -fsum : fsum;
            for (int m = 0; m < D; ++m) atomicAdd(&vforce[3 * lk.v[m] + a], (double)lk.vw[m] * Fa);
            if (lk.body == my_body || my_body < 0) {
              my_body = lk.body;
              Fd[a] += Fa;
            } else {
              atomicAdd(&bforce[3 * lk.body + a], Fa);
            }
          }
        }
      }
    }
  }
  __syncwarp();
}

// Warps stride over the boundary nodes [first, count) (count = nfixed +
// immersed when last < 0, else last).
template <int Q, int S>
__device__ __forceinline__ void grad_warp_range(const Grid &g, typename Store<S>::T *f,
                                                const uint8_t *__restrict__ flags,
                                                const BNode *__restrict__ bnodes,
                                                const int *__restrict__ nbn, int nfixed, int cap,
                                                int first, int last, const Link *__restrict__ links,
                                                const BoundaryParams &bp, double *vforce,
                                                double *bforce, int nbodies, int w0, int nw) {
  __shared__ GradWarpSh<Q, typename Store<S>::C> sh[4];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  int dyn = nbn ? *nbn : 0;
  if (dyn > cap - nfixed) dyn = cap - nfixed;
  const int count = last < 0 ? nfixed + dyn : last;
  int my_body = -1;
  double Fd[3] = {0, 0, 0};
  for (int t = first + w0; t < count; t += nw)
    grad_warp_node<Q, S>(t, g, f, flags, bnodes, nfixed, links, bp, vforce, bforce, sh[wl], lane,
                         my_body, Fd);
  body_reduce(nbodies, my_body, Fd, bforce);
}

template <int Q, int S>
__global__ void __launch_bounds__(128)
    k_grad_warp(Grid g, typename Store<S>::T *f, const uint8_t *__restrict__ flags,
                const BNode *__restrict__ bnodes, const int *__restrict__ nbn, int nfixed, int cap,
                int first, int last, const Link *__restrict__ links, BoundaryParams bp,
                double *vforce, double *bforce, int nbodies) {
  grad_warp_range<Q, S>(g, f, flags, bnodes, nbn, nfixed, cap, first, last, links, bp, vforce,
                        bforce, nbodies, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
                        (int)((gridDim.x * blockDim.x) >> 5));
}

// 3-D boundary fill in one launch: the first face_blocks CTAs take the face
// nodes in FP32 (one thread each), the rest the immersed nodes in FP64 with
// the force gather (one warp each), so the two sets run side by side.
template <int Q, int S>
__global__ void __launch_bounds__(128)
    k_grad_split(Grid g, typename Store<S>::T *f, const uint8_t *__restrict__ flags,
                 const BNode *__restrict__ bnodes, const int *__restrict__ nbn, int nfixed, int cap,
                 const Link *__restrict__ links, BoundaryParams bp, double *vforce, double *bforce,
                 int nbodies, int face_blocks) {
  if ((int)blockIdx.x < face_blocks)
    grad_body<Q, S, float>(blockIdx.x * blockDim.x + threadIdx.x, g, f, flags, bnodes, nullptr,
                           nfixed, cap, 0, nfixed, links, bp, vforce, bforce, 0);
  else
    grad_warp_range<Q, S>(g, f, flags, bnodes, nbn, nfixed, cap, nfixed, -1, links, bp, vforce,
                          bforce, nbodies,
                          (int)(((blockIdx.x - face_blocks) * blockDim.x + threadIdx.x) >> 5),
                          (int)(((gridDim.x - face_blocks) * blockDim.x) >> 5));
}

__global__ void k_step_counter(int *step) { *step += 1; }

// ---------------------------------------------------------------- launchers
static inline unsigned nb_(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// Grid of the link-fill pass: four 128-thread CTAs per SM, warps striding
// over the boundary-node list.
static unsigned fill_grid() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 128;
  }
  return 4u * (unsigned)sms;
}

static cudaError_t launch_link_fill(int Q, const Grid &g, const SurfaceDev &sd, const uint8_t *flags,
                                    const BNode *bnodes, const int *nbn, int bcap, Link *links,
                                    cudaStream_t s) {
  if (Q == 9)
    k_link_fill<9><<<fill_grid(), 128, 0, s>>>(g, sd, flags, bnodes, nbn, bcap, links);
  else
    k_link_fill<27><<<fill_grid(), 128, 0, s>>>(g, sd, flags, bnodes, nbn, bcap, links);
  return cudaGetLastError();
}

cudaError_t launch_mark_ghosts(const Grid &g, uint8_t *flags, cudaStream_t s) {
  k_mark_ghosts<<<nb_(g.N, 256), 256, 0, s>>>(g, flags);
  return cudaGetLastError();
}

cudaError_t launch_face_nodes(const Grid &g, BNode *out, int *count, int cap, cudaStream_t s) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  k_face_nodes<<<nb_(n, 256), 256, 0, s>>>(g, out, count, cap);
  return cudaGetLastError();
}

static cudaError_t launch_fresh(int Q, int storage, const Grid &g, void *f, const uint8_t *flags,
                                const int64_t *fresh, const int *nfresh, int cap,
                                const SurfaceDev &sd, cudaStream_t s) {
  KBC_DISPATCH(Q, storage, {
    k_fresh_init<QQ, SS><<<nb_(cap, 128), 128, 0, s>>>(g, (typename Store<SS>::T *)f, flags, fresh,
                                                       nfresh, cap, sd);
    return cudaGetLastError();
  });
}

cudaError_t launch_geometry(int Q, int storage, const Grid &g, const Band &bd, const SurfaceDev &sd,
                            uint8_t *flags, void *f, int64_t *fresh, int *nfresh, int fresh_cap,
                            int track_fresh, BNode *bnodes, int *nbn, int bcap, Link *links,
                            int *nl, int lcap, int *err, cudaStream_t s) {
  const long long nb = (long long)(bd.x1 - bd.x0) * (bd.y1 - bd.y0) * (bd.z1 - bd.z0);
  if (nb <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaMemsetAsync(nfresh, 0, sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(nbn, 0, sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(nl, 0, sizeof(int), s)) != cudaSuccess) return e;
  if (sd.box) {
    k_surface_box<<<1, 256, 0, s>>>(sd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // nodes inside the surface's box go to a second, warp-per-node pass; the
  // immersed-node list (rebuilt below) holds their indices meanwhile, its
  // counter counts them
  int *near_list = reinterpret_cast<int *>(bnodes);
  const int near_cap = (int)((long long)bcap * sizeof(BNode) / sizeof(int));
  k_solid_flags<<<nb_(nb, 128), 128, 0, s>>>(g, bd, sd, flags, fresh, nfresh, fresh_cap,
                                              track_fresh, near_list, nbn, near_cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_solid_near<<<fill_grid(), 128, 0, s>>>(g, bd, sd, flags, fresh, nfresh, fresh_cap, track_fresh,
                                           near_list, nbn, near_cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(nbn, 0, sizeof(int), s)) != cudaSuccess) return e;
  if (track_fresh && (e = launch_fresh(Q, storage, g, f, flags, fresh, nfresh, fresh_cap, sd, s)) !=
                         cudaSuccess)
    return e;
  if (Q == 9)
    k_build_links<9><<<nb_(nb, 128), 128, 0, s>>>(g, bd, sd, flags, bnodes, nbn, bcap, links, nl,
                                                   lcap, err);
  else
    k_build_links<27><<<nb_(nb, 128), 128, 0, s>>>(g, bd, sd, flags, bnodes, nbn, bcap, links,
                                                    nl, lcap, err);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return e2;
  return launch_link_fill(Q, g, sd, flags, bnodes, nbn, bcap, links, s);
}

cudaError_t launch_grad(int Q, int storage, const Grid &g, void *f, const uint8_t *flags,
                        const BNode *bnodes, const int *nbn, int nfixed, int cap,
                        const Link *links, const BoundaryParams &bp, double *vforce,
                        double *bforce, int nbodies, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  KBC_DISPATCH(Q, storage, {
    using T = typename Store<SS>::T;
    if (QQ == 9) {
      // 2-D: face and immersed nodes both in FP64, one launch, one warp per
      // node (striding over the lists)
      k_grad_warp<QQ, SS><<<fill_grid(), 128, 0, s>>>(g, (T *)f, flags, bnodes, nbn, nfixed, cap, 0,
                                                      -1, links, bp, vforce, bforce, nbodies);
      return cudaGetLastError();
    }
    // 3-D face nodes in FP32 (their count scales with the lattice faces),
    // immersed nodes in FP64; both sets in one launch when both exist
    if (nfixed > 0 && cap > nfixed) {
      const int fb = (int)nb_(nfixed, 128);
      k_grad_split<QQ, SS><<<fb + fill_grid(), 128, 0, s>>>(
          g, (T *)f, flags, bnodes, nbn, nfixed, cap, links, bp, vforce, bforce, nbodies, fb);
      return cudaGetLastError();
    }
    if (nfixed > 0) {
      if (QQ == 9)
        k_grad<QQ, SS, double><<<nb_(nfixed, 128), 128, 0, s>>>(
            g, (T *)f, flags, bnodes, nullptr, nfixed, cap, 0, nfixed, links, bp, vforce, bforce,
            0);
      else
        k_grad<QQ, SS, float><<<nb_(nfixed, 128), 128, 0, s>>>(
            g, (T *)f, flags, bnodes, nullptr, nfixed, cap, 0, nfixed, links, bp, vforce, bforce,
            0);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    // immersed boundary nodes in FP64 arithmetic, with the force gather
    if (cap > nfixed) {
      k_grad<QQ, SS, double><<<nb_(cap - nfixed, 128), 128, 0, s>>>(
          g, (T *)f, flags, bnodes, nbn, nfixed, cap, nfixed, -1, links, bp, vforce, bforce,
          nbodies);
    }
    return cudaGetLastError();
  });
}

cudaError_t launch_build_links(int Q, const Grid &g, const Band &bd, const SurfaceDev &sd,
                               const uint8_t *flags, BNode *bnodes, int *nbn, int bcap,
                               Link *links, int *nl, int lcap, int *err, cudaStream_t s) {
  const long long nb = (long long)(bd.x1 - bd.x0) * (bd.y1 - bd.y0) * (bd.z1 - bd.z0);
  if (nb <= 0) return cudaSuccess;
  if (Q == 9)
    k_build_links<9><<<nb_(nb, 128), 128, 0, s>>>(g, bd, sd, flags, bnodes, nbn, bcap, links, nl,
                                                   lcap, err);
  else
    k_build_links<27><<<nb_(nb, 128), 128, 0, s>>>(g, bd, sd, flags, bnodes, nbn, bcap, links,
                                                    nl, lcap, err);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return e2;
  return launch_link_fill(Q, g, sd, flags, bnodes, nbn, bcap, links, s);
}

// ---------------------------------------------------------------- batched phases
// Zero the force accumulators of every lattice and reset the sweep's tile ticket.
__global__ void k_batch_pre(const InstDesc *__restrict__ d, int *ticket) {
  const InstDesc &b = d[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ticket = 0;
  if (b.nbodies == 0) return;
  if (t < 3 * b.nv) b.vforce[t] = 0.0;
  if (t < 3 * b.nbodies) b.bforce[t] = 0.0;
}

template <int Q, int S>
__global__ void __launch_bounds__(128) k_grad_batch(const InstDesc *__restrict__ d, int parity) {
  const InstDesc &b = d[blockIdx.y];
  if ((int)(blockIdx.x * blockDim.x) >= b.cap) return;  // whole block idle
  typename Store<S>::T *f = (typename Store<S>::T *)b.f[(b.cur0 + parity) & 1];
  grad_body<Q, S, double>(blockIdx.x * blockDim.x + threadIdx.x, b.g, f, b.flags, b.bnodes, b.nbn,
                          b.nfixed, b.cap, 0, -1, b.links, b.bp, b.vforce, b.bforce, b.nbodies);
}

__global__ void k_geom_reset_batch(const InstDesc *__restrict__ d, const int *__restrict__ idx,
                                   int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const InstDesc &b = d[idx[t]];
  *b.nbn = 0;
  *b.nl = 0;
  *b.nfresh = 0;
}

__global__ void __launch_bounds__(256) k_surface_box_batch(const InstDesc *__restrict__ d,
                                                           const int *__restrict__ idx) {
  const InstDesc &b = d[idx[blockIdx.x]];
  if (b.sd.box) surface_box_body(b.sd);
}

__global__ void k_solid_flags_batch(const InstDesc *__restrict__ d, const int *__restrict__ idx) {
  const InstDesc &b = d[idx[blockIdx.y]];
  // one pass: across 64 members the in-box nodes already fill the GPU one
  // thread each (the warp-per-node pass measured slower here)
  solid_flags_body(blockIdx.x * (long long)blockDim.x + threadIdx.x, b.g, b.band, b.sd, b.flags,
                   b.fresh, b.nfresh, b.lcap, 1);
}

template <int Q, int S>
__global__ void k_fresh_batch(const InstDesc *__restrict__ d, const int *__restrict__ idx,
                              int parity) {
  const InstDesc &b = d[idx[blockIdx.y]];
  typename Store<S>::T *f = (typename Store<S>::T *)b.f[(b.cur0 + parity) & 1];
  fresh_init_body<Q, S>(blockIdx.x * blockDim.x + threadIdx.x, b.g, f, b.flags, b.fresh, b.nfresh,
                        b.lcap, b.sd);
}

template <int Q>
__global__ void k_links_batch(const InstDesc *__restrict__ d, const int *__restrict__ idx) {
  const InstDesc &b = d[idx[blockIdx.y]];
  build_links_body<Q>(blockIdx.x * (long long)blockDim.x + threadIdx.x, b.g, b.band, b.sd, b.flags,
                      b.bnodes + b.nfixed, b.nbn, b.lcap, b.links, b.nl, b.lcap, b.err);
}

template <int Q>
__global__ void __launch_bounds__(128) k_link_fill_batch(const InstDesc *__restrict__ d,
                                                         const int *__restrict__ idx) {
  const InstDesc &b = d[idx[blockIdx.y]];
  link_fill_body<Q>(b.g, b.sd, b.flags, b.bnodes + b.nfixed, b.nbn, b.lcap, b.links,
                    (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
                    (int)((gridDim.x * blockDim.x) >> 5));
}

cudaError_t launch_batch_pre(const InstDesc *d, int n, int max_nv3, int *ticket, cudaStream_t s) {
  dim3 grid(nb_(max_nv3 > 0 ? max_nv3 : 1, 128), n);
  k_batch_pre<<<grid, 128, 0, s>>>(d, ticket);
  return cudaGetLastError();
}

cudaError_t launch_grad_batch(int Q, int storage, const InstDesc *d, int n, int max_cap, int parity,
                              cudaStream_t s) {
  if (max_cap <= 0) return cudaSuccess;
  dim3 grid(nb_(max_cap, 128), n);
  KBC_DISPATCH(Q, storage, {
    k_grad_batch<QQ, SS><<<grid, 128, 0, s>>>(d, parity);
    return cudaGetLastError();
  });
}

cudaError_t launch_geometry_batch(int Q, int storage, const InstDesc *d, const int *idx, int n,
                                  long long max_band, int max_fresh, int parity, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_geom_reset_batch<<<nb_(n, 128), 128, 0, s>>>(d, idx, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 gb(nb_(max_band, 128), n), gf(nb_(max_fresh, 128), n);
  k_surface_box_batch<<<n, 256, 0, s>>>(d, idx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_solid_flags_batch<<<gb, 128, 0, s>>>(d, idx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  KBC_DISPATCH(Q, storage, {
    k_fresh_batch<QQ, SS><<<gf, 128, 0, s>>>(d, idx, parity);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // 64 CTAs (256 warps) per member: the largest member's boundary nodes,
    // one warp each, bound the pass; surplus warps of small members exit
    const dim3 gl(64, n);
    if (QQ == 9) k_links_batch<9><<<gb, 128, 0, s>>>(d, idx);
    else k_links_batch<27><<<gb, 128, 0, s>>>(d, idx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (QQ == 9) k_link_fill_batch<9><<<gl, 128, 0, s>>>(d, idx);
    else k_link_fill_batch<27><<<gl, 128, 0, s>>>(d, idx);
    return cudaGetLastError();
  });
}

cudaError_t launch_step_counter(int *step, cudaStream_t s) {
  k_step_counter<<<1, 1, 0, s>>>(step);
  return cudaGetLastError();
}

}  // namespace kbc
