/*
 * kbc_oracle_bc.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Double-precision CPU statement of the boundary treatment of the KBC step:
 * Grad's approximation for the missing populations of fluid nodes next to a
 * wall, an open face or an immersed moving surface, and the momentum-exchange
 * force on the surface (Dorschner, Chikatamarla & Karlin, arXiv 1710.02375,
 * section "Fluid boundary conditions", Eq. (grad) and the Pi^eq / Pi^neq
 * closure that follows it; section "Solid boundary conditions").
 *
 * The paper defers the target values to earlier work.  Readings used here
 * (the CUDA library implements the same written reading with its own code):
 *   missing set M(x_b): directions i whose source node x_b - c_i is solid,
 *     or lies beyond a non-periodic face.
 *   Link data: immersed link i has q_i in (0,1] (wall point
 *     x_w = x_b - q_i c_i, the nearest crossing of the surface) and wall
 *     velocity u_w interpolated linearly along the hit segment (2-D) or
 *     barycentrically on the hit triangle (3-D); a wall face has q = 1/2 and
 *     the face velocity.
 *   Open node (a missing link crosses an inlet, outlet or free-stream face;
 *     first such face in the order -x,+x,-y,+y,-z,+z):
 *       inlet:       u_t = prescribed velocity, rho_t = rho(x_n, t-1)
 *       outlet:      u_t = u(x_n, t-1),         rho_t = 1
 *       (x_n: the next node inward across that face, x_b itself if x_n is
 *       not fluid)
 *       free stream: u_t = face velocity,        rho_t = 1, grad u = 0
 *   Wall node (all missing links are walls or immersed):
 *       u_i = (u_w,i + q_i u(x_b + c_i, t-1)) / (1 + q_i) if x_b + c_i is
 *             fluid, else u_w,i;  u_t = mean of u_i over M
 *       rho_t = sum_{i not in M} f_i + sum_{i in M} [f'_opp(i)(x_b, t-1)
 *               + 6 W_i c_i . u_w,i]      (moving-wall bounce-back density)
 *   grad u: finite differences of the previous-step velocity u(t-1): per
 *     axis the central difference when both neighbours are fluid, else the
 *     one-sided second-order difference through x_b itself (first order if
 *     only one fluid node lies on that side), else 0.  (Taking the target u_t
 *     at x_b in the one-sided stencil instead is unstable at beta = 1/2.)
 *   Pi = rho c_s^2 I + rho u u - rho c_s^2/(2 beta) (grad u + grad u^T);
 *   f*_i = W_i [rho + rho c_i.u / c_s^2 + (Pi - rho c_s^2 I):(c_i c_i - c_s^2 I)/(2 c_s^4)]
 *     replaces every missing population of the node (and only those).
 *   Force on the surface per immersed link: -c_i (f'_opp(i)(x_b,t-1) + f*_i - 2 W_i)
 *     (momentum exchange relative to the rest state f = W, i.e. with the
 *     uniform ambient pressure rho0 c_s^2 taken out; it cancels on a closed
 *     body but not on one attached to another), split over the hit element's
 *     vertices by the same interpolation weights.
 *   u(x, t-1) and rho(x, t-1) are the moments of the stored post-collision
 *   populations (collisions conserve them).
 *
 * Surface meshes: closed polygons (2-D: segments, element = 2 vertex ids) or
 * closed triangle meshes (3-D: element = 3 vertex ids), one body id per
 * element; node (x,y,z) of the interior is the centre of its cell, at
 * position (x + 1/2, y + 1/2, z + 1/2) in lattice units.  A node is
 * solid when it lies on the surface (within 1e-12) or inside any body
 * (crossing-number test per body along a fixed generic ray).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXQ 27

/* ---- lattice (own copy; the periodic oracle file keeps its tables static) */
typedef struct {
  int Q, D;
  int c[MAXQ][3];
  double w[MAXQ];
} lat_t;

static int lat_make(int lat, lat_t *L) {
  const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  if (lat != 9 && lat != 27) return -1;
  L->Q = lat;
  L->D = lat == 9 ? 2 : 3;
  for (int i = 0; i < lat; ++i) {
    int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = (lat == 27) ? i / 9 - 1 : 0;
    L->c[i][0] = cx; L->c[i][1] = cy; L->c[i][2] = cz;
    L->w[i] = w1[cx + 1] * w1[cy + 1] * (lat == 27 ? w1[cz + 1] : 1.0);
  }
  return 0;
}

/* Collision of one node (defined in kbc_oracle.c). */
int or_collide(int lat, double beta, int mode, const double *f, double *fout, double *gamma,
               double *ds, double *dh, double *feq);
int or_equilibrium(int lat, double rho, const double *u, double *feq);

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3, BC_FREESTREAM = 4 };

typedef struct {
  int dim;
  int nv, ne, nb;
  const double *x;    /* [nv][dim] */
  const double *v;    /* [nv][dim] */
  const int32_t *e;   /* [ne][dim] */
  const int32_t *eb;  /* [ne] body id */
} surf_t;

/* ------------------------------------------------------------ geometry */
/* Ray directions chosen to avoid passing through lattice-aligned vertices. */
static const double RAY2[2] = {0.8191520442889918, 0.5735764363510461};       /* 35 deg */
static const double RAY3[3] = {0.6245004513516506, 0.4806291366599437, 0.6155950585117604};

/* crossing of the ray p + t d (t > 0) with segment a-b at s in [0, 1):
 * t = tn/den, s = sn/den, compared without dividing */
static int ray_hits_segment(const double *p, const double *d, const double *a, const double *b) {
  double ex = b[0] - a[0], ey = b[1] - a[1];
  double den = d[0] * (-ey) - d[1] * (-ex);
  if (fabs(den) < 1e-300) return 0;
  double rx = a[0] - p[0], ry = a[1] - p[1];
  double tn = rx * (-ey) - ry * (-ex);
  double sn = d[0] * ry - d[1] * rx;
  if (den > 0.0) return tn > 0.0 && sn >= 0.0 && sn < den;
  return tn < 0.0 && sn <= 0.0 && sn > den;
}

static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Moller-Trumbore: p + t d hits triangle (a,b,c) at barycentrics (1-u-v, u, v). */
static int ray_triangle(const double *p, const double *d, const double *a, const double *b,
                        const double *c, double *t, double *u, double *v) {
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double pv[3];
  cross3(d, e2, pv);
  double det = dot3(e1, pv);
  if (fabs(det) < 1e-300) return 0;
  double inv = 1.0 / det;
  double tv[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  *u = dot3(tv, pv) * inv;
  double qv[3];
  cross3(tv, e1, qv);
  *v = dot3(d, qv) * inv;
  *t = dot3(e2, qv) * inv;
  return 1;
}

static int point_inside_body(const surf_t *S, int body, const double *p) {
  int cnt = 0;
  for (int k = 0; k < S->ne; ++k) {
    if (S->eb[k] != body) continue;
    if (S->dim == 2) {
      const double *a = S->x + 2 * S->e[2 * k], *b = S->x + 2 * S->e[2 * k + 1];
      cnt += ray_hits_segment(p, RAY2, a, b);
    } else {
      const double *a = S->x + 3 * S->e[3 * k], *b = S->x + 3 * S->e[3 * k + 1],
                   *c = S->x + 3 * S->e[3 * k + 2];
      double t, u, v;
      if (ray_triangle(p, RAY3, a, b, c, &t, &u, &v) && t > 0.0 && u >= 0.0 && v >= 0.0 &&
          u + v < 1.0)
        cnt++;
    }
  }
  return cnt & 1;
}

/* A point lying on the surface (within 1e-12 lattice units of an element) is
 * solid: the parity test alone would split nodes sitting exactly on a face
 * between solid and fluid depending on the ray direction. */
static int point_on_surface(const surf_t *S, const double *p) {
  const double tol = 1e-12;
  for (int k = 0; k < S->ne; ++k) {
    if (S->dim == 2) {
      const double *a = S->x + 2 * S->e[2 * k], *b = S->x + 2 * S->e[2 * k + 1];
      const double ex = b[0] - a[0], ey = b[1] - a[1];
      const double px = p[0] - a[0], py = p[1] - a[1];
      const double len2 = ex * ex + ey * ey;
      const double cr = ex * py - ey * px, dt = ex * px + ey * py;
      /* a zero-length element has no surface */
      if (len2 > 0.0 && fabs(cr) <= tol * sqrt(len2) && dt >= 0.0 && dt <= len2) return 1;
    } else {
      const double *a = S->x + 3 * S->e[3 * k], *b = S->x + 3 * S->e[3 * k + 1],
                   *c = S->x + 3 * S->e[3 * k + 2];
      const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      const double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
      double nrm[3];
      cross3(e1, e2, nrm);
      const double nn = sqrt(dot3(nrm, nrm));
      if (nn == 0.0 || fabs(dot3(nrm, w)) > tol * nn) continue;
      /* barycentric coordinates in the plane */
      const double d11 = dot3(e1, e1), d12 = dot3(e1, e2), d22 = dot3(e2, e2);
      const double dw1 = dot3(w, e1), dw2 = dot3(w, e2);
      const double den = d11 * d22 - d12 * d12;
      const double u = (d22 * dw1 - d12 * dw2) / den, v = (d11 * dw2 - d12 * dw1) / den;
      if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) return 1;
    }
  }
  return 0;
}

/* solid[n] (interior nodes) = 1 inside (or on) any body, else 0. */
int or_solid_mask(int dim, int nx, int ny, int nz, int nv, int ne, int nb, const double *x,
                  const int32_t *e, const int32_t *eb, uint8_t *solid) {
  surf_t S = {dim, nv, ne, nb, x, NULL, e, eb};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int xx = 0; xx < nx; ++xx) {
        double p[3] = {xx + 0.5, y + 0.5, z + 0.5};
        int in = point_on_surface(&S, p);
        for (int b = 0; b < nb && !in; ++b) in = point_inside_body(&S, b, p);
        solid[((long)z * ny + y) * nx + xx] = (uint8_t)in;
      }
  return 0;
}

/* Nearest crossing of the link x_b -> x_b - c (parameter s in (0, 1]) with the
 * surface.  Returns element id (or -1), q, wall velocity, vertex weights. */
static int link_hit(const surf_t *S, const double *xb, const int *c, double *q, double *uw,
                    int *vid, double *vw) {
  const double eps = 1e-9;
  int best = -1;
  double bs = 2.0;
  double bw[3] = {0, 0, 0};
  double d[3] = {-(double)c[0], -(double)c[1], -(double)c[2]};
  for (int k = 0; k < S->ne; ++k) {
    if (S->dim == 2) {
      const double *a = S->x + 2 * S->e[2 * k], *b = S->x + 2 * S->e[2 * k + 1];
      double ex = b[0] - a[0], ey = b[1] - a[1];
      double den = d[0] * (-ey) - d[1] * (-ex);
      if (fabs(den) < 1e-300) continue;
      double rx = a[0] - xb[0], ry = a[1] - xb[1];
      double s = (rx * (-ey) - ry * (-ex)) / den;
      double t = (d[0] * ry - d[1] * rx) / den;
      if (s > eps && s <= 1.0 + eps && t >= -eps && t <= 1.0 + eps && s < bs) {
        bs = s;
        best = k;
        double tt = t < 0 ? 0 : (t > 1 ? 1 : t);
        bw[0] = 1.0 - tt; bw[1] = tt; bw[2] = 0.0;
      }
    } else {
      const double *a = S->x + 3 * S->e[3 * k], *b = S->x + 3 * S->e[3 * k + 1],
                   *cc = S->x + 3 * S->e[3 * k + 2];
      double s, u, v;
      if (!ray_triangle(xb, d, a, b, cc, &s, &u, &v)) continue;
      if (s > eps && s <= 1.0 + eps && u >= -eps && v >= -eps && u + v <= 1.0 + eps && s < bs) {
        bs = s;
        best = k;
        double l0 = 1.0 - u - v;
        bw[0] = l0; bw[1] = u; bw[2] = v;
      }
    }
  }
  if (best < 0) return -1;
  *q = bs > 1.0 ? 1.0 : bs;
  for (int a = 0; a < 3; ++a) uw[a] = 0.0;
  for (int m = 0; m < S->dim; ++m) {
    vid[m] = S->e[S->dim * best + m];
    vw[m] = bw[m];
    for (int a = 0; a < S->dim; ++a) uw[a] += bw[m] * S->v[S->dim * vid[m] + a];
  }
  return best;
}

/* ------------------------------------------------------------ the step */
typedef struct {
  const lat_t *L;
  int n[3];
  int periodic[3];
  const uint8_t *solid;
  const double *fin;
  long N;
} field_t;

static long nid(const field_t *F, const int *p) { return ((long)p[2] * F->n[1] + p[1]) * F->n[0] + p[0]; }

/* map a position into the domain (periodic wrap); returns 0 if beyond a
 * non-periodic face */
static int in_domain(const field_t *F, int *p) {
  for (int a = 0; a < 3; ++a) {
    if (p[a] < 0 || p[a] >= F->n[a]) {
      if (!F->periodic[a]) return 0;
      p[a] = ((p[a] % F->n[a]) + F->n[a]) % F->n[a];
    }
  }
  return 1;
}

static int is_fluid(const field_t *F, const int *p0) {
  int p[3] = {p0[0], p0[1], p0[2]};
  if (!in_domain(F, p)) return 0;
  return F->solid[nid(F, p)] == 0;
}

static void node_moments(const field_t *F, const int *p0, double *rho, double *u) {
  int p[3] = {p0[0], p0[1], p0[2]};
  in_domain(F, p);
  long k = nid(F, p);
  double r = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < F->L->Q; ++i) {
    double v = F->fin[i * F->N + k];
    r += v;
    for (int a = 0; a < 3; ++a) j[a] += F->L->c[i][a] * v;
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

static void grad_u(const field_t *F, const int *x, double G[3][3] /* G[a][b] = d u_a / d x_b */) {
  double r, u0[3];
  node_moments(F, x, &r, u0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[a][b] = 0.0;
  for (int b = 0; b < F->L->D; ++b) {
    int p1[3] = {x[0], x[1], x[2]}, m1[3] = {x[0], x[1], x[2]};
    int p2[3] = {x[0], x[1], x[2]}, m2[3] = {x[0], x[1], x[2]};
    p1[b] += 1; m1[b] -= 1; p2[b] += 2; m2[b] -= 2;
    int fp = is_fluid(F, p1), fm = is_fluid(F, m1);
    double up1[3], um1[3], up2[3], um2[3];
    if (fp && fm) {
      node_moments(F, p1, &r, up1);
      node_moments(F, m1, &r, um1);
      for (int a = 0; a < 3; ++a) G[a][b] = 0.5 * (up1[a] - um1[a]);
    } else if (fp) {
      node_moments(F, p1, &r, up1);
      if (is_fluid(F, p2)) {
        node_moments(F, p2, &r, up2);
        for (int a = 0; a < 3; ++a) G[a][b] = 0.5 * (-3.0 * u0[a] + 4.0 * up1[a] - up2[a]);
      } else {
        for (int a = 0; a < 3; ++a) G[a][b] = up1[a] - u0[a];
      }
    } else if (fm) {
      node_moments(F, m1, &r, um1);
      if (is_fluid(F, m2)) {
        node_moments(F, m2, &r, um2);
        for (int a = 0; a < 3; ++a) G[a][b] = 0.5 * (3.0 * u0[a] - 4.0 * um1[a] + um2[a]);
      } else {
        for (int a = 0; a < 3; ++a) G[a][b] = u0[a] - um1[a];
      }
    }
  }
}

/* Grad's approximation, Eq. (grad), for direction i. */
static double grad_pop(const lat_t *L, int i, double rho, const double *u, const double Pi[3][3]) {
  const double cs2 = 1.0 / 3.0;
  double cu = 0.0;
  for (int a = 0; a < 3; ++a) cu += L->c[i][a] * u[a];
  double contr = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double A = Pi[a][b] - (a == b ? rho * cs2 : 0.0);
      double B = L->c[i][a] * L->c[i][b] - (a == b ? cs2 : 0.0);
      contr += A * B;
    }
  return L->w[i] * (rho + rho * cu / cs2 + contr / (2.0 * cs2 * cs2));
}

/* Fluid stress at a node from its pre-collision populations f (section
 * "Fluid-structure coupling": sigma_f = -p I - (1 - beta) Pi^(1)), with the
 * pressure relative to the rest state, p = (rho - 1) c_s^2, and
 * Pi^(1) = Pi - Pi_eq, both second moments summed over the populations and
 * over the entropic equilibrium of (rho, u).  out: xx, yy, zz, xy, xz, yz
 * (zz = 0 on D2Q9), then 1. */
static void node_stress(const lat_t *L, int lat, double beta, const double *f, double *out) {
  double rho = 0.0, j[3] = {0, 0, 0};
  for (int i = 0; i < L->Q; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * f[i];
  }
  double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double feq[MAXQ];
  or_equilibrium(lat, rho, u, feq);
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  const double p = (rho - 1.0) / 3.0;
  for (int m = 0; m < 6; ++m) {
    double P = 0.0, E = 0.0;
    for (int i = 0; i < L->Q; ++i) {
      const double cc = (double)(L->c[i][ia[m]] * L->c[i][ib[m]]);
      P += cc * f[i];
      E += cc * feq[i];
    }
    out[m] = (m < 3 ? -p : 0.0) - (1.0 - beta) * (P - E);
  }
  if (L->D == 2) out[2] = 0.0;
  out[6] = 1.0;
}

/* One time step with boundaries.
 *  bc[6], face_u[6][3]: face kinds / velocities; inlet_u: per face an array
 *  [3][face nodes] (NULL entries: face_u is used), scaled by inlet_scale.
 *  solid[n]: immersed solid mask (interior); surface: mesh for link data.
 *  fin/fout: [Q][n] post-collision states (fout of solid nodes is set to 0).
 *  vforce[nv][3] and bforce[nb][3] are overwritten with the momentum-exchange
 *  force of this step (may be NULL).  sigma[n][7] (may be NULL): at every
 *  fluid node with an immersed solid neighbour the fluid stress of its
 *  pre-collision populations (node_stress), other nodes untouched.
 *  Returns the number of immersed links. */
int or_step_bc(int lat, int nx, int ny, int nz, double beta, int mode, const int *bc,
               const double *face_u, const double *const *inlet_u, double inlet_scale,
               const uint8_t *solid, int nv, int ne, int nb, const double *vx, const double *vv,
               const int32_t *el, const int32_t *eb, const double *fin, double *fout,
               double *vforce, double *bforce, double *sigma) {
  lat_t L;
  if (lat_make(lat, &L)) return -1;
  field_t F;
  F.L = &L;
  F.n[0] = nx; F.n[1] = ny; F.n[2] = nz;
  for (int a = 0; a < 3; ++a) F.periodic[a] = (bc[2 * a] == BC_PERIODIC);
  if (L.D == 2) F.periodic[2] = 1;
  F.solid = solid;
  F.fin = fin;
  F.N = (long)nx * ny * nz;
  surf_t S = {L.D, nv, ne, nb, vx, vv, el, eb};
  if (vforce) memset(vforce, 0, sizeof(double) * 3 * (size_t)nv);
  if (bforce) memset(bforce, 0, sizeof(double) * 3 * (size_t)nb);
  int nlinks = 0;
  const int Q = L.Q;

  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int xb[3] = {x, y, z};
        long k = nid(&F, xb);
        if (solid[k]) {
          for (int i = 0; i < Q; ++i) fout[i * F.N + k] = 0.0;
          continue;
        }
        double f[MAXQ];
        int miss[MAXQ], face_of[MAXQ];
        int nmiss = 0;
        for (int i = 0; i < Q; ++i) {
          int p[3] = {x - L.c[i][0], y - L.c[i][1], z - L.c[i][2]};
          miss[i] = 0;
          face_of[i] = -1;
          for (int a = 0; a < 3; ++a) {
            if (!F.periodic[a] && (p[a] < 0 || p[a] >= F.n[a])) {
              /* first crossed face in axis order */
              if (face_of[i] < 0) face_of[i] = 2 * a + (p[a] < 0 ? 0 : 1);
            }
          }
          if (face_of[i] >= 0) {
            miss[i] = 1;
          } else {
            in_domain(&F, p);
            long ks = nid(&F, p);
            if (solid[ks]) miss[i] = 1;
            else f[i] = fin[i * F.N + ks];
          }
          nmiss += miss[i];
        }
        if (nmiss) {
          /* ---- targets */
          int open_face = -1;
          for (int fc = 0; fc < 6 && open_face < 0; ++fc)
            for (int i = 0; i < Q; ++i)
              if (miss[i] && face_of[i] == fc &&
                  (bc[fc] == BC_INLET || bc[fc] == BC_OUTLET || bc[fc] == BC_FREESTREAM)) {
                open_face = fc;
                break;
              }
          double q[MAXQ], uw[MAXQ][3], vwt[MAXQ][3];
          int hit[MAXQ], vid[MAXQ][3];
          for (int i = 0; i < Q; ++i) {
            hit[i] = -1;
            if (!miss[i]) continue;
            if (face_of[i] >= 0) {
              q[i] = 0.5;
              for (int a = 0; a < 3; ++a) uw[i][a] = face_u[3 * face_of[i] + a];
            } else {
              double xbd[3] = {x + 0.5, y + 0.5, z + 0.5};
              hit[i] = link_hit(&S, xbd, L.c[i], &q[i], uw[i], vid[i], vwt[i]);
              if (hit[i] < 0) { /* no crossing found: treat as a wall half-way, at rest */
                q[i] = 0.5;
                uw[i][0] = uw[i][1] = uw[i][2] = 0.0;
              } else {
                nlinks++;
              }
            }
          }
          double rho_t, ut[3] = {0, 0, 0};
          int zero_grad = 0;
          if (open_face >= 0) {
            /* the interior neighbour across the open face */
            const int ax = open_face / 2;
            int xin[3] = {x, y, z};
            xin[ax] += (open_face % 2 == 0) ? 1 : -1;
            double r0 = 1.0, u0[3] = {0, 0, 0};
            if (is_fluid(&F, xin)) node_moments(&F, xin, &r0, u0);
            else node_moments(&F, xb, &r0, u0);
            if (bc[open_face] == BC_INLET) {
              const double *prof = inlet_u ? inlet_u[open_face] : NULL;
              if (prof) {
                long fidx, fn;
                if (ax == 0) { fidx = (long)z * ny + y; fn = (long)ny * nz; }
                else if (ax == 1) { fidx = (long)z * nx + x; fn = (long)nx * nz; }
                else { fidx = (long)y * nx + x; fn = (long)nx * ny; }
                for (int a = 0; a < L.D; ++a) ut[a] = inlet_scale * prof[a * fn + fidx];
              } else {
                for (int a = 0; a < L.D; ++a) ut[a] = inlet_scale * face_u[3 * open_face + a];
              }
              rho_t = r0;
            } else if (bc[open_face] == BC_OUTLET) {
              for (int a = 0; a < 3; ++a) ut[a] = u0[a];
              rho_t = 1.0;
            } else {
              for (int a = 0; a < L.D; ++a) ut[a] = face_u[3 * open_face + a];
              rho_t = 1.0;
              zero_grad = 1;
            }
          } else {
            rho_t = 0.0;
            for (int i = 0; i < Q; ++i) {
              if (!miss[i]) { rho_t += f[i]; continue; }
              double cuw = 0.0;
              for (int a = 0; a < 3; ++a) cuw += L.c[i][a] * uw[i][a];
              rho_t += fin[(Q - 1 - i) * F.N + k] + 6.0 * L.w[i] * cuw;
              int pn[3] = {x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]};
              double ui[3];
              if (is_fluid(&F, pn)) {
                double rn, un[3];
                node_moments(&F, pn, &rn, un);
                for (int a = 0; a < 3; ++a) ui[a] = (uw[i][a] + q[i] * un[a]) / (1.0 + q[i]);
              } else {
                for (int a = 0; a < 3; ++a) ui[a] = uw[i][a];
              }
              for (int a = 0; a < 3; ++a) ut[a] += ui[a] / nmiss;
            }
          }
          double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          if (!zero_grad) grad_u(&F, xb, G);
          double Pi[3][3];
          const double cs2 = 1.0 / 3.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double eq = (a == b ? rho_t * cs2 : 0.0) + rho_t * ut[a] * ut[b];
              double neq = -rho_t * cs2 / (2.0 * beta) * (G[a][b] + G[b][a]);
              Pi[a][b] = eq + neq;
            }
          for (int i = 0; i < Q; ++i) {
            if (!miss[i]) continue;
            f[i] = grad_pop(&L, i, rho_t, ut, Pi);
            if (hit[i] >= 0) {
              /* gauge form: the reference state f = W (uniform ambient
               * pressure rho0 c_s^2) is taken out of both populations */
              double fo = fin[(Q - 1 - i) * F.N + k] - L.w[i];
              int body = eb[hit[i]];
              for (int a = 0; a < L.D; ++a) {
                double Fa = -L.c[i][a] * (fo + (f[i] - L.w[i]));
                if (bforce) bforce[3 * body + a] += Fa;
                if (vforce)
                  for (int m = 0; m < L.D; ++m) vforce[3 * vid[i][m] + a] += vwt[i][m] * Fa;
              }
            }
          }
        }
        if (sigma) {
          int immersed = 0;
          for (int i = 0; i < Q; ++i) immersed |= miss[i] && face_of[i] < 0;
          if (immersed) node_stress(&L, lat, beta, f, sigma + 7 * k);
        }
        double fo[MAXQ];
        or_collide(lat, beta, mode, f, fo, NULL, NULL, NULL, NULL);
        for (int i = 0; i < Q; ++i) fout[i * F.N + k] = fo[i];
      }
  return nlinks;
}

/* Immersed cut links of a static configuration: for every fluid node x_b and
 * direction i whose source x_b - c_i is solid, the crossing found by
 * link_hit.  Writes up to cap entries: node (linear interior index), i, q,
 * element, and the wall velocity; returns the number of links (may exceed
 * cap).  Periodic wrap is applied to the source node only (the link itself is
 * taken in unwrapped coordinates, as in or_step_bc). */
int or_links(int lat, int nx, int ny, int nz, const int *periodic, const uint8_t *solid, int nv,
             int ne, int nb, const double *vx, const double *vv, const int32_t *el,
             const int32_t *eb, int cap, int32_t *node, int32_t *dir, double *q, int32_t *elem,
             double *uw) {
  lat_t L;
  if (lat_make(lat, &L)) return -1;
  surf_t S = {L.D, nv, ne, nb, vx, vv, el, eb};
  int n[3] = {nx, ny, nz};
  int cnt = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long k = ((long)z * ny + y) * nx + x;
        if (solid[k]) continue;
        for (int i = 0; i < L.Q; ++i) {
          int p[3] = {x - L.c[i][0], y - L.c[i][1], z - L.c[i][2]};
          int out = 0;
          for (int a = 0; a < 3; ++a) {
            if (p[a] < 0 || p[a] >= n[a]) {
              if (!periodic[a]) out = 1;
              else p[a] = ((p[a] % n[a]) + n[a]) % n[a];
            }
          }
          if (out) continue;
          if (!solid[((long)p[2] * ny + p[1]) * nx + p[0]]) continue;
          double xb[3] = {x + 0.5, y + 0.5, z + 0.5}, qq, u[3];
          int vid[3];
          double vw[3];
          int e = link_hit(&S, xb, L.c[i], &qq, u, vid, vw);
          if (cnt < cap) {
            node[cnt] = (int32_t)k;
            dir[cnt] = i;
            q[cnt] = e >= 0 ? qq : -1.0;
            elem[cnt] = e;
            for (int a = 0; a < 3; ++a) uw[3 * cnt + a] = e >= 0 ? u[a] : 0.0;
          }
          cnt++;
        }
      }
  return cnt;
}

/* Nodes that leave the solid when the surface moves ("fresh" nodes; the
 * paper accounts for the mass swept by the object through the target
 * density, the state of uncovered nodes is left open).  Reading: a node with
 * old_solid = 1 and new_solid = 0 is set to the entropic equilibrium of
 * rho_bar = mean density of its neighbours x + c_i (i not the rest
 * direction) that are fluid in the new mask and not fresh themselves (1 if
 * none), and of the velocity of the nearest surface vertex (lowest index on
 * ties).  f is the post-collision state [Q][n], updated in place.  Returns
 * the number of fresh nodes. */
int or_fresh_init(int lat, int nx, int ny, int nz, const int *periodic, const uint8_t *old_solid,
                  const uint8_t *new_solid, int nv, const double *vx, const double *vv, double *f) {
  lat_t L;
  if (lat_make(lat, &L)) return -1;
  field_t F;
  F.L = &L;
  F.n[0] = nx; F.n[1] = ny; F.n[2] = nz;
  for (int a = 0; a < 3; ++a) F.periodic[a] = periodic[a];
  F.solid = new_solid;
  F.fin = f;
  F.N = (long)nx * ny * nz;
  int nfresh = 0;
  for (long k = 0; k < F.N; ++k)
    if (old_solid[k] && !new_solid[k]) nfresh++;
  if (!nfresh) return 0;
  double *rho_bar = (double *)malloc(sizeof(double) * nfresh);
  long *idx = (long *)malloc(sizeof(long) * nfresh);
  int m = 0;
  for (long k = 0; k < F.N; ++k) {
    if (!(old_solid[k] && !new_solid[k])) continue;
    int p0[3] = {(int)(k % nx), (int)((k / nx) % ny), (int)(k / ((long)nx * ny))};
    double rs = 0.0;
    int rn = 0;
    for (int i = 0; i < L.Q; ++i) {
      if (!L.c[i][0] && !L.c[i][1] && !L.c[i][2]) continue;
      int p[3] = {p0[0] + L.c[i][0], p0[1] + L.c[i][1], p0[2] + L.c[i][2]};
      if (!in_domain(&F, p)) continue;
      long kn = nid(&F, p);
      if (new_solid[kn]) continue;
      if (old_solid[kn]) continue; /* fresh itself */
      double r, u[3];
      node_moments(&F, p, &r, u);
      rs += r;
      rn++;
    }
    rho_bar[m] = rn ? rs / rn : 1.0;
    idx[m] = k;
    m++;
  }
  for (int q = 0; q < nfresh; ++q) {
    long k = idx[q];
    double p[3] = {(k % nx) + 0.5, ((k / nx) % ny) + 0.5, (k / ((long)nx * ny)) + 0.5};
    int best = 0;
    double bd = 1e300;
    for (int v = 0; v < nv; ++v) {
      double d2 = 0.0;
      for (int a = 0; a < L.D; ++a) {
        double dd = vx[L.D * v + a] - p[a];
        d2 += dd * dd;
      }
      if (d2 < bd) { bd = d2; best = v; }
    }
    double u[3] = {0, 0, 0}, feq[MAXQ];
    for (int a = 0; a < L.D; ++a) u[a] = vv[L.D * best + a];
    or_equilibrium(lat, rho_bar[q], u, feq);
    for (int i = 0; i < L.Q; ++i) f[i * F.N + k] = feq[i];
  }
  free(rho_bar);
  free(idx);
  return nfresh;
}
