/*
 * kbc_lbm.h -- C ABI of the GB300 (sm_103a) entropic lattice Boltzmann
 * library for fluid-structure interaction.
 *
 * Method: Dorschner, Chikatamarla & Karlin, "Fluid-structure interaction with
 * the entropic lattice Boltzmann method" (arXiv 1710.02375):
 *   - fluid step: KBC collide-and-stream, Eqs. (f_equations), (popSplit),
 *     (f_mirr), (feq_min), (conservationLaws), (gamma_min_approx); viscosity
 *     nu = c_s^2 (1/(2 beta) - 1/2), Eq. (visc);
 *   - moving walls: Grad's approximation for missing populations, Eq. (grad),
 *     with target values (section "Fluid boundary conditions");
 *   - force on the structure (section "Solid boundary conditions").
 *
 * General rules for every call:
 *   - All arguments are plain pointers and sizes.  A pointer argument may be
 *     host memory or device memory of the context's device; the library tells
 *     them apart with cudaPointerGetAttributes.  Caller-owned arrays are only
 *     read (inputs) or written (outputs) during the call; the library keeps
 *     no reference to them.  Exception: a call documented as asynchronous
 *     (lbm_update_surface) reads device or page-locked host inputs in the
 *     order of the context's stream, after it returns; keep them unchanged
 *     until the stream has passed the call.  Device inputs must be complete
 *     when the call is made: work that writes them on another stream has to
 *     be finished or ordered before the context's stream.
 *   - Work runs in order on one CUDA stream (the caller's, given in
 *     lbm_config.stream, or one the library creates).  lbm_step returns
 *     without waiting for the GPU; every lbm_get_* call waits for the stream.
 *   - Every call returns an lbm_status.  On failure lbm_last_error() gives a
 *     one-line message.  A CUDA error poisons the context: every later call
 *     except lbm_last_error/lbm_destroy returns LBM_ESTATE.
 *   - A context belongs to the CUDA device that is current when lbm_create
 *     runs; calls on a context with another device current return
 *     LBM_EINVAL.
 *   - Units are lattice units (dx = dt = 1).
 *
 * Population layout (the interface layout of every populations array):
 *   structure of arrays f[i][z][y][x] with x fastest, interior nodes only,
 *   direction index i = (cz+1)*9 + (cy+1)*3 + (cx+1) for D3Q27 and
 *   i = (cy+1)*3 + (cx+1) for D2Q9 (nz = 1); the opposite direction of i is
 *   Q-1-i.  Weights are tensor products of (1/6, 2/3, 1/6).
 */
#ifndef KBC_LBM_H
#define KBC_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* bad argument */
  LBM_ENOMEM = -2,    /* workspace too small or allocation failed */
  LBM_ECUDA = -3,     /* CUDA runtime error (context poisoned) */
  LBM_EUNSTABLE = -4, /* non-finite or non-positive density met */
  LBM_ETIMEOUT = -5,  /* a bounded device wait gave up */
  LBM_ECAPACITY = -6, /* a fixed-capacity buffer overflowed */
  LBM_ESTATE = -7     /* context poisoned by an earlier error, or wrong call order */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q27 = 27 };

/* Storage of populations in device memory (computation in FP32 except F64):
 *   F32  stores f_i - W_i        (deviation from the lattice weight)
 *   F16  stores f_i / W_i - 1    (scaled deviation, IEEE half, round to nearest even)
 *   BF16 stores f_i / W_i - 1    (scaled deviation, bfloat16, round to nearest even)
 *   F16N stores f_i / W_i - 1    (scaled deviation, 16-bit float with the
 *        exponent range narrowed to [2^-6, 2): sign, 3 exponent bits, 12
 *        stored significand bits, evenly spaced steps of 2^-18 below 2^-6;
 *        round to nearest, ties away from zero; |f_i/W_i - 1| >= 2 saturates).
 *        The same bytes as F16 with a step four times finer for the O(u)
 *        deviations.
 *   F64  stores f_i - W_i in double precision and computes the sweep and
 *        the boundary fill in FP64 (D2Q9 only; the test storage).  Inputs
 *        kept in FP32 by the boundary data (link fractions, wall and face
 *        velocities, inlet profiles) stay FP32. */
enum { LBM_STORE_F32 = 0, LBM_STORE_F16 = 1, LBM_STORE_BF16 = 2, LBM_STORE_F64 = 3,
       LBM_STORE_F16N = 4 };

/* Collision: KBC (entropic multi-relaxation time, gamma from
 * Eq. gamma_min_approx) or BGK (gamma fixed to 2, i.e. LBGK with omega = 2 beta). */
enum { LBM_COLLIDE_KBC = 0, LBM_COLLIDE_BGK = 1 };

/* Face boundary kinds, faces ordered -x, +x, -y, +y, -z, +z. */
enum {
  LBM_BC_PERIODIC = 0,   /* both faces of the axis must be periodic */
  LBM_BC_WALL = 1,       /* planar no-slip wall half a cell outside the face (Grad, q = 1/2),
                            moving with face_velocity */
  LBM_BC_INLET = 2,      /* prescribed velocity (face_velocity, or the per-node profile) */
  LBM_BC_OUTLET = 3,     /* rho = 1, velocity extrapolated from the interior */
  LBM_BC_FREESTREAM = 4  /* rho = 1, u = face_velocity, no velocity gradient */
};

typedef struct {
  int lattice;            /* LBM_D2Q9 or LBM_D3Q27 */
  int nx, ny, nz;         /* interior nodes; nz = 1 for D2Q9 */
  double beta;            /* relaxation parameter in (0,1); nu = (1/(2 beta) - 1/2)/3, Eq. (visc) */
  int storage;            /* LBM_STORE_* */
  int collision;          /* LBM_COLLIDE_* */
  int bc[6];              /* LBM_BC_* per face */
  double face_velocity[6][3]; /* wall / inlet / free-stream velocity per face */
  int max_links;          /* capacity of the cut-link list (0: no immersed bodies) */
  int max_vertices;       /* capacity of surface-mesh vertices over all bodies */
  int max_elements;       /* capacity of surface-mesh elements over all bodies */
  int inlet_ramp_steps;   /* inlet velocity ramp (1 - cos(pi t/T))/2 over T steps, 0: none */
  void *stream;           /* cudaStream_t to run on; NULL: the library creates one */
  int multiphase;         /* 1: reserve the fields of the multiphase model (lbm_set_multiphase) */
} lbm_config;

/* Bytes of device workspace lbm_create needs for this configuration. */
lbm_status lbm_workspace_size(const lbm_config *cfg, size_t *bytes);

/* Create a context.  workspace: device memory of at least
 * lbm_workspace_size() bytes, 256-byte aligned, owned by the caller and kept
 * alive until lbm_destroy; NULL makes the library allocate (and free) it with
 * cudaMalloc.  The populations start at rest: f_i = W_i. */
lbm_status lbm_create(const lbm_config *cfg, void *workspace, size_t workspace_bytes,
                      lbm_ctx **out);

/* Set every interior node to the entropic equilibrium of the given density
 * rho[nz][ny][nx] and velocity u[dim][nz][ny][nx] (FP64), Eq. (feq_min). */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u);

/* Set / get the populations of all interior nodes as FP64 absolute values in
 * the interface layout f[Q][nz][ny][nx] (post-collision state). */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f);
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f);

/* Advance n time steps: per step, the Grad fill at boundary nodes and the
 * fused pull-stream + KBC collision sweep, Eq. (f_equations).  Asynchronous. */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* ---------------------------------------------------------------------------
 * Boundaries (section "Fluid boundary conditions"): every fluid node with a
 * missing population (its source x - c_i is solid or beyond a non-periodic
 * face) gets Grad's approximation, Eq. (grad), with Pi = Pi_eq + Pi_neq as
 * stated after it, from target values:
 *   wall node: u_t = mean over missing links of (u_w + q u(x_b + c_i))/(1 + q),
 *     rho_t = moving-wall bounce-back density, grad u by finite differences of
 *     the previous-step velocity;
 *   open face (first inlet/outlet/free-stream face crossed): prescribed u and
 *     rho of the next inward node (inlet), rho = 1 and u of the next inward
 *     node (outlet), rho = 1 and the face velocity with grad u = 0 (free stream).
 * ------------------------------------------------------------------------- */

/* Prescribed inlet velocity of face `face` (must be LBM_BC_INLET): u[3][m]
 * FP64, m = the face's node count, indexed by the two other interior
 * coordinates in (z, y, x) order with the face axis removed (face -x: z*ny+y;
 * face -y: z*nx+x; face -z: y*nx+x).  Copied.  Without it the inlet uses
 * face_velocity.  LBM_EINVAL if the face is not an inlet. */
lbm_status lbm_set_inlet_profile(lbm_ctx *ctx, int face, const double *u);

/* Immersed bodies (section "Fluid boundary conditions": the structure's
 * surface mesh passed to the fluid solver).  verts[nv][dim] positions in
 * lattice units (interior node (x,y,z) is the centre of its cell, at
 * (x + 1/2, y + 1/2, z + 1/2); a node on the surface counts as solid), elems[ne][dim]
 * closed polygons (2-D, segments) or closed triangle meshes (3-D),
 * elem_body[ne] in [0, nbodies), vert_vel[nv][dim] wall velocities (NULL:
 * at rest).  Nodes inside a body become solid; cut links (nearest crossing
 * along each lattice link) are built on the device.  band_margin: how far
 * (lattice units) the surface may later move from this position; bodies plus
 * margin must stay 2 nodes inside non-periodic faces (LBM_EINVAL), and at
 * most 16 bodies.  LBM_ECAPACITY if the mesh exceeds max_vertices /
 * max_elements or the links exceed max_links.  Arrays are copied; synchronises. */
lbm_status lbm_set_geometry(lbm_ctx *ctx, int nbodies, const double *verts, int nv,
                            const int32_t *elems, int ne, const int32_t *elem_body,
                            const double *vert_vel, double band_margin);

/* New vertex positions / velocities of the same mesh (moving surface, the
 * coupling step of the conventional serial staggered scheme).  Solid flags
 * and cut links of the band are rebuilt on the device; nodes that leave the
 * solid are set to the entropic equilibrium of the mean density of their
 * fluid neighbours and the velocity of the nearest vertex.  Asynchronous; a
 * link-list overflow is reported by lbm_check as LBM_ECAPACITY. */
lbm_status lbm_update_surface(lbm_ctx *ctx, const double *verts, const double *vert_vel);

/* Momentum-exchange force of the last step on the immersed surface,
 * accumulated in FP64: vert_force[nv][3] (each link's force split over the
 * hit element's vertices by its interpolation weights) and
 * body_force[nbodies][3] totals.  Either may be NULL.  Per link i of fluid
 * node x_b: -c_i (f'_opp(i)(x_b, t-1) + f*_i(x_b, t) - 2 W_i), the momentum
 * exchange relative to the rest state (gauge pressure).  Synchronises. */
lbm_status lbm_get_interface_force(lbm_ctx *ctx, double *vert_force, double *body_force);

/* Force probe that allocates nothing (the paper has no counterpart: this is a
 * service for callers).  Some callers cannot allocate device memory where
 * they need the interface force: code that runs under a device-memory budget
 * fixed at start-up, or on a path that must not call cudaMalloc because it
 * may synchronise the device or fail under memory pressure.  This call gives
 * them the momentum-exchange force the next lbm_step would produce for the
 * current populations and surface: vert_force[nv][3] and
 * body_force[nbodies][3] (either may be NULL; host or device memory), the
 * same quantities lbm_get_interface_force reports after that step.
 * It rebuilds the cut links of the current solid flags and runs the Grad fill
 * and force gather with all scratch (node list, link list, counters, FP64
 * accumulators) in one fixed file-scope device array of about 5.4 MB that
 * every GPU loading the library keeps until the process exits; it calls no
 * cudaMalloc, cudaFree or allocating library routine.  Fixed maxima: 16384
 * surface vertices, 65536 boundary nodes, 65536 cut links; beyond them it
 * returns LBM_ECAPACITY with a message.  The context's device must be
 * current (LBM_EINVAL otherwise): the first call on a device looks up the
 * array's device address for that device (cudaGetSymbolAddress, once per
 * device, safe when several host threads make their first call together).
 * The probe synchronises its stream, so it must not be called while that
 * stream is being captured (LBM_ESTATE).  All calls share the array: calls
 * that overlap on the GPU (several streams or host threads at once) race on
 * it.  The Grad values written into solid slots are the ones the next step
 * writes there anyway.  Synchronises. */
lbm_status lbm_probe_interface_force_static(lbm_ctx *ctx, double *vert_force, double *body_force);

/* info[4] = {face boundary nodes, immersed boundary nodes, cut links,
 * inlet-ramp step counter}.  Synchronises. */
lbm_status lbm_get_boundary_info(lbm_ctx *ctx, int *info);

/* ---------------------------------------------------------------------------
 * Structure (section "Structural modeling"): 2-D geometrically nonlinear
 * co-rotational Euler-Bernoulli beam in FP64 on the GPU, one-step-theta
 * scheme Eq. (timeInt) in the two-field (v, u) form, Newton-Raphson with the
 * constant line-search relaxation lambda (the paper uses 0.7).
 * Element a-b: N = EA (L - L0)/L0, M1 = 2EI/L0 (2 t1 + t2),
 * M2 = 2EI/L0 (t1 + 2 t2), t = nodal rotation minus chord rotation;
 * consistent Hermite mass.  DOFs per node: (ux, uy, theta).
 * ------------------------------------------------------------------------- */
typedef struct fem_ctx fem_ctx;

typedef struct {
  int nn;                 /* beam nodes, 2..48 */
  const double *X;        /* [nn][2] reference node positions (lattice units), copied */
  double EA, EI, rhoA;    /* axial / bending stiffness, mass per length */
  double thickness;       /* flag thickness h (surface offset h/2 each side) */
  const int32_t *fixed;   /* [3 nn] 1 = DOF held at zero, copied */
  double theta;           /* theta of Eq. (timeInt), (0, 1] */
  double lambda;          /* Newton relaxation, (0, 1] */
  double rtol, atol;      /* stop when |R| <= rtol |R_0| + atol */
  int max_it;             /* Newton iteration limit */
  double dt;              /* structural time step (lattice steps) */
  void *stream;           /* cudaStream_t, NULL: library-owned */
  int solve_fp64;         /* 0: Newton matrix and its solve in FP32 (an inexact
                             Newton step: residual, stopping test and state stay
                             FP64); 1: matrix and solve in FP64 (the exact Newton
                             step) */
} fem_beam_config;

lbm_status fem_beam_workspace_size(const fem_beam_config *cfg, size_t *bytes);
/* workspace: device memory of fem_beam_workspace_size() bytes (256-byte
 * aligned, caller-owned) or NULL (cudaMalloc).  State starts at rest. */
lbm_status fem_beam_create(const fem_beam_config *cfg, void *workspace, size_t bytes,
                           fem_ctx **out);
/* One theta-scheme step with nodal loads F1[3 nn] at the new time (the
 * previous call's loads serve as F0).  Asynchronous. */
lbm_status fem_beam_step(fem_ctx *f, const double *F1);
/* u[3nn], v[3nn] (either may be NULL) and the last step's Newton iteration
 * count (negative: not converged within max_it).  Synchronises. */
lbm_status fem_beam_get_state(fem_ctx *f, double *u, double *v, int *iterations);
lbm_status fem_beam_set_state(fem_ctx *f, const double *u, const double *v, const double *F0);
const char *fem_last_error(const fem_ctx *f);
void fem_destroy(fem_ctx *f);

/* ---------------------------------------------------------------------------
 * 3-D structure: co-rotational flat shell for the plate (replaces the paper's
 * Q2 continuum elements of section "Structural modeling"), FP64 on the GPU.
 * Structured nx x ny node grid, node i*ny + j at X[node][3]; element (i, j)
 * joins nodes (i,j), (i+1,j), (i+1,j+1), (i,j+1).  Six DOFs per node:
 * translations (ux, uy, uz) and a rotation, reported as a 3x3 rotation
 * matrix (row-major) and, for velocities and loads, as angular components.
 * Local element: plane-stress membrane and Mindlin bending (2x2 Gauss), MITC4
 * transverse shear, drilling stiffness 1e-3 D; co-rotational frame and
 * projector; lumped mass.  Theta-scheme (Eq. timeInt), Newton with the
 * constant relaxation lambda (stop at |R| <= rtol |R0| + atol, R0 the
 * residual at the step's start), linearised systems by Jacobi-preconditioned
 * conjugate gradients in FP64 to cg_rtol (0: 1e-3, an inexact Newton step;
 * the residual and its stopping test stay FP64, and with lambda = 0.7 the
 * Newton count is the same as with exact solves; 1e-14: the FP64 solve of
 * the exact Newton step) within max_cg iterations (0: 4 x DOFs); one
 * cooperative launch per step.
 * ------------------------------------------------------------------------- */
typedef struct fem_shell_ctx fem_shell_ctx;
typedef struct {
  int nx, ny;             /* nodes along the length and the width, nx*ny <= 4096 */
  const double *X;        /* [nx*ny][3] reference positions (host or device) */
  double E, nu, h, rho;   /* Young's modulus, Poisson ratio, thickness, density */
  const int32_t *fixed;   /* [6 nn] 1: DOF held at its reference value */
  double theta, lambda, rtol, atol;
  int max_it;
  double dt;
  int max_cg;
  double cg_rtol;
  void *stream;           /* cudaStream_t; NULL: library-owned */
} fem_shell_config;
lbm_status fem_shell_workspace_size(const fem_shell_config *c, size_t *bytes);
lbm_status fem_shell_create(const fem_shell_config *c, void *workspace, size_t bytes,
                            fem_shell_ctx **out);
/* One structural step with loads F1[nn][6] (forces, then moments; global
 * axes); the previous step's loads are kept (zero before the first step). */
lbm_status fem_shell_step(fem_shell_ctx *s, const double *F1);
/* u[nn][3], R[nn][9], v[nn][6] (translational, angular) and iters[2]
 * (Newton iterations of the last step, negative when max_it was reached;
 * conjugate-gradient iterations of that step); NULL skips.  Synchronises. */
lbm_status fem_shell_get_state(fem_shell_ctx *s, double *u, double *R, double *v, int *iters);
lbm_status fem_shell_set_state(fem_shell_ctx *s, const double *u, const double *R,
                               const double *v, const double *F0);
const char *fem_shell_last_error(const fem_shell_ctx *s);
void fem_shell_destroy(fem_shell_ctx *s);

/* ---------------------------------------------------------------------------
 * The paper's structural model (section "Structural modeling"), FP64 on the
 * GPU: total-Lagrangian St Venant-Kirchhoff continuum, S = lambda tr(E) I +
 * 2 mu E, E = (F^T F - I) / 2, P = F S, lambda and mu from E and nu by the
 * printed Lame relations; Q2 Lagrange elements (dim 2: 9-node
 * quadrilaterals in plane strain; dim 3: 27-node hexahedra), the geometry
 * mapped from each element's corner nodes by the bilinear (trilinear) map,
 * 3 Gauss points per axis; consistent mass (rho psi, psi).
 * Time step: the two-field theta scheme of Eq. (timeInt) for v and u.  The
 * displacement equation is linear, so v1 is eliminated and Newton runs on
 * u1 with the residual G(u) = M (u - u0 - dt v0) / (theta dt^2) + theta R(u)
 * - theta F1 - (1 - theta) (F0 - R(u0)) and the tangent M / (theta dt^2) +
 * theta A'(u) (the analytic Gateaux derivative printed after Eq.
 * (matrixForm2)); steps relaxed by lambda, stop at |G| <= rtol |G_0| +
 * atol (G_0 at the predictor u0 + dt v0).  Linear systems: Jacobi-
 * preconditioned conjugate gradients on element products to cg_rtol |G|
 * (0: 1e-3, an inexact Newton step; the residual and its stopping test stay
 * FP64, so the converged state is that of exact solves) within max_cg
 * iterations (0: the DOF count).  One cooperative launch per step.
 * Element-local node a = i + 3 j (+ 9 k), i, j, k = 0, 1, 2 along the
 * element's reference axes; nodes are dim-vectors, DOF index node * dim + d.
 * ------------------------------------------------------------------------- */
typedef struct fem_svk_ctx fem_svk_ctx;
typedef struct {
  int dim;                /* 2 or 3 */
  int nn, ne;             /* nodes, elements */
  const double *X;        /* [nn][dim] reference positions (host or device; copied) */
  const int32_t *conn;    /* [ne][3^dim] element nodes (copied); corner-map Jacobians must be > 0 */
  const int32_t *fixed;   /* [nn * dim] 1: DOF held at zero (copied) */
  double E, nu, rho;      /* Young's modulus, Poisson ratio (0 <= nu < 0.5), density */
  double theta, lambda, rtol, atol;
  int max_it;
  double dt;
  int max_cg;
  double cg_rtol;
  void *stream;           /* cudaStream_t; NULL: library-owned */
  int solve_fp64;         /* 0: the element products inside CG in FP32 (residual, stopping
                             test and state stay FP64); 1: in FP64 */
} fem_svk_config;
lbm_status fem_svk_workspace_size(const fem_svk_config *c, size_t *bytes);
/* workspace: device memory (256-byte aligned, caller-owned) or NULL
 * (cudaMalloc).  LBM_EINVAL for a bad config, a node index out of range or
 * an inverted element; LBM_ECUDA when cooperative launch is unavailable.
 * State starts at rest with zero loads. */
lbm_status fem_svk_create(const fem_svk_config *c, void *workspace, size_t bytes,
                          fem_svk_ctx **out);
/* One step with nodal loads F1[nn * dim] at the new time; the previous
 * step's loads serve as F0.  Asynchronous. */
lbm_status fem_svk_step(fem_svk_ctx *s, const double *F1);
/* Consistent nodal loads of a uniform body force per unit mass b[dim]:
 * F[nn * dim] = (rho b, psi_a) (overwritten; host or device).  Synchronises. */
lbm_status fem_svk_body_load(fem_svk_ctx *s, const double *b, double *F);
/* u, v [nn * dim] (either may be NULL) and iters[2]: the last step's Newton
 * iterations (negative: not converged within max_it) and its total CG
 * iterations.  Synchronises. */
lbm_status fem_svk_get_state(fem_svk_ctx *s, double *u, double *v, int *iters);
/* Replace u, v and the loads F0 of the next step (any may be NULL). */
lbm_status fem_svk_set_state(fem_svk_ctx *s, const double *u, const double *v, const double *F0);
const char *fem_svk_last_error(const fem_svk_ctx *s);
void fem_svk_destroy(fem_svk_ctx *s);

/* Couple a plate (fem_shell) to a D3Q27 lattice: the shell's surface
 * occupies vertices [first_vertex, first_vertex + 2 nn) of the geometry --
 * vertex first_vertex + n lies h/2 above node n along the rotated reference
 * normal (the node's rotation applied to (0, 0, 1)), first_vertex + nn + n
 * h/2 below it (the triangles are the caller's).  From then on every
 * lbm_step runs fluid -> forces -> nodal loads (each node: the forces of its
 * two vertices, no moments) -> one shell step -> surface positions and
 * velocities -> geometry, on the lattice stream (create the shell on the
 * lattice's stream).  The surface is set from the shell state at once.
 * s NULL uncouples. */
lbm_status fsi_couple_shell(lbm_ctx *ctx, fem_shell_ctx *s, int first_vertex);

/* Couple a beam to the lattice (conventional serial staggered scheme,
 * section "Fluid-structure coupling"): the beam's flag surface occupies
 * surface vertices [first_vertex, first_vertex + 2 nn) of the geometry given
 * to lbm_set_geometry (bottom edge in node order, then the top edge in
 * reverse node order).  Every lbm_step then runs, on the lattice stream:
 * fluid step with Grad boundaries -> momentum-exchange forces -> nodal loads
 * (sum of the node's two vertex forces; moments about the centre line are
 * not transferred) -> structural step ->
 * new flag vertices and velocities -> solid flags, fresh nodes and cut links.
 * The fem context must stay alive while coupled.  LBM_EINVAL on a bad range. */
lbm_status fsi_couple(lbm_ctx *ctx, fem_ctx *f, int first_vertex);

/* Quasi-two-dimensional coupling of a beam to a D3Q27 lattice (section
 * "Turek Benchmark": a few lattice points spanwise, periodic for the fluid,
 * plane strain for the solid).  The z axis must be periodic; the flag is
 * the beam's polygon extruded along z over [z0, z1] with z0 < 0 and
 * z1 > nz (the closed triangle mesh, end caps included, is the caller's
 * geometry; the caps lie outside the periodic box).  The polygon's vertices
 * at z0 are surface vertices [first_vertex_z0, first_vertex_z0 + 2 nn), those
 * at z1 [first_vertex_z1, first_vertex_z1 + 2 nn), each range in the order of
 * fsi_couple.  Nodal loads are per unit span: the four vertex forces of a
 * beam node summed and divided by nz (the beam's stiffness and mass are per
 * unit span, the plane-strain values for a flag of the paper's kind).  The
 * structural step and the transfer back to the surface are those of
 * fsi_couple.  LBM_EINVAL on a bad lattice, z axis, span or vertex range; no
 * surrogate with this coupling. */
lbm_status fsi_couple_span(lbm_ctx *ctx, fem_ctx *f, int first_vertex_z0, int first_vertex_z1,
                           double z0, double z1);

/* Advance n * repeats steps by replaying a CUDA graph of n steps (n even, so
 * the two population buffers return to their roles).  The graph is captured
 * on the first call and again after any call that changes what a step
 * launches (geometry, coupling, inlet profile, sweep variant) or when n
 * changes.  Same results as lbm_step; no host work per step.  Asynchronous. */
lbm_status lbm_step_graph(lbm_ctx *ctx, int n, int repeats);

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices (same lattice type, storage and stream;
 * any sizes, geometries and couplings) advanced together with one launch per
 * phase: boundary fill + force for all lattices, a persistent sweep whose
 * CTAs take tiles (lattice, rows, 128-node x segment) from an atomic ticket,
 * one CTA per coupled beam, and the geometry rebuild of all moving surfaces.
 * Results equal stepping each lattice on its own (up to the order of FP64
 * force additions).  While batched, step the member contexts only through the
 * batch; the contexts must outlive it.  The paper has no counterpart (its
 * cases are single runs); this serves ensembles.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_workspace_size(lbm_ctx *const *ctxs, int n, size_t *bytes);
/* workspace: device memory (256-byte aligned, caller-owned) or NULL (cudaMalloc). */
lbm_status lbm_batch_create(lbm_ctx *const *ctxs, int n, void *workspace, size_t bytes,
                            lbm_batch **out);
lbm_status lbm_batch_step(lbm_batch *b, int n);
/* n * repeats steps by replaying a CUDA graph of n batched steps (n even). */
lbm_status lbm_batch_step_graph(lbm_batch *b, int n, int repeats);
/* Tile height (rows per tile, 1..64) and resident CTAs per SM of the sweep.
 * Defaults: 5 CTAs per SM; D2Q9 4 rows (gathered together by each
 * thread), D3Q27 1 row. */
lbm_status lbm_batch_set_tuning(lbm_batch *b, int rows_per_tile, int ctas_per_sm);
/* Times every (rows per tile, CTAs per SM) candidate over `steps` batched
 * steps and keeps the fastest; the trial steps advance the simulation. */
lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *best_rows, int *best_ctas,
                              float *best_us_per_step);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* ---------------------------------------------------------------------------
 * MLP for the structural-step surrogate (the paper has no counterpart; it
 * solves every structural step with Newton, section "Structural modeling").
 * Fully connected layers dims[0] -> ... -> dims[n_layers], exact-erf GELU on
 * hidden layers, linear output; BF16 tensor-core GEMMs (mma.sync m16n8k16)
 * with FP32 accumulation, FP32 master parameters, Adam, mean-squared error.
 * Parameter vector layout (FP32): for each layer W[dims[l+1]][dims[l]] then
 * b[dims[l+1]].  Batches are row-major [B][width] FP32, host or device.
 * ------------------------------------------------------------------------- */
typedef struct mlp_ctx mlp_ctx;
typedef struct {
  int n_layers;           /* 1..8 weight layers */
  int dims[9];            /* layer widths, 1..4096 */
  int max_batch;          /* largest batch passed to any call */
  double lr, beta1, beta2, eps;  /* Adam */
  void *stream;           /* cudaStream_t, NULL: library-owned */
} mlp_config;
lbm_status mlp_workspace_size(const mlp_config *cfg, size_t *bytes);
lbm_status mlp_create(const mlp_config *cfg, void *workspace, size_t bytes, mlp_ctx **out);
/* Copy the FP32 parameters in (resets the Adam state) / out.  Synchronise. */
lbm_status mlp_set_params(mlp_ctx *x, const float *params);
lbm_status mlp_get_params(mlp_ctx *x, float *params);
long long mlp_param_count(const mlp_ctx *x);
/* Y[B][dims[n]] = MLP(X[B][dims[0]]).  Synchronises. */
lbm_status mlp_forward(mlp_ctx *x, const float *X, int B, float *Y);
/* Gradients of mean((MLP(X) - Y)^2) w.r.t. the parameters (same layout as
 * the parameter vector) and the loss; no update.  Synchronises. */
lbm_status mlp_gradients(mlp_ctx *x, const float *X, const float *Y, int B, float *grads,
                         float *loss);
/* One Adam step on the batch; loss (may be NULL) of the batch before the
 * step.  Asynchronous when loss is NULL. */
lbm_status mlp_train_step(mlp_ctx *x, const float *X, const float *Y, int B, float *loss);
/* Adam learning rate of the following steps (> 0); keeps the Adam state. */
lbm_status mlp_set_learning_rate(mlp_ctx *x, double lr);
const char *mlp_last_error(const mlp_ctx *x);
void mlp_destroy(mlp_ctx *x);

/* Surrogate for the coupled beam's structural step (no counterpart in the
 * paper).  Each coupled step then builds the network input on the GPU --
 * the out-of-balance loads F(t) - f(u), F(t-1) - f(u), F(t-2) - f(u) (F: the
 * nodal loads, each node's two surface-vertex forces summed, zero moment;
 * f: the internal force at the state u before the step; zero loads before
 * the surrogate was set), then u and v; each block on the 3 nn - 3 free DOFs
 * of nodes 1..nn-1 in (ux, uy, theta) order -- normalises it with in_mean /
 * in_std, runs the network (batch 1) and takes u + dt v + (output * out_std
 * + out_mean) as the Newton initial guess of the structural step.  The guess
 * is accepted when the theta-scheme residual satisfies
 * |R| <= accept_tol |theta F1 + (1 - theta) F0| (free DOFs); otherwise Newton
 * continues from it (FEM fallback) to the usual stopping test, which stays
 * relative to the residual at the start u.  Network: 15 nn - 15 inputs,
 * 3 nn - 3 outputs (LBM_EINVAL otherwise).
 * With a coupled shell (fsi_couple_shell) the same scheme runs on its nf
 * free DOFs (6 per node not held, node-major, in (ux, uy, uz, phix, phiy,
 * phiz) order): input blocks F(t) - f, F(t-1) - f, F(t-2) - f (nodal loads
 * as in fsi_couple_shell; f: the internal force at the state before the
 * step), the state (translations and nodal rotation vectors) and the
 * velocities; output: the step's increment (translations, rotation vector
 * of R1 R0^T) beyond dt v.  Network: 5 nf inputs, nf outputs; the guess is
 * accepted when |R| <= accept_tol |theta F1 + (1 - theta) F0|.
 * mlp NULL removes the surrogate; fsi_couple / fsi_couple_shell remove it
 * too.  The network context must outlive its use by the lattice. */
lbm_status fsi_set_surrogate(lbm_ctx *ctx, mlp_ctx *mlp, const float *in_mean, const float *in_std,
                             const float *out_mean, const float *out_std, double accept_tol);
/* Structural-step counters of the coupled beam or shell since fsi_couple
 * (fsi_couple_shell),
 * fsi_set_surrogate or the last reset: stats[0] guesses accepted, stats[1]
 * guesses rejected, stats[2] Newton solves (linearised systems solved),
 * stats[3] structural steps.  reset != 0 zeroes them after reading.
 * Synchronises. */
lbm_status fsi_get_structure_stats(lbm_ctx *ctx, int stats[4], int reset);

/* Fluid-stress traction on the immersed surfaces (the paper's force path,
 * section "Fluid-structure coupling"; the momentum-exchange force of
 * lbm_get_interface_force is the primary one).  While enabled, every step
 * evaluates sigma_f = -(rho - 1) c_s^2 I - (1 - beta) (Pi - Pi_eq) at the
 * immersed boundary nodes from the step's pre-collision populations (after
 * the Grad fill), gives each surface element the stress of the boundary node
 * nearest to its centroid (ties: lower node index), and integrates
 * t = sigma n over the element (n: outward unit normal of its body in the
 * current configuration; length per unit depth in 2-D, area in 3-D).
 * Outputs (FP64, like lbm_get_interface_force): vert_force[nv][3] (each
 * element's force shared equally by its vertices) and body_force[nbodies][3].
 * lbm_get_traction_force fails with LBM_ESTATE while the output is off.
 * Synchronises. */
lbm_status lbm_set_traction_output(lbm_ctx *ctx, int enable);
lbm_status lbm_get_traction_force(lbm_ctx *ctx, double *vert_force, double *body_force);

/* Density rho[nz][ny][nx] and velocity u[dim][nz][ny][nx] of the current
 * state (FP64 outputs; solid nodes give rho = 0, u = 0).  Synchronises.
 * Field arrays of lbm_init_equilibrium / lbm_get_macros may be device
 * memory, page-locked host memory (cudaHostAlloc, cudaHostRegister; the
 * kernel reads or writes it in place over the host link, no staging copy)
 * or pageable host memory (staged through the workspace in chunks). */
lbm_status lbm_get_macros(lbm_ctx *ctx, double *rho, double *u);
/* The same fields in FP32 (rho = 1 + sum of the stored deviations and
 * u = j / rho formed in FP32; half the bytes of lbm_get_macros).  Same
 * layouts and memory kinds.  Synchronises. */
lbm_status lbm_get_macros_f32(lbm_ctx *ctx, float *rho, float *u);

/* Kernel form of the fused sweep.  AUTO (default) and PAIR: one thread per
 * two neighbouring nodes of a row, the collision of both on the paired FP32
 * instructions (two results per instruction), the c_x = 0 sources as aligned
 * two-element loads and the results as two-element stores.  DIRECT: one
 * thread per node, Q coalesced global loads and stores.  ROWS: a persistent
 * kernel that fetches the Q source rows of every output row into shared
 * memory with bulk asynchronous copies (mbarrier pipeline), when its
 * shared-memory plan fits the device.  ASYNC (FP32 storage): each thread
 * prefetches the 27 source values of its node in the next row with
 * per-thread asynchronous copies into shared memory while it collides the
 * current one (other storage: DIRECT).  DIRECT, ROWS and ASYNC give
 * identical results; PAIR performs the same IEEE operations on the paired
 * instructions and agrees with them to the last bit or so.  In the
 * multiphase model (lbm_set_multiphase) AUTO, DIRECT, ROWS and ASYNC run the
 * one-node forced sweep and PAIR its two-node form.  LBM_EINVAL for an
 * unknown value. */
enum { LBM_SWEEP_AUTO = 0, LBM_SWEEP_DIRECT = 1, LBM_SWEEP_ROWS = 2, LBM_SWEEP_ASYNC = 3,
       LBM_SWEEP_PAIR = 4 };
lbm_status lbm_set_sweep_variant(lbm_ctx *ctx, int variant);

/* ---------------------------------------------------------------------------
 * Multiphase model (section "Extensions to fluid-structure interaction in
 * multiphase flow"): the body force F = F_f of Eq. (Force) (mean-field
 * force, Eqs. (force1) and (Korteweg)) imposed by the exact difference
 * method, Eq. (force_mp), with gamma of Eq. (gamma_min_approx) taken in the
 * shifted entropic product <X|Y> = sum X_i Y_i / feq_i(rho, u + du).
 *
 * Per step: rho(x) = sum_i f_i(x - c_i) (the pulled populations),
 * phi = sqrt(max(rho c_s^2 - p(rho), 0)), lap rho = 6 sum_i W_i (rho(x + c_i)
 * - rho(x)), and at every node
 *     F = 2 phi d(phi) + kappa rho d(lap rho) + rho g,
 *     d_a psi(x) = 3 sum_i W_i c_ia psi(x + c_i)   (isotropic lattice gradient),
 *     du = F / rho,   u = j / rho,
 *     f_i' = f_i - beta (2 ds_i + gamma dh_i) + feq_i(rho, u + du) - feq_i(rho, u).
 * The sign of the capillary term is that of the divergence of the Korteweg
 * tensor (Eq. (force2) prints it negative).  p: LBM_EOS_PAPER, the
 * polynomial of Eq. (eos) (coexisting densities about 7.55 and 0.073), or
 * LBM_EOS_IDEAL, p = rho c_s^2 (phi = 0).  g: a uniform acceleration.
 *
 * Walls: the two faces of one axis may be LBM_BC_WALL at rest (the other
 * faces periodic): the wall nodes get Grad's approximation of their missing
 * populations (the face-wall targets at q = 1/2, with the pre-collision
 * target velocity u - F/(2 rho) of the exact difference method and the
 * velocities of the previous step taken as fluid velocities (j - F/2) /
 * rho), the fields of the stencils are mirrored across the walls, and the
 * wetting force F_s = kappa_w rho sum_i W_i s(x + c_i) c_i (s = 1 beyond a
 * wall; the paper leaves the weights open) is added to F.  kappa_w < 0 is
 * hydrophobic, > 0 hydrophilic.
 *
 * Scope: periodic faces or one pair of walls, no immersed bodies; FP32
 * storage (D2Q9 and D3Q27) or FP64 storage (D2Q9).  The lattice must be
 * created with lbm_config.multiphase = 1 (the workspace then holds the
 * densities and (phi, lap rho) pairs per node in the compute precision).
 *
 * lbm_set_multiphase switches the context to the multiphase step (params
 * copied; NULL switches back to the single-phase step).  LBM_EINVAL for a
 * context outside the scope (other face kinds, moving walls), kappa < 0,
 * non-finite values or an unknown eos; LBM_ESTATE when the context was
 * created without multiphase = 1.
 * While the model is on, lbm_get_macros / lbm_get_macros_f32 return the
 * fluid velocity (j - F/2) / rho of the stored post-collision state, F the
 * force of the step that produced it (F = 0 before the first step and after
 * lbm_init_equilibrium / lbm_set_populations).
 * lbm_get_force_field writes that force, F[3][nz][ny][nx] (FP64; z
 * components zero for D2Q9; host or device memory).  Synchronises. */
enum { LBM_EOS_PAPER = 0, LBM_EOS_IDEAL = 1 };
typedef struct {
  double kappa;   /* capillary coefficient of Eq. (Korteweg), >= 0 */
  int eos;        /* LBM_EOS_* */
  double g[3];    /* uniform acceleration (lattice units) */
  double kappa_w; /* wetting strength of the walls (ignored without walls) */
} lbm_multiphase_params;
lbm_status lbm_set_multiphase(lbm_ctx *ctx, const lbm_multiphase_params *params);
lbm_status lbm_get_force_field(lbm_ctx *ctx, double *F);

/* ---------------------------------------------------------------------------
 * Two-level grid refinement (the multi-domain refinement the validation
 * cases of section "Validation" run on; the paper cites the algorithm
 * without printing it).  D2Q9, FP32 or FP64 storage.
 *
 * A coupled pair: `coarse`, a periodic lattice, and `fine`, a patch at half
 * the spacing over the coarse cells [i0, i0 + nx_f / 2) x [j0, j0 + ny_f / 2)
 * (cell-centred: fine node (p, q) sits at coarse coordinates (i0 + (p +
 * 1/2) / 2, j0 + (q + 1/2) / 2)), with the viscosity of the fine units,
 * nu_f = 2 nu_c, i.e. beta_f = 1 / (2 / beta_c - 1).  lbm_step(coarse, n)
 * then runs n coarse steps of the pair; each:
 *   - the coarse step over every coarse cell;
 *   - two fine steps: the populations a fine boundary node pulls from
 *     outside the patch are Grad's approximation, Eq. (grad), with beta_f,
 *     of the coarse rho, u and grad u (central differences, halved in fine
 *     units) interpolated bicubically to the node and linearly in time to
 *     the fine time level (t + 1/2, t + 1);
 *   - each covered coarse cell is replaced by the cubic midpoint values
 *     (weights -1, 9, 9, -1 over 16 per axis) of the fine density and
 *     momentum and the velocity gradient of the midpoint differences of the
 *     fine velocity (doubled to coarse units; the coarse values of t + 1
 *     beyond the patch), through Grad's approximation with beta_c and the
 *     coarse collision.
 * The covered coarse cells are overwritten each step (their own coarse
 * step only feeds the interpolation); mass is conserved to the interface
 * truncation.
 *
 * Requirements (LBM_EINVAL otherwise): both D2Q9 with the same storage (FP32
 * or FP64), collision and stream; coarse periodic on every face, fine with
 * non-periodic x and y faces (their kinds are ignored: the coupling fills
 * the fine ghost layer), nx_f and ny_f even and >= 4, the patch inside the
 * coarse grid (0 <= i0, i0 + nx_f / 2 <= nx_c, nx_f / 2 <= nx_c - 2, the same
 * for y), beta_f as
 * above to 1e-12; no immersed bodies, beams, shells or multiphase model on
 * either (LBM_ESTATE for a context with those, or one already coupled).
 *
 * lbm_refine_workspace_size: bytes of device scratch for the pair (the
 * coarse fields interpolated to the ring around the patch, and a mask of
 * the covered coarse cells deeper than three cells inside the patch edge,
 * which skip the coarse step: the restriction replaces them).
 * lbm_refine_couple: workspace = device memory of at least that size
 * (256-byte aligned, caller-owned, outliving the coupling) or NULL
 * (cudaMalloc, freed when the pair is uncoupled or the coarse context is
 * destroyed).  fine = NULL uncouples `coarse`.  While coupled, lbm_step and
 * lbm_step_graph on `fine` return LBM_ESTATE (the coarse context steps it);
 * every other call on either context works as before (the fine context's
 * state is its interior nodes).  lbm_check(coarse) also reports a bad
 * density met on the fine patch.  Destroying either context uncouples the
 * pair. */
lbm_status lbm_refine_workspace_size(lbm_ctx *coarse, lbm_ctx *fine, size_t *bytes);
lbm_status lbm_refine_couple(lbm_ctx *coarse, lbm_ctx *fine, int i0, int j0, void *workspace,
                             size_t workspace_bytes);

/* Wait for the stream and report LBM_EUNSTABLE if any sweep since the last
 * check met a non-finite or non-positive density, LBM_ETIMEOUT if a bounded
 * device wait of the row-staged sweep gave up (the affected step is void). */
lbm_status lbm_check(lbm_ctx *ctx);

/* The cudaStream_t the context runs on (for CUDA-event timing by the caller). */
void *lbm_stream(const lbm_ctx *ctx);

const char *lbm_last_error(const lbm_ctx *ctx);
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* KBC_LBM_H */
