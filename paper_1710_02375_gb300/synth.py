"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
draws fields (density, velocity, random population vectors, surface meshes)
that both the CUDA path and the CPU oracle take as inputs.  Each side turns
them into populations with its own code.

Workloads (sizes follow the paper's set-ups in lattice units):
  * Taylor-Green vortex (periodic box): node-centred x = 2 pi (i + 1/2) / N,
      u =  u0 sin x cos y cos z,  v = -u0 cos x sin y cos z,  w = 0,
      rho = 1 + 3 (u0^2/16) (cos 2x + cos 2y)(cos 2z + 2)   (p = rho / 3).
  * Random near-equilibrium population vectors f_i = W_i (1 + a xi_i),
    xi ~ U(-1, 1), for brute-force comparisons on small lattices.
"""
from __future__ import annotations

import numpy as np


def lattice_weights(q: int) -> np.ndarray:
    """Tensor-product D1Q3 weights in the library's direction order
    (x fastest, then y, then z; component -1, 0, +1)."""
    w1 = np.array([1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0])
    if q == 9:
        return np.einsum("y,x->yx", w1, w1).reshape(9)
    if q == 27:
        return np.einsum("z,y,x->zyx", w1, w1, w1).reshape(27)
    raise ValueError(q)


def tgv_fields(nx: int, ny: int, nz: int, u0: float, three_d: bool = True):
    """Taylor-Green vortex density rho[nz,ny,nx] and velocity u[3,nz,ny,nx].

    three_d=False gives the 2-D vortex (uniform in z, rho from the 2-D pressure)."""
    x = 2.0 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2.0 * np.pi * (np.arange(ny) + 0.5) / ny
    z = 2.0 * np.pi * (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    if three_d:
        u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
        u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
        rho = 1.0 + 3.0 * (u0 * u0 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    else:
        u[0] = u0 * np.sin(X) * np.cos(Y)
        u[1] = -u0 * np.cos(X) * np.sin(Y)
        rho = 1.0 + 3.0 * (u0 * u0 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y))
    return rho, u


def random_state(q: int, shape, amp: float, seed: int) -> np.ndarray:
    """Random population field f[q, *shape] = W_i (1 + amp xi), xi ~ U(-1,1)."""
    rng = np.random.default_rng(seed)
    w = lattice_weights(q).reshape((q,) + (1,) * len(shape))
    xi = rng.uniform(-1.0, 1.0, size=(q,) + tuple(shape))
    return w * (1.0 + amp * xi)


def random_macros(shape, u_amp: float, rho_amp: float, seed: int, dim: int = 3):
    """Smooth-free random density and velocity fields (for equilibrium initial states)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, size=shape)
    u = np.zeros((3,) + tuple(shape))
    u[:dim] = u_amp * rng.uniform(-1, 1, size=(dim,) + tuple(shape))
    return rho, u


# ---------------------------------------------------------------- surface meshes
def circle_polygon(cx: float, cy: float, r: float, n: int, phase: float = 0.5):
    """Closed polygon of n segments approximating a circle; vertices at angles
    2 pi (k + phase) / n.  Returns (x[n,2], e[n,2])."""
    t = 2 * np.pi * (np.arange(n) + phase) / n
    x = np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).astype(np.int32)
    return x, e


def rect_polygon(x0: float, y0: float, x1: float, y1: float):
    """Closed counter-clockwise rectangle (x[4,2], e[4,2])."""
    x = np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.float64)
    e = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], dtype=np.int32)
    return x, e


def icosphere(center, r: float, level: int = 2, rotate: float = 0.3):
    """Closed triangulated sphere (subdivided icosahedron, rotated by `rotate`
    radians about a generic axis so no vertex sits on a lattice line).
    Returns (x[nv,3], e[ne,3])."""
    p = (1 + 5 ** 0.5) / 2
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
         (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(a, dtype=np.float64) / np.linalg.norm(a) for a in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    X = np.array(verts)
    ax = np.array([0.48, 0.6, 0.64])
    ax /= np.linalg.norm(ax)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + np.sin(rotate) * K + (1 - np.cos(rotate)) * K @ K
    X = X @ R.T
    return np.asarray(center, dtype=np.float64) + r * X, np.array(faces, dtype=np.int32)


def parabolic_profile(ny: int, u_max: float, noise: float = 0.0, seed: int = 0):
    """Inlet profile u[3, ny] (one x-face column, nz = 1) between walls half a
    cell outside the faces: u_x = 4 u_max (y + 1/2)(H - y - 1/2)/H^2, H = ny,
    times a static multiplicative noise (1 + noise * N(0,1)) drawn once."""
    y = np.arange(ny)
    H = float(ny)
    u = np.zeros((3, ny))
    u[0] = 4 * u_max * (y + 0.5) * (H - y - 0.5) / H ** 2
    if noise:
        rng = np.random.default_rng(seed)
        u[0] *= 1.0 + noise * rng.standard_normal(ny)
    return u


def cylinder_flag_2d(cx=20.0, cy=20.0, d=10.0, flag_len=35.0, flag_h=2.0, n_cyl=64,
                     n_beam=20, with_flag=True):
    """Turek-type rigid cylinder plus an attached flag as closed polygons.

    Body 0: cylinder of diameter d (n_cyl segments).  Body 1: the flag, a
    rectangle of length flag_len and thickness flag_h whose centre line runs
    from the cylinder's downstream side x0 = cx + sqrt(r^2 - (h/2)^2) to
    cx + r + flag_len at y = cy, with n_beam + 1 vertices on each long edge
    (one per beam node).  Returns (x[nv,2], e[ne,2], body[ne], beam_x[n_beam+1])."""
    r = d / 2
    xc, ec = circle_polygon(cx, cy, r, n_cyl)
    if not with_flag:
        return xc, ec, np.zeros(len(ec), np.int32), None
    x0 = cx + np.sqrt(r * r - (flag_h / 2) ** 2)
    x1 = cx + r + flag_len
    bx = np.linspace(x0, x1, n_beam + 1)
    bot = np.stack([bx, np.full_like(bx, cy - flag_h / 2)], axis=1)
    top = np.stack([bx[::-1], np.full_like(bx, cy + flag_h / 2)], axis=1)
    xf = np.concatenate([bot, top])
    nf = len(xf)
    ef = np.stack([np.arange(nf), (np.arange(nf) + 1) % nf], axis=1).astype(np.int32)
    x = np.concatenate([xc, xf])
    e = np.concatenate([ec, ef + len(xc)])
    body = np.array([0] * len(ec) + [1] * len(ef), dtype=np.int32)
    return x, e, body, bx


def c1_flag_beam(cx=20.0, cy=20.0, d=10.0, flag_len=35.0, flag_h=2.0, n_beam=20, u_max=0.05,
                 Ae=1.4e3, density_ratio=10.0):
    """Beam data of the C1 flag: reference nodes X[n_beam+1, 2] on the centre
    line, EA, EI, rhoA per unit depth (E from the aeroelastic number
    Ae = E / (rho_f U_mean^2), U_mean = 2/3 u_max, rho_f = 1) and the clamped
    root mask."""
    r = d / 2
    x0 = cx + np.sqrt(r * r - (flag_h / 2) ** 2)
    x1 = cx + r + flag_len
    X = np.stack([np.linspace(x0, x1, n_beam + 1), np.full(n_beam + 1, cy)], axis=1)
    U = 2.0 / 3.0 * u_max
    E = Ae * U * U
    A, I = flag_h, flag_h ** 3 / 12.0
    fixed = np.zeros(3 * (n_beam + 1), np.int32)
    fixed[:3] = 1
    return X, E * A, E * I, density_ratio * A, fixed



def flag_channel(s, Re, Ae=1.4e3, seed=0, n_cyl=48, n_beam=20, u_max=0.05):
    """One flag-in-channel case at scale s: nx = round(200 s), ny = round(40 s),
    cylinder of diameter D = ny / 4.1 at (2D, 2D), flag of length 3.5 D and
    thickness 0.2 D (n_beam beam elements), parabolic inflow u_max with 1e-4
    static noise (seed), Re on the mean inflow speed 2/3 u_max and D,
    aeroelastic number Ae, density ratio 10.  Returns a dict with the lattice
    size, beta, inflow profile, surface mesh (cylinder then flag) and beam
    data."""
    nx, ny = int(round(200 * s)), int(round(40 * s))
    D = ny / 4.1
    U = 2.0 / 3.0 * u_max
    nu = U * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof = parabolic_profile(ny, u_max, noise=1e-4, seed=seed)
    x, e, body, _ = cylinder_flag_2d(cx=2 * D, cy=2 * D, d=D, flag_len=3.5 * D, flag_h=0.2 * D,
                                     n_cyl=n_cyl, n_beam=n_beam)
    X, EA, EI, rhoA, fixed = c1_flag_beam(cx=2 * D, cy=2 * D, d=D, flag_len=3.5 * D,
                                          flag_h=0.2 * D, n_beam=n_beam, u_max=u_max, Ae=Ae)
    return dict(nx=nx, ny=ny, beta=beta, Re=Re, Ae=Ae, D=D, inlet=prof, x=x, e=e, body=body,
                ncyl=n_cyl, beam=(X, EA, EI, rhoA, fixed), h=0.2 * D)


def c5_case(Re, seed=0):
    """The surrogate workload: the flag channel at scale 4 (800 x 160,
    D = 39.0), a 31-element flag (32 beam nodes, 64 surface vertices)."""
    return flag_channel(4.0, Re, seed=seed, n_beam=31)


def c4_instances(n=64, seed=0, n_cyl=48, n_beam=20, u_max=0.05, Ae0=1.4e3):
    """The batched ensemble: n flag-in-channel instances.  Instance k draws
    (seed + k) a scale s ~ U[1, 4] (nx = round(200 s), ny = round(40 s), so
    domains span 200x40 .. 800x160), Re ~ U[50, 200] on the cylinder diameter
    D = ny / 4.1 with the cylinder at (2D, 2D), a flag of length 3.5 D and
    thickness 0.2 D, and an aeroelastic number Ae log-uniform on
    [Ae0 / sqrt(10), Ae0 sqrt(10)] (stiffness over one decade).  Returns a
    list of dicts with the lattice size, beta, inflow profile, surface mesh
    (cylinder then flag) and beam data."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        s = rng.uniform(1.0, 4.0)
        Re = rng.uniform(50.0, 200.0)
        Ae = Ae0 * 10 ** rng.uniform(-0.5, 0.5)
        out.append(flag_channel(s, Re, Ae=Ae, seed=seed + k, n_cyl=n_cyl, n_beam=n_beam,
                                u_max=u_max))
    return out


def plate_surface(nx, ny):
    """Closed triangle mesh of a thin plate around an nx x ny node mid-surface
    grid (node i*ny + j): top vertices 0..nn-1 (vertex n above node n),
    bottom vertices nn..2nn-1, two triangles per top and bottom quad and per
    side quad of the rim, all wound with the outward normal for a plate whose
    mid-surface normal is (i, j) -> x_i cross y_j.  Returns e[ne, 3]."""
    nn = nx * ny

    def nid(i, j):
        return i * ny + j
    tri = []
    for i in range(nx - 1):
        for j in range(ny - 1):
            a, b, c, d = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
            tri += [(a, b, c), (a, c, d)]                                  # top, normal +n
            tri += [(nn + a, nn + c, nn + b), (nn + a, nn + d, nn + c)]    # bottom, normal -n
    rim = ([nid(i, 0) for i in range(nx)] + [nid(nx - 1, j) for j in range(1, ny)] +
           [nid(i, ny - 1) for i in range(nx - 2, -1, -1)] + [nid(0, j) for j in range(ny - 2, 0, -1)])
    for k in range(len(rim)):
        p, q = rim[k], rim[(k + 1) % len(rim)]
        tri += [(p, nn + p, nn + q), (p, nn + q, q)]
    return np.array(tri, dtype=np.int32)


def plate_case(nxl=256, nyl=128, nzl=128, L=40.0, b=20.0, h=2.0, x0=64.0, u_in=0.04, Re=400.0,
               K_B=1e-4, nu_s=0.4, density_ratio=None, ex=16, ey=8, perturb=1e-3):
    """The plate-in-crossflow case: D3Q27 channel nxl x nyl x nzl, inflow
    u_in along +x (-x face), outlet on +x, periodic in y (span), free stream
    on the z faces; a plate of length L (x), width b (y), thickness h (z),
    clamped at its leading edge x = x0, centred in y and z, as an ex x ey
    element flat shell.  Re = u_in L / nu; bending number
    K_B = E h^3 / (12 (1 - nu_s^2) rho_f u_in^2 L^3); density ratio L / h
    unless given.  Initial shape: a tip deflection perturb * L along z with
    the quadratic profile of a clamped plate, rotations consistent with it.
    Returns a dict (lattice size, beta, bc, face velocities, shell data,
    surface mesh, initial u and R)."""
    nu = u_in * L / Re
    beta = 1.0 / (6 * nu + 1)
    E = K_B * 12 * (1 - nu_s ** 2) * u_in ** 2 * L ** 3 / h ** 3
    rho_s = (L / h) if density_ratio is None else density_ratio
    nx, ny = ex + 1, ey + 1
    zc, yc = nzl / 2.0, nyl / 2.0
    xs = x0 + np.linspace(0.0, L, nx)
    ys = yc + np.linspace(-b / 2, b / 2, ny)
    X = np.array([[x, y, zc] for x in xs for y in ys])
    fixed = np.zeros(6 * nx * ny, np.int32)
    fixed[: 6 * ny] = 1
    xi = (X[:, 0] - x0) / L
    u0 = np.zeros((nx * ny, 3))
    u0[:, 2] = perturb * L * xi ** 2
    th_y = -2.0 * perturb * xi          # slope d(u_z)/dx, rotation about y tilts the normal to -x
    R0 = np.zeros((nx * ny, 3, 3))
    c, s = np.cos(th_y), np.sin(th_y)
    R0[:, 0, 0] = c
    R0[:, 0, 2] = s
    R0[:, 1, 1] = 1.0
    R0[:, 2, 0] = -s
    R0[:, 2, 2] = c
    face_u = np.zeros((6, 3))
    face_u[0, 0] = u_in
    face_u[4, 0] = face_u[5, 0] = u_in
    return dict(nx=nxl, ny=nyl, nz=nzl, beta=beta, bc=(2, 3, 0, 0, 4, 4), face_u=face_u, u_in=u_in,
                shell=dict(X=X, nx=nx, ny=ny, E=E, nu=nu_s, h=h, rho=rho_s, fixed=fixed),
                e=plate_surface(nx, ny), u0=u0, R0=R0, L=L)


def plate_vertices(X, u, R, h):
    """Surface vertices [2 nn, 3] of the plate around the shell state: node
    position plus / minus h/2 times the rotated reference normal (0, 0, 1)."""
    d = R[:, :, 2]
    x = X + u
    return np.concatenate([x + 0.5 * h * d, x - 0.5 * h * d])


def box_surface(lo, hi):
    """Closed triangle mesh of the axis-aligned box [lo, hi] (8 corners, 12
    triangles wound with outward normals).  Returns (x[8,3], e[12,3])."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x = np.array([[(hi if (k >> a) & 1 else lo)[a] for a in range(3)] for k in range(8)])
    # corner k has bit a set when it sits on the hi side of axis a
    quads = [(0, 4, 6, 2), (1, 3, 7, 5),    # x = lo, x = hi
             (0, 1, 5, 4), (2, 6, 7, 3),    # y = lo, y = hi
             (0, 2, 3, 1), (4, 5, 7, 6)]    # z = lo, z = hi
    e = []
    for a, b, c, d in quads:
        e += [(a, b, c), (a, c, d)]
    return x, np.array(e, dtype=np.int32)


def _ear_clip(poly):
    """Triangles (index triples into poly, counter-clockwise) of a simple
    counter-clockwise polygon poly[n,2] by ear clipping."""
    idx = list(range(len(poly)))
    tris = []

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    guard = 0
    while len(idx) > 3 and guard < 100000:
        guard += 1
        for k in range(len(idx)):
            i0, i1, i2 = idx[k - 1], idx[k], idx[(k + 1) % len(idx)]
            a, b, c = poly[i0], poly[i1], poly[i2]
            if cross(a, b, c) <= 0.0:
                continue  # reflex or degenerate corner
            inside = False
            for j in idx:
                if j in (i0, i1, i2):
                    continue
                p = poly[j]
                if cross(a, b, p) >= 0.0 and cross(b, c, p) >= 0.0 and cross(c, a, p) >= 0.0:
                    inside = True
                    break
            if not inside:
                tris.append((i0, i1, i2))
                idx.pop(k)
                break
    tris.append(tuple(idx))
    return tris


def extrude_polygons(x, e, body, z0, z1):
    """Closed triangle meshes of 2-D closed counter-clockwise polygons (x[n,2],
    segments e[m,2], body per segment) extruded along z over [z0, z1]: vertex
    k at z0 is k, at z1 is n + k; two side triangles per segment and both end
    caps (ear-clipped), all wound with outward normals.  Returns
    (x3[2n,3], e3[ne,3], body3[ne])."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    x3 = np.concatenate([np.column_stack([x, np.full(n, z0)]), np.column_stack([x, np.full(n, z1)])])
    tri, tb = [], []
    for (a, b), bd in zip(np.asarray(e), np.asarray(body)):
        tri += [(a, b, n + b), (a, n + b, n + a)]
        tb += [bd, bd]
    for bd in np.unique(body):
        segs = np.asarray(e)[np.asarray(body) == bd]
        nxt = {int(a): int(b) for a, b in segs}
        loop = [int(segs[0, 0])]
        while nxt[loop[-1]] != loop[0]:
            loop.append(nxt[loop[-1]])
        for i, j, k in _ear_clip(x[loop]):
            tri.append((n + loop[i], n + loop[j], n + loop[k]))   # top cap, normal +z
            tri.append((loop[i], loop[k], loop[j]))               # bottom cap, normal -z
            tb += [bd, bd]
    return x3, np.array(tri, dtype=np.int32), np.array(tb, dtype=np.int32)


# ------------------------------------------------------------------ two-phase inputs
RHO_L, RHO_V = 7.55, 0.073   # liquid and vapour densities quoted for the polynomial EOS


def slab_density(n, rho_l=RHO_L, rho_v=RHO_V, width=3.0, frac=0.5):
    """1-D periodic density profile [n]: a liquid slab of length frac*n centred
    in the box, tanh interfaces of the given width on both sides."""
    x = np.arange(n) + 0.5
    a, b = 0.5 * n * (1 - frac), 0.5 * n * (1 + frac)
    return rho_v + (rho_l - rho_v) * 0.5 * (np.tanh((x - a) / width) - np.tanh((x - b) / width))


def droplet_density(shape, radius, center=None, rho_l=RHO_L, rho_v=RHO_V, width=2.0, noise=0.0,
                    seed=0):
    """Density field [nz, ny, nx] of a liquid droplet (circle for nz = 1,
    sphere otherwise) of the given radius in vapour, tanh interface; optional
    multiplicative noise of relative amplitude `noise`."""
    nz, ny, nx = shape
    if center is None:
        center = (0.5 * nx, 0.5 * ny, 0.5 * nz)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    d2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    if nz > 1:
        d2 = d2 + (z - center[2]) ** 2
    rho = rho_v + (rho_l - rho_v) * 0.5 * (1 - np.tanh((np.sqrt(d2) - radius) / width))
    if noise:
        rho = rho * (1 + noise * np.random.default_rng(seed).uniform(-1, 1, size=rho.shape))
    return rho


def q2_box_mesh(n, lengths, origin=None, distort=None):
    """Mesh of a box for Q2 elements (9-node quadrilaterals for len(n) = 2,
    27-node hexahedra for 3): n[d] elements along axis d, nodes on the (2 n +
    1) lattice with x fastest; element-local node i + 3 j (+ 9 k).  Returns
    (X[nn, dim], conn[ne, 3^dim]).  distort(Y) may move the element-corner
    nodes; every other node is then placed by the multilinear map of its
    element's corners (so the elements stay straight-sided)."""
    import itertools
    dim = len(n)
    origin = np.zeros(dim) if origin is None else np.asarray(origin, float)
    m = [2 * k + 1 for k in n]
    axes = [origin[d] + np.linspace(0.0, lengths[d], m[d]) for d in range(dim)]
    idx = np.stack(np.unravel_index(np.arange(int(np.prod(m))), m[::-1])[::-1], 1)  # x fastest
    X = np.stack([axes[d][idx[:, d]] for d in range(dim)], 1)
    stride = np.cumprod([1] + m[:-1])
    local = np.array([l[::-1] for l in itertools.product(range(3), repeat=dim)])
    elems = np.array([e[::-1] for e in itertools.product(*[range(k) for k in n[::-1]])])
    conn = ((2 * elems[:, None, :] + local[None, :, :]) * stride).sum(2).astype(np.int64)
    if distort is not None:
        corner = np.all(idx % 2 == 0, axis=1)
        Xc = X.copy()
        Xc[corner] = distort(X[corner])
        cl = np.array([sum(2 * c[d] * 3 ** d for d in range(dim))
                       for c in (cc[::-1] for cc in itertools.product(range(2), repeat=dim))])
        cbits = np.array([cc[::-1] for cc in itertools.product(range(2), repeat=dim)])
        xi = local - 1.0                                   # node positions in [-1, 1]
        wts = np.prod(np.where(cbits[None, :, :] == 1, 0.5 * (1 + xi[:, None, :]),
                               0.5 * (1 - xi[:, None, :])), axis=2)   # [nen, ncorner]
        for el in conn:
            X[el] = wts @ Xc[el[cl]]
    return X, conn
