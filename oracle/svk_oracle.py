"""Oracle of the paper's structural model (test infrastructure: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs use it).

Total-Lagrangian St Venant-Kirchhoff continuum, section "Structural modeling"
of arXiv 1710.02375, in plain numpy / scipy, FP64:
  - S = lambda tr(E) I + 2 mu E, E = (F^T F - I) / 2, F = I + grad u, P = F S;
    lambda, mu from E_s, nu_s by the printed Lame relations;
  - Q2 Lagrange elements: 9-node quadrilaterals (dim 2, plane strain) or
    27-node hexahedra (dim 3), the geometry mapped from the element's corner
    nodes by the bilinear (trilinear) map, 3-point Gauss rule per axis;
  - the weak form Eq. (weakForm_solid0) with the consistent mass (rho psi, psi);
  - the one-step theta scheme Eq. (timeInt) for both fields, Eqs.
    (timeDiscrete_solid_velocity), (timeDiscrete_solid_displacement);
  - Newton with the analytic Gateaux derivative A'(U)(dU, Psi) printed after
    Eq. (matrixForm2), relaxed by lambda (0.7 in the paper).
Readings: the displacement equation is linear (u1 - u0 = dt (theta v1 + (1 -
theta) v0) at every node), so v1 is eliminated and Newton runs on u1 alone
with the tangent M / (theta dt^2) + theta K(u1); a relaxed step keeps the
linear equation satisfied, so this is Newton on the two-field system.  The
printed signs of the explicit terms (the body force inside the (1 - theta)
bracket) are read as in the theta-rule itself: theta (F^{n+1} - R(u^{n+1})) +
(1 - theta) (F^n - R(u^n)).  Clamped DOFs keep u = v = 0.

Element-local node a = i + 3 j (+ 9 k): i, j, k in {0, 1, 2} along the
reference axes at xi = -1, 0, 1.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_G = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GW = np.array([5.0, 8.0, 5.0]) / 9.0


def _q2_1d(x):
    """Quadratic Lagrange functions on xi = -1, 0, 1 and their derivatives."""
    return (np.array([0.5 * x * (x - 1), 1 - x * x, 0.5 * x * (x + 1)]),
            np.array([x - 0.5, -2 * x, x + 0.5]))


def _q1_1d(x):
    return np.array([0.5 * (1 - x), 0.5 * (1 + x)]), np.array([-0.5, 0.5])


def reference_tables(dim):
    """Per Gauss point g: weight w[g], Q2 values N[g, a] and reference gradients
    dN[g, a, d]; trilinear corner functions L[g, c], dL[g, c, d] (corner c =
    i + 2 j (+ 4 k)) and the element-local index of each corner."""
    pts = [p[::-1] for p in itertools.product(range(3), repeat=dim)]  # x fastest
    ng = 3 ** dim
    w = np.zeros(ng)
    N = np.zeros((ng, 3 ** dim))
    dN = np.zeros((ng, 3 ** dim, dim))
    L = np.zeros((ng, 2 ** dim))
    dL = np.zeros((ng, 2 ** dim, dim))
    for g, gp in enumerate(pts):
        xi = [_G[k] for k in gp]
        w[g] = np.prod([_GW[k] for k in gp])
        q = [_q2_1d(x) for x in xi]
        l1 = [_q1_1d(x) for x in xi]
        for a, node in enumerate(pts):
            N[g, a] = np.prod([q[d][0][node[d]] for d in range(dim)])
            for d in range(dim):
                dN[g, a, d] = np.prod([q[e][1][node[e]] if e == d else q[e][0][node[e]]
                                       for e in range(dim)])
        cor = [c[::-1] for c in itertools.product(range(2), repeat=dim)]
        for c, cc in enumerate(cor):
            L[g, c] = np.prod([l1[d][0][cc[d]] for d in range(dim)])
            for d in range(dim):
                dL[g, c, d] = np.prod([l1[e][1][cc[e]] if e == d else l1[e][0][cc[e]]
                                       for e in range(dim)])
    corner_local = [sum(2 * cc[d] * 3 ** d for d in range(dim))
                    for cc in [c[::-1] for c in itertools.product(range(2), repeat=dim)]]
    return w, N, dN, L, dL, np.array(corner_local)


class SVK:
    """The continuum of nn nodes X[nn, dim] and ne Q2 elements conn[ne, 3^dim];
    E, nu: Young's modulus and Poisson ratio (the Lame relations of the
    paper), rho: density; fixed[nn * dim]: clamped DOFs (node-major)."""

    def __init__(self, X, conn, E, nu, rho, fixed, theta=0.5, lam=0.7, rtol=1e-10,
                 atol=1e-13, max_it=500):
        self.X = np.asarray(X, float)
        self.conn = np.asarray(conn, np.int64)
        self.nn, self.dim = self.X.shape
        self.ne = len(self.conn)
        self.mu = E / (2 * (1 + nu))
        self.lmb = E * nu / ((1 + nu) * (1 - 2 * nu))
        self.rho = rho
        self.fixed = np.asarray(fixed, bool)
        self.free = ~self.fixed
        self.theta, self.lam, self.rtol, self.atol, self.max_it = theta, lam, rtol, atol, max_it
        w, N, dN, L, dL, cl = reference_tables(self.dim)
        self.N = N
        corners = self.X[self.conn[:, cl]]                       # [ne, nc, dim]
        J = np.einsum("ecd,gcf->egdf", corners, dL)              # dX_d / dxi_f
        self.detJ = np.linalg.det(J)
        if np.any(self.detJ <= 0):
            raise ValueError("inverted element")
        Jinv = np.linalg.inv(J)                                  # dxi_f / dX_d
        self.dNX = np.einsum("gaf,egfd->egad", dN, Jinv)         # dN_a / dX_d
        self.wdet = w[None, :] * self.detJ                       # [ne, ng]
        self.M = self._mass()

    # ---------------------------------------------------------------- kinematics
    def _H(self, u):
        ue = u.reshape(self.nn, self.dim)[self.conn]             # [ne, nen, dim]
        return np.einsum("ead,egaf->egdf", ue, self.dNX)         # du_d / dX_f

    def _stress(self, u):
        I = np.eye(self.dim)
        F = I + self._H(u)
        E = 0.5 * (np.einsum("egki,egkj->egij", F, F) - I)
        trE = np.trace(E, axis1=2, axis2=3)
        S = self.lmb * trE[..., None, None] * I + 2 * self.mu * E
        return F, E, S

    def _scatter(self, fe):
        out = np.zeros((self.nn, self.dim))
        np.add.at(out, self.conn, fe)
        return out.ravel()

    def internal_force(self, u):
        """R_a = sum over Gauss points of w det J P grad N_a (the term (P,
        grad psi) of Eq. (weakForm_solid0)), node-major [nn * dim]."""
        F, _, S = self._stress(u)
        P = np.einsum("egik,egkj->egij", F, S)
        fe = np.einsum("eg,egij,egaj->eai", self.wdet, P, self.dNX)
        return self._scatter(fe)

    def energy(self, u):
        """Strain energy: the SVK density lambda/2 (tr E)^2 + mu E:E integrated."""
        _, E, _ = self._stress(u)
        trE = np.trace(E, axis1=2, axis2=3)
        psi = 0.5 * self.lmb * trE ** 2 + self.mu * np.einsum("egij,egij->eg", E, E)
        return float(np.sum(self.wdet * psi))

    def tangent_apply(self, u, du):
        """A'(u)(du, psi_a) for every test function: the printed Gateaux form
        (grad du S + F (mu (grad du^T F + F^T grad du) + lambda tr(F^T grad du) I), grad psi)."""
        F, _, S = self._stress(u)
        dH = self._H(du)
        I = np.eye(self.dim)
        FtdH = np.einsum("egki,egkj->egij", F, dH)
        inner = self.mu * (np.swapaxes(FtdH, 2, 3) + FtdH) + \
            self.lmb * np.trace(FtdH, axis1=2, axis2=3)[..., None, None] * I
        Q = np.einsum("egik,egkj->egij", dH, S) + np.einsum("egik,egkj->egij", F, inner)
        fe = np.einsum("eg,egij,egaj->eai", self.wdet, Q, self.dNX)
        return self._scatter(fe)

    def element_tangent(self, u):
        """Element blocks K[e, a, i, b, d] of A'(u): the printed form expanded
        for du = e_d N_b, psi = e_i N_a (with g_a = F grad N_a):
        delta_id grad N_a . S grad N_b + mu (g_b,i g_a,d + (F F^T)_id grad N_a .
        grad N_b) + lambda g_a,i g_b,d."""
        F, _, S = self._stress(u)
        ne, ng, nen, D = self.dNX.shape
        w = self.wdet[:, :, None]
        dN = self.dNX
        g = dN @ np.swapaxes(F, 2, 3)                          # g[e,g,a,i] = (F grad N_a)_i
        nSn = dN @ S @ np.swapaxes(dN, 2, 3)                   # [e, g, a, b]
        nn_ = dN @ np.swapaxes(dN, 2, 3)
        FFt = F @ np.swapaxes(F, 2, 3)
        # Gauss sums as batched products over g
        gf = g.reshape(ne, ng, nen * D)
        R = np.swapaxes(w * gf, 1, 2) @ gf                     # R[e,(a,i),(b,d)] = sum g_a,i g_b,d
        R = R.reshape(ne, nen, D, nen, D)
        T3 = (np.swapaxes(w * nn_.reshape(ne, ng, -1), 1, 2) @ FFt.reshape(ne, ng, -1))
        T3 = T3.reshape(ne, nen, nen, D, D).transpose(0, 1, 3, 2, 4)   # [e, a, i, b, d]
        geo = np.sum(w[..., None] * nSn, axis=1)              # [e, a, b]
        K = geo[:, :, None, :, None] * np.eye(D)[None, None, :, None, :]
        K = K + self.mu * (R.transpose(0, 1, 4, 3, 2) + T3) + self.lmb * R
        return K

    def _pattern(self):
        """Sparsity of the assembled element blocks (computed once)."""
        nen, dim, n = self.conn.shape[1], self.dim, self.nn * self.dim
        dof = (self.conn[:, :, None] * dim + np.arange(dim)).reshape(self.ne, -1)
        rows = np.repeat(dof, nen * dim, axis=1).ravel()
        cols = np.tile(dof, (1, nen * dim)).ravel()
        lin, inv = np.unique(rows * n + cols, return_inverse=True)
        r, c = lin // n, lin % n
        self._pat = (inv, c, np.searchsorted(r, np.arange(n + 1)), r, c)

    def assemble(self, Ke, dirichlet=False):
        """CSR matrix of element blocks [ne, nen, dim, nen, dim]; with
        dirichlet the clamped rows and columns become identity."""
        if not hasattr(self, "_pat"):
            self._pattern()
        inv, idx, ptr, r, c = self._pat
        n = self.nn * self.dim
        data = np.bincount(inv, weights=Ke.reshape(-1), minlength=len(idx))
        if dirichlet:
            fr, fc = self.fixed[r], self.fixed[c]
            data[fr | fc] = 0.0
            data[fr & (r == c)] = 1.0
        return sp.csr_matrix((data, idx, ptr), shape=(n, n))

    def tangent_matrix(self, u):
        """The sparse matrix of A'(u)."""
        return self.assemble(self.element_tangent(u))

    def _mass(self):
        """Consistent mass (rho psi, psi) on every component, as element blocks
        and assembled."""
        Me = np.einsum("eg,ga,gb->eab", self.rho * self.wdet, self.N, self.N)
        self.Me = np.einsum("eab,id->eaibd", Me, np.eye(self.dim))
        return self.assemble(self.Me)

    def body_load(self, b):
        """Consistent nodal loads of a uniform body force per unit mass b[dim]:
        (rho b, psi_a)."""
        fe = np.einsum("eg,ga,i->eai", self.rho * self.wdet, self.N, np.asarray(b, float))
        return self._scatter(fe)

    # ---------------------------------------------------------------- solvers
    def step(self, u0, v0, F0, F1, dt):
        """One theta step from (u0, v0) with external nodal loads F0 (t^n) and F1
        (t^{n+1}).  Returns (u1, v1, Newton iterations; -1 if not converged)."""
        th, fr = self.theta, self.free
        u0, v0 = np.asarray(u0, float), np.asarray(v0, float)
        cM = 1.0 / (th * dt * dt)
        rhs0 = th * F1 + (1 - th) * (F0 - self.internal_force(u0))
        u = u0 + dt * v0 * fr
        g0 = None
        for it in range(self.max_it + 1):
            G = cM * (self.M @ (u - u0 - dt * v0)) + th * self.internal_force(u) - rhs0
            gn = np.linalg.norm(G[fr])
            g0 = gn if g0 is None else g0
            if gn <= self.rtol * g0 + self.atol:
                break
            if it == self.max_it:
                return u, (u - u0) / (th * dt) - (1 - th) / th * v0, -1
            T = self.assemble(cM * self.Me + th * self.element_tangent(u), dirichlet=True)
            rhs = -G
            rhs[self.fixed] = 0.0
            u = u + self.lam * spla.spsolve(T.tocsc(), rhs)
        v = (u - u0) / (th * dt) - (1 - th) / th * v0
        v[self.fixed] = 0.0
        return u, v, it

    def static(self, F, u=None, tol=1e-9, max_it=100):
        """Equilibrium R(u) = F on the free DOFs (full Newton steps until the
        increment is below tol of the displacement)."""
        u = np.zeros(self.nn * self.dim) if u is None else np.asarray(u, float).copy()
        for it in range(max_it):
            G = self.internal_force(u) - F
            G[self.fixed] = 0.0
            K = self.assemble(self.element_tangent(u), dirichlet=True)
            du = spla.spsolve(K.tocsc(), -G)
            u += du
            if np.linalg.norm(du) <= tol * np.linalg.norm(u):
                return u, it + 1
        return u, -1
