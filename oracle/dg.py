"""FP64 CPU oracle of the 1-D nodal DG streaming term (TEST INFRASTRUCTURE).

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import it; the CUDA library never does.

The paper solves Eq. (1), df_p/dt + c . grad_x f_p = sum_q Q^(pq), by
Runge-Kutta discontinuous Galerkin in one space dimension (Sec. 3.3 and the
Couette case of Table 2: DG order 3, purely diffuse walls) and defers the
formulas to its references.  This module writes out the textbook scheme it
names, in plain numpy with loops over elements:

* space: [x0, x1] split into Ne equal elements; on each, the solution is the
  Lagrange interpolant on the K Gauss-Legendre nodes xi_j of [-1, 1]
  ("DG order K"), and the same nodes are the quadrature, so the element mass
  matrix is J diag(w) with J = h_e / 2;
* weak form of df/dt = -c_x df/dx against each basis function phi_i:
      J w_i df_i/dt = c_x sum_j w_j phi_i'(xi_j) f_j
                      - phi_i(+1) F_right + phi_i(-1) F_left,
  where F is the upwind numerical flux c_x f taken from the side the
  velocity comes from;
* purely diffuse walls: for velocities entering the domain, the wall state is
  n_w M_w(c), the wall Maxwellian (m/(pi T_w))^{3/2} exp(-m |c - u_w|^2/T_w)
  (the Maxwellian convention used throughout this repository), with n_w
  chosen so that the discrete net mass flux sum_c c_x f(c) through the wall
  is zero;
* time: the three-stage strong-stability-preserving Runge-Kutta scheme in
  Shu-Osher form, with L(f) = streaming(f) + sum_q Q^(pq)(f).

Layout: f[P][S][N^3] with P = Ne K points, point index e K + j (element
major), and velocity index (ix N + iy) N + iz on the cell-centred grid
c = -L + (i + 1/2) h.
"""
import numpy as np

from . import gauss_legendre


def lagrange_values(nodes, x):
    """phi_i(x) for the Lagrange basis on `nodes`: array [len(nodes)]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    K = len(nodes)
    v = np.ones(K)
    for i in range(K):
        for m in range(K):
            if m != i:
                v[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return v


def lagrange_derivative(nodes):
    """D[i][j] = phi_i'(xi_j), from the product rule applied to
    phi_i(x) = prod_{m != i} (x - xi_m) / (xi_i - xi_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    K = len(nodes)
    D = np.zeros((K, K))
    for i in range(K):
        den = 1.0
        for m in range(K):
            if m != i:
                den *= nodes[i] - nodes[m]
        for j in range(K):
            x = nodes[j]
            s = 0.0
            for l in range(K):
                if l == i:
                    continue
                p = 1.0
                for m in range(K):
                    if m != i and m != l:
                        p *= x - nodes[m]
                s += p
            D[i, j] = s / den
    return D


def maxwellian(N, L, m, n, u, T):
    h = 2.0 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    e = ((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) * m / T
    return (n * (m / (np.pi * T)) ** 1.5 * np.exp(-e)).reshape(-1)


class Slab:
    """Ne elements of K Gauss nodes on [x0, x1]; S species on an N^3 grid of
    [-L, L]^3; walls = ((T_left, u_left[3]), (T_right, u_right[3]))."""

    def __init__(self, Ne, K, x0, x1, N, L, masses, walls):
        self.Ne, self.K, self.N, self.L = int(Ne), int(K), int(N), float(L)
        self.S = len(masses)
        self.masses = [float(m) for m in masses]
        self.xi, self.w = gauss_legendre(self.K)
        self.D = lagrange_derivative(self.xi)
        self.phiL = lagrange_values(self.xi, -1.0)
        self.phiR = lagrange_values(self.xi, 1.0)
        self.he = (x1 - x0) / self.Ne
        self.J = self.he / 2.0
        self.x = np.array([x0 + (e + 0.5) * self.he + self.J * xj for e in range(self.Ne) for xj in self.xi])
        h = 2.0 * self.L / self.N
        c = -self.L + (np.arange(self.N) + 0.5) * h
        self.cx = np.repeat(c, self.N * self.N)  # x component of every velocity, index (ix N + iy) N + iz
        self.walls = walls
        # wall Maxwellians (unit density) per wall and species
        self.Mw = [[maxwellian(self.N, self.L, m, 1.0, walls[s][1], walls[s][0]) for m in self.masses]
                   for s in range(2)]

    @property
    def P(self):
        return self.Ne * self.K

    def wall_state(self, side, p, trace):
        """n_w M_w for one species at the left (side 0) or right (1) wall, with
        n_w from zero net mass flux given the interior trace there."""
        M = self.Mw[side][p]
        cx = self.cx
        if side == 0:  # domain on the right: entering velocities have c_x > 0
            out = np.sum(cx[cx < 0] * trace[cx < 0])
            inn = np.sum(cx[cx > 0] * M[cx > 0])
        else:
            out = np.sum(cx[cx > 0] * trace[cx > 0])
            inn = np.sum(cx[cx < 0] * M[cx < 0])
        return (-out / inn) * M

    def traces(self, f):
        """(left, right): element 0 at xi = -1 and element Ne-1 at xi = +1, [S][N^3]."""
        f = np.asarray(f, dtype=np.float64)
        K = self.K
        left = np.stack([self.phiL @ f[0:K, p, :] for p in range(self.S)])
        right = np.stack([self.phiR @ f[(self.Ne - 1) * K:self.Ne * K, p, :] for p in range(self.S)])
        return left, right

    def streaming(self, f, halo_left=None, halo_right=None):
        """-c_x df/dx in the DG weak form: f[P][S][N^3] -> [P][S][N^3].  A halo
        (the neighbouring slab's trace at the shared face, [S][N^3]) replaces
        the wall at that side."""
        Ne, K = self.Ne, self.K
        f = np.asarray(f, dtype=np.float64)
        out = np.zeros_like(f)
        cx = self.cx
        pos = cx > 0
        for p in range(self.S):
            for e in range(Ne):
                u = f[e * K:(e + 1) * K, p, :]  # [K][n]
                uL_in = self.phiL @ u  # this element's trace at its left face
                uR_in = self.phiR @ u
                if e > 0:
                    uL_out = self.phiR @ f[(e - 1) * K:e * K, p, :]
                elif halo_left is not None:
                    uL_out = halo_left[p]
                else:
                    uL_out = self.wall_state(0, p, uL_in)
                if e < Ne - 1:
                    uR_out = self.phiL @ f[(e + 1) * K:(e + 2) * K, p, :]
                elif halo_right is not None:
                    uR_out = halo_right[p]
                else:
                    uR_out = self.wall_state(1, p, uR_in)
                FL = cx * np.where(pos, uL_out, uL_in)  # left face: upwind is the left side when c_x > 0
                FR = cx * np.where(pos, uR_in, uR_out)
                for i in range(K):
                    vol = cx * sum(self.w[j] * self.D[i, j] * u[j] for j in range(K))
                    out[e * K + i, p, :] = (vol - self.phiR[i] * FR + self.phiL[i] * FL) / (self.J * self.w[i])
        return out

    def rhs(self, f, Q=None):
        """streaming(f) + sum_q Q[P][S][S][N^3] (Q may be None)."""
        r = self.streaming(f)
        if Q is not None:
            r = r + np.asarray(Q, dtype=np.float64).sum(axis=2)
        return r

    def mass_rate(self, g):
        """d/dt of the total mass of each species for a rate g[P][S][N^3]:
        sum over elements and nodes of J w_j, times h^3 sum over velocities."""
        h3 = (2.0 * self.L / self.N) ** 3
        wq = np.tile(self.w, self.Ne) * self.J
        return h3 * np.einsum("j,jpv->p", wq, np.asarray(g))

    def ssp_rk3(self, f, dt, collide=None):
        """One SSP-RK3 step (Shu-Osher form); collide(f) -> Q[P][S][S][N^3] or None."""
        L = lambda g: self.rhs(g, collide(g) if collide is not None else None)
        f0 = np.asarray(f, dtype=np.float64)
        f1 = f0 + dt * L(f0)
        f2 = 0.75 * f0 + 0.25 * (f1 + dt * L(f1))
        return f0 / 3.0 + (2.0 / 3.0) * (f2 + dt * L(f2))
