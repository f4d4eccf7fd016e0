"""Seeded synthetic inputs for the collision operator.

This module makes velocity distributions and problem parameters only; it holds
none of the collision operator's arithmetic, and both the CUDA path and the
CPU oracle consume what it makes.  It imports neither of them.

The workloads follow the shapes of the paper's cases (Jaiswal et al., PASC'19):
the spatially homogeneous Krook-Wu mixture of Sec. 3.2 and the 1-D slab of the
Couette case of Sec. 3.3 (Table 2 gives N = 32, N_rho = 8, M = 12).  The
paper's own inputs are analytic, so seeded Maxwellian mixtures and
Hermite-perturbed Maxwellians stand in for them; no external dataset exists.

Conventions
-----------
* Velocity grid: cell centred, c_j = -L + (j + 1/2) h, h = 2L/N, array index
  [ix, iy, iz] with x slowest.
* Maxwellian of a species of mass m with density n, bulk velocity u and
  temperature T (non-dimensional, u0 = sqrt(2 kB T0 / m0), Sec. 2):
  f = n (m / (pi T))^{3/2} exp(-m |c - u|^2 / T).
* Pair parameters of unlike pairs are arithmetic means of the species values
  (this reproduces Table 2's omega_12, alpha_12 and d_12).
"""
import math

import numpy as np

__all__ = [
    "CONFIGS", "velocity_grid", "maxwellian", "two_maxwellians", "perturbed_maxwellian",
    "pair_params", "make_problem", "krook_wu_problem", "relaxation_batch",
]


def velocity_grid(N, L):
    h = 2.0 * L / N
    return -L + (np.arange(N) + 0.5) * h


def maxwellian(N, L, m, n, u, T):
    c = velocity_grid(N, L)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    r2 = (cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2
    return n * (m / (math.pi * T)) ** 1.5 * np.exp(-m * r2 / T)


def two_maxwellians(rng, N, L, m):
    """Sum of two Maxwellians: n ~ U[0.5, 1.5], u ~ N(0, 0.5^2)^3, T ~ U[0.7, 1.3]."""
    f = np.zeros((N, N, N))
    for _ in range(2):
        n = rng.uniform(0.5, 1.5)
        u = rng.normal(0.0, 0.5, size=3)
        T = rng.uniform(0.7, 1.3)
        f += maxwellian(N, L, m, n, u, T)
    return f


def _hermite_e(k, x):
    """Probabilists' Hermite polynomial He_k(x) by its three-term recurrence."""
    if k == 0:
        return np.ones_like(x)
    h0, h1 = np.ones_like(x), x
    for j in range(1, k):
        h0, h1 = h1, x * h1 - j * h0
    return h1


def perturbed_maxwellian(rng, N, L, m, n, u, T, amp=0.1, max_order=3):
    """Maxwellian x (1 + amp * sum_{1<=a+b+c<=3} eps_abc He_a He_b He_c(xi) / sqrt(a!b!c! #modes)),
    xi = sqrt(2m/T) (c - u), eps ~ N(0, 1)."""
    c = velocity_grid(N, L)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    s = math.sqrt(2.0 * m / T)
    xi = (s * (cx - u[0]), s * (cy - u[1]), s * (cz - u[2]))
    modes = [(a, b, cc) for a in range(max_order + 1) for b in range(max_order + 1)
             for cc in range(max_order + 1) if 1 <= a + b + cc <= max_order]
    eps = rng.normal(0.0, 1.0, size=len(modes))
    pert = np.zeros((N, N, N))
    for e, (a, b, cc) in zip(eps, modes):
        norm = math.sqrt(math.factorial(a) * math.factorial(b) * math.factorial(cc) * len(modes))
        pert += e * _hermite_e(a, xi[0]) * _hermite_e(b, xi[1]) * _hermite_e(cc, xi[2]) / norm
    return maxwellian(N, L, m, n, u, T) * (1.0 + amp * pert)


def pair_params(omega, alpha, d, beta_override=None):
    """Per-pair (omega, alpha, d) from per-species values, p-major order.
    Unlike pairs take arithmetic means (Table 2's mixing)."""
    S = len(omega)
    out = []
    for p in range(S):
        for q in range(S):
            pr = {"omega": 0.5 * (omega[p] + omega[q]), "alpha": 0.5 * (alpha[p] + alpha[q]),
                  "d": 0.5 * (d[p] + d[q])}
            if beta_override is not None:
                pr["beta_override"] = float(beta_override[p * S + q])
            out.append(pr)
    return out


# The workloads.  "collide" configs describe the operator's parameters and how
# many spatial points the batch holds; f is made by make_problem().
CONFIGS = {
    # small homogeneous case: one point, all 4 pair operators, FP64
    "c1_homog_n16": dict(N=16, L=8.0, M=6, Nrho=8, masses=[1.0, 2.0], omega=[0.81, 0.81],
                         alpha=[1.0, 1.0], d=[1.0, 1.2], points=1, kind="two_maxwellians", seed=1),
    # 1-D DG slab: 8 elements x 3 Gauss points, VSS, N=32, M=12, N_rho=8
    "c2_slab_n32": dict(N=32, L=10.0, M=12, Nrho=8, masses=[1.0, 4.0], omega=[0.75, 0.75],
                        alpha=[1.4, 1.4], d=[1.0, 1.2], points=24, elements=8, order=3,
                        kind="slab", T_left=1.0, T_right=1.5, seed=2),
    # precision sweep: N=48, M=12, N_rho=16, 32 elements x 4 points
    "c3_sweep_n48": dict(N=48, L=12.0, M=12, Nrho=16, masses=[1.0, 2.0], omega=[0.81, 0.81],
                         alpha=[1.0, 1.0], d=[1.0, 1.2], points=128, elements=32, order=4,
                         kind="slab", T_left=1.0, T_right=1.5, seed=3),
    # adjoint workload: 64 points, float32 data
    "c4_adjoint_n32": dict(N=32, L=10.0, M=12, Nrho=8, masses=[1.0, 2.0], omega=[0.81, 0.81],
                           alpha=[1.0, 1.0], d=[1.0, 1.2], points=64, elements=16, order=4,
                           kind="slab", T_left=1.0, T_right=1.5, seed=4),
    # heat-transfer slab for the DG step: 16 elements x 3 Gauss points, purely
    # diffuse walls at T = 1 (x = 0) and T = 2 (x = 1), at rest
    "c5_heat_slab_n32": dict(N=32, L=8.0, M=12, Nrho=8, masses=[1.0, 2.0], omega=[0.81, 0.81],
                             alpha=[1.0, 1.0], d=[1.0, 1.2], points=48, elements=16, order=3,
                             kind="slab", T_left=1.0, T_right=2.0, seed=5,
                             walls=((1.0, (0.0, 0.0, 0.0)), (2.0, (0.0, 0.0, 0.0)))),
}


def _gauss_points_on_elements(elements, order):
    """x positions of `order` Gauss-Legendre points in each of `elements`
    equal elements of [0, 1] (the DG solution points of the slab)."""
    xg, _ = np.polynomial.legendre.leggauss(order)
    h = 1.0 / elements
    xs = [(e + 0.5) * h + 0.5 * h * x for e in range(elements) for x in xg]
    return np.array(xs)


def make_problem(name, points=None, dtype=np.float64):
    """Return a dict with the operator parameters and f of shape [P][S][N][N][N]."""
    cfg = dict(CONFIGS[name])
    N, L = cfg["N"], cfg["L"]
    S = len(cfg["masses"])
    P = cfg["points"] if points is None else int(points)
    rng = np.random.default_rng(cfg["seed"])
    f = np.empty((P, S, N, N, N))
    if cfg["kind"] == "two_maxwellians":
        for i in range(P):
            for p in range(S):
                f[i, p] = two_maxwellians(rng, N, L, cfg["masses"][p])
    elif cfg["kind"] == "slab":
        xs = _gauss_points_on_elements(cfg["elements"], cfg["order"])
        for i in range(P):
            x = xs[i % len(xs)]
            T = cfg["T_left"] + (cfg["T_right"] - cfg["T_left"]) * x
            for p in range(S):
                f[i, p] = perturbed_maxwellian(rng, N, L, cfg["masses"][p], 1.0, (0.0, 0.0, 0.0), T)
    else:
        raise ValueError(cfg["kind"])
    pairs = pair_params(cfg["omega"], cfg["alpha"], cfg["d"])
    out = dict(name=name, N=N, L=L, M=cfg["M"], Nrho=cfg["Nrho"], masses=list(cfg["masses"]),
               pairs=pairs, f=f.astype(dtype))
    for k in ("elements", "order", "walls"):
        if k in cfg:
            out[k] = cfg[k]
    return out


def krook_wu_problem(N, M, Nrho, m1=1.0, m2=1.0, L=12.0):
    """Parameters of the Krook-Wu test of Sec. 3.2: constant kernel
    B_pq = lambda_qp / (4 pi n_q) with n1 = n2 = 1, lambda_11 = lambda_22 = 1,
    lambda_12 = lambda_21 = 1/2 (omega = 1, alpha = 1)."""
    lam = [[1.0, 0.5], [0.5, 1.0]]
    nn = [1.0, 1.0]
    bo = [lam[q][p] / (4.0 * math.pi * nn[q]) for p in range(2) for q in range(2)]
    pairs = pair_params([1.0, 1.0], [1.0, 1.0], [1.0, 1.0], beta_override=bo)
    return dict(N=N, L=L, M=M, Nrho=Nrho, masses=[m1, m2], pairs=pairs)


def relaxation_batch(count=256, seed=5):
    """`count` spatially homogeneous relaxation problems with uneven
    parameters: N from {24, 32, 48} on [-L, L]^3 with L = N / 3.2 (the grid
    spacing of the 1-D slab workload), 2 or 3 species with distinct masses
    from {1, 2, 4}, M from {6, 12}, N_rho from {8, 16}, VHS (alpha = 1) or VSS
    (alpha = 1.4) with omega = 0.81, and two-Maxwellian data per species.
    Returns a list of dicts with the operator parameters and f of shape
    [1][S][N][N][N]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice([24, 32, 48]))
        L = N / 3.2
        S = int(rng.choice([2, 3]))
        masses = sorted(float(m) for m in rng.choice([1.0, 2.0, 4.0], size=S, replace=False))
        M = int(rng.choice([6, 12]))
        Nrho = int(rng.choice([8, 16]))
        alpha = 1.0 if rng.uniform() < 0.5 else 1.4
        pairs = pair_params([0.81] * S, [alpha] * S, [1.0 + 0.1 * j for j in range(S)])
        f = np.stack([two_maxwellians(rng, N, L, m) for m in masses])[None]
        out.append(dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs, alpha=alpha, f=f))
    return out
