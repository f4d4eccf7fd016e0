"""Pin of the operator's odd-moment response: the heat flux of Maxwell molecules
relaxes at two thirds of the stress rate (Prandtl number 2/3), for any angular
kernel.

With B = beta (1 + t)^{alpha-1} (Eq. 3 at omega = 1), equal masses and zero mean
velocity, the sigma-average of phi(v') - phi(v) for phi = v_x |v|^2 keeps, after
the v <-> v_* symmetrisation, only the terms even in u = v - v_*:
(a1 / 2) |u|^2 G_x + ((a1 + a2 - b0) / 2) u_x (u . G), where G = (v + v_*)/2 and
a1, a1 + a2, b0 are the sigma-averages of (1 - t^2)/2, t^2 and 1 with weight
b(t) times 2 pi.  Both integrate against f f_* to n int f v_x |v|^2, so

    d/dt int f v_x |v|^2 = -(n / 2) 2 pi int b (1 - t^2) dt  int f v_x |v|^2,

two thirds of the traceless-stress rate (n / 2) 2 pi (3/2) int b (1 - t^2) dt.
The linearised response to M (1 + eps v_x (|v|^2 - 5/2)) (zero mean velocity)
is taken as the odd part in eps of two evaluations; with
M = pi^{-3/2} exp(-|v|^2) it is nu_q = 2 pi beta 2^{alpha+1} / ((alpha+1)(alpha+2)).

Unlike the stress, this odd moment needs a fine grid: the oracle meets it to
2e-5 at h = 1/3 (N = 48, L = 8; also 2.6e-5 at N = 48, L = 9), but is 2 % off
at h = 1/2 and 16 % at h = 0.58.  Bound 2e-4."""
import numpy as np

import oracle as O

N, L, M, NRHO, EPS = 48, 8.0, 6, 12, 0.05


def test_heat_flux_relaxes_at_two_thirds_of_the_stress_rate():
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    c2 = cx ** 2 + cy ** 2 + cz ** 2
    Mx = np.exp(-c2) / np.pi ** 1.5
    alpha = 1.0
    pair = O.Problem(N, L, M, NRHO, [1.0], [dict(omega=1.0, alpha=alpha, d=1.0)]).pair(0, 0)
    phi = cx * c2
    psi = cx * (c2 - 2.5)
    num = den = 0.0
    for s in (1.0, -1.0):
        f = Mx * (1.0 + s * EPS * psi)
        Q, _ = pair.collide(f, f)
        num += s * float((phi * Q).sum())
        den += s * float((phi * f).sum())
    nu_q = -num / den
    want = 2.0 * np.pi * pair.beta * 2.0 ** (alpha + 1) / ((alpha + 1) * (alpha + 2))
    assert abs(nu_q / want - 1.0) <= 2e-4, (nu_q, want)
