"""Precision sweep at full size: N = 48 on [-12, 12]^3, M = 12, N_rho = 16,
128 points (32 elements x 4 Gauss points), masses (1, 2), VHS omega = 0.81.
Every form evaluates all 128 points in one call (the launch configuration of
a full batch); the FP64 oracle checks sampled points, and the conservation
defects of each form (mass of Q^pq, momentum and energy of Q^pq + Q^qp) are
compared with the oracle's."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SAMPLE = [0, 127]
BOUND = {"fp64": 1e-12, "fp32_tc": 1e-5, "bf16x3": 1e-3, "tf32": None}


@pytest.fixture(scope="module")
def sweep():
    pb = W.make_problem("c3_sweep_n48")
    O.set_threads(max(1, len(__import__("os").sched_getaffinity(0))))
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(pb["f"], points=SAMPLE)
    return pb, Qo


def _defects(pb, Q):
    """[P][S][S][5] moments -> (mass of Q^pq, momentum and energy of Q^pq + Q^qp)."""
    m = Q[..., 0]
    mom = Q[..., 1:4] + np.swapaxes(Q[..., 1:4], 1, 2)
    en = Q[..., 4] + np.swapaxes(Q[..., 4], 1, 2)
    return m, mom, en


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc", "bf16x3", "tf32"])
def test_c3_sweep_n48_form(sweep, prec):
    pb, Qo = sweep
    P = pb["f"].shape[0]
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P)
    f = torch.from_numpy(pb["f"]).to("cuda", plan.dtype)
    Q = plan.collide(f)
    plan.check()
    mom_gpu = plan.moments(Q).cpu().numpy()[SAMPLE]
    Qs = Q[SAMPLE].double().cpu().numpy()
    err = np.abs(Qs - Qo).max() / np.abs(Qo).max()
    print("\n%s: relative max-norm error vs oracle %.3e" % (prec, err))
    if BOUND[prec] is not None:
        assert err <= BOUND[prec]
    else:
        assert err < 5e-2  # single TF32 product: reported, sanity only
    # conservation defects agree with the oracle's: a moment is a weighted sum
    # over the grid, so its error is at most max|Q_gpu - Q_orc| times the
    # L1 norm of its weights (h^3 {1, m abs(c_x), m abs(c)^2} summed over the grid)
    S = len(pb["masses"])
    mom_orc = np.zeros_like(mom_gpu)
    for i in range(len(SAMPLE)):
        for p in range(S):
            for q in range(S):
                mom_orc[i, p, q] = O.moments(pb["N"], pb["L"], pb["masses"][p], Qo[i, p, q])
    N, L = pb["N"], pb["L"]
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    mmax = max(pb["masses"])
    w1 = [h ** 3 * N ** 3, h ** 3 * mmax * np.abs(c).sum() * N * N, h ** 3 * mmax * 3 * (c ** 2).sum() * N * N]
    qerr = np.abs(Qs - Qo).max()
    scale = np.abs(mom_orc).max()
    for a, b, w in zip(_defects(pb, mom_gpu), _defects(pb, mom_orc), w1):
        assert np.abs(a - b).max() <= 2.02 * qerr * w + 1e-13 * scale, (prec, np.abs(a - b).max(), qerr * w)
