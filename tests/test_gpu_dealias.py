"""Dealiased operator (linear convolution of Eq. (7) by the 3/2 rule) on the
GPU against the dealiased oracle, in FP64 and on the tensor cores."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import dealias as DA
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(N, L, M, Nrho, alpha, P, seed):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.0]
    pairs = W.pair_params([0.81, 0.75], [alpha, alpha], [1.0, 1.2])
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    return masses, pairs, f


def _oracle(N, L, M, Nrho, masses, pairs, f):
    S = len(masses)
    out = np.zeros((f.shape[0], S, S, N, N, N))
    for p in range(S):
        for q in range(S):
            pp = pairs[p * S + q]
            dp = DA.DealiasedPair(N, L, M, Nrho, masses[p], masses[q], pp["omega"], pp["alpha"], pp["d"])
            for i in range(f.shape[0]):
                out[i, p, q] = dp.collide(f[i, p], f[i, q])
    return out


@pytest.mark.parametrize("N,M,Nrho,alpha,prec,tol", [
    (8, 6, 4, 1.4, "fp64", 1e-12),
    (16, 6, 4, 1.0, "fp64", 1e-12),
    (16, 12, 3, 1.4, "fp32_tc", 1e-5),
    (32, 6, 3, 1.0, "fp32_tc", 1e-5),
])
def test_dealiased_matches_oracle(N, M, Nrho, alpha, prec, tol):
    L = N / 3.2
    masses, pairs, f = _case(N, L, M, Nrho, alpha, 2 if N <= 16 else 1, seed=N + M)
    Np = 3 * N // 2
    plan = B.Plan(Np, L, M, Nrho, masses, pairs, prec, f.shape[0])
    fd = torch.from_numpy(f).to("cuda", plan.dtype)
    Q = plan.collide_dealiased(fd, N).double().cpu().numpy()
    plan.check()
    Qo = _oracle(N, L, M, Nrho, masses, pairs, f.astype(np.float32).astype(np.float64) if prec != "fp64" else f)
    assert np.abs(Q - Qo).max() <= tol * np.abs(Qo).max()


def test_dealiased_argument_errors():
    masses, pairs, f = _case(8, 2.5, 6, 3, 1.0, 1, 1)
    plan = B.Plan(12, 2.5, 6, 3, masses, pairs, "fp64", 1)
    fd = torch.from_numpy(f).cuda()
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_dealias_work_bytes(plan._h, 1, 10)  # 3 * 10 / 2 != 12
    assert e.value.status == 1
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    Q = torch.empty((1, 2, 2, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_collide_dealiased(plan._h, 1, 8, fd, Q, small)
    assert e.value.status == 1
