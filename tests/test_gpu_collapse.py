"""Declared fast variant: the sum over design directions before the forward
transforms (exact when b_rs does not depend on s, i.e. alpha = 1).  It must
give the literal Algorithm 2 result (the oracle) to the form's tolerance, and
differ from the literal GPU order only by rounding."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _vhs(N, M, Nrho, S, P, seed):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.0, 4.0][:S]
    pairs = W.pair_params([0.81, 0.7, 0.6][:S], [1.0] * S, [1.0, 1.2, 0.9][:S])
    L = N / 3.2
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    return dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs), f


@pytest.mark.parametrize("N,M,Nrho,S,P", [(8, 6, 4, 2, 3), (16, 12, 5, 2, 2), (12, 6, 3, 3, 1), (32, 12, 8, 2, 2)])
def test_fp64_collapse_matches_oracle_and_literal_order(N, M, Nrho, S, P):
    pb, f = _vhs(N, M, Nrho, S, P, seed=N + M)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", P)
    assert plan.info()["collapse"] == 1  # on by default for VHS plans
    fd = torch.from_numpy(f).cuda()
    Qc = plan.collide(fd).cpu().numpy()
    plan.set_collapse(False)
    assert plan.info()["collapse"] == 0
    Ql = plan.collide(fd).cpu().numpy()
    Qo = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"]).collide_all(f)
    scale = np.abs(Qo).max()
    assert np.abs(Qc - Qo).max() <= 1e-12 * scale
    assert np.abs(Ql - Qo).max() <= 1e-12 * scale
    assert np.abs(Qc - Ql).max() <= 1e-13 * scale


def test_collapse_refused_for_vss_plans():
    pb = W.make_problem("c2_slab_n32", points=1)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    assert plan.info()["collapse"] == 0
    with pytest.raises(B.DgfsError) as e:
        plan.set_collapse(True)
    assert e.value.status == 5


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x3"])
@pytest.mark.parametrize("N,M,Nrho,S,P", [(8, 6, 5, 2, 3), (16, 12, 4, 2, 2), (24, 6, 3, 3, 1), (32, 12, 8, 2, 2)])
def test_tensor_core_collapse_matches_oracle(prec, N, M, Nrho, S, P):
    pb, f = _vhs(N, M, Nrho, S, P, seed=3 * N + M)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P)
    assert plan.info()["collapse"] == 1
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    Qc = plan.collide(fd).double().cpu().numpy()
    plan.check()
    plan.set_collapse(False)
    Ql = plan.collide(fd).double().cpu().numpy()
    Qo = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"]).collide_all(f)
    scale = np.abs(Qo).max()
    tol = 1e-5 if prec == "fp32_tc" else 1e-3
    assert np.abs(Qc - Qo).max() <= tol * scale
    assert np.abs(Ql - Qo).max() <= tol * scale
