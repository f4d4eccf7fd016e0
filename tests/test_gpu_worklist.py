"""The work-list schedule (dgfs_plan_set_schedule(plan, 1),
dgfs_batch_set_schedule(batch, 1)): one launch whose CTAs claim stage tasks
from a device queue with dependency counters runs the same stage bodies on the
same data as the per-stage launches, so the results must be the same bits.  Covers N = 24
(ragged plane tiles), 32 and 48, FP32 and BF16 splits, the sigma collapse,
several chunks of points per pair (each job reuses the plan's workspace after
the previous one), same-species translate sharing, graph capture, and uneven
batches against their round launches and the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instance(N, S, M, Nrho, P, prec, seed, vhs=False, max_points=None):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.0, 4.0][:S]
    alpha = [1.0, 1.0, 1.0] if vhs else [1.0, 1.4, 1.2]
    pairs = W.pair_params([0.81, 0.75, 0.7][:S], alpha[:S], [1.0, 1.2, 0.9][:S])
    L = N / 3.2
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    plan = B.Plan(N, L, M, Nrho, masses, pairs, prec, max_points or P)
    dt = torch.float64 if prec == "fp64" else torch.float32
    fd = torch.from_numpy(f).to("cuda", dt)
    return dict(plan=plan, f=fd, fnp=f, P=P, pb=dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs))


CASES = [
    # N, S, M, Nrho, P, precision, seed, vhs
    (24, 3, 6, 4, 2, "fp32_tc", 31, False),   # 9 pairs, 3 of them same-species; 5-plane tiles
    (32, 2, 12, 8, 30, "fp32_tc", 32, False),  # 30 points: two chunks (24 + 6) per pair
    (48, 2, 6, 4, 3, "fp32_tc", 33, False),
    (32, 2, 6, 4, 2, "bf16x3", 34, False),
    (32, 2, 12, 4, 2, "fp32_tc", 35, True),    # sigma collapse (VHS)
    (24, 2, 12, 8, 3, "tf32", 36, False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%d_S%d_M%d_Nr%d_P%d_%s%s" % (c[:6] + ("_vhs" if c[7] else "",)))
def test_plain_call_worklist_equals_stage_launches(case):
    N, S, M, Nrho, P, prec, seed, vhs = case
    inst = _instance(N, S, M, Nrho, P, prec, seed, vhs)
    plan = inst["plan"]
    if vhs:
        plan.set_collapse(1)
    assert plan.schedule() == 0
    ref = plan.collide(inst["f"]).clone()
    plan.check()
    plan.set_schedule(1)
    assert plan.schedule() == 1
    l0 = plan.launch_count()
    for _ in range(2):  # the second call reuses the zeroed counters
        Q = torch.full_like(ref, float("nan"))
        plan.collide(inst["f"], Q)
        torch.cuda.synchronize()
        plan.check()
        assert torch.equal(Q, ref)
    # forward transform, one work-list launch, the finishing passes
    assert plan.launch_count() - l0 < 2 * 12


def test_worklist_matches_oracle_n24():
    inst = _instance(24, 2, 6, 4, 1, "fp32_tc", 41)
    plan = inst["plan"]
    plan.set_schedule(1)
    Q = plan.collide(inst["f"]).double().cpu().numpy()
    plan.check()
    pb = inst["pb"]
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(inst["fnp"])
    for p in range(2):
        for q in range(2):
            a, b = Q[0, p, q], Qo[0, p, q]
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err < 1e-5, (p, q, err)


def test_worklist_in_cuda_graph():
    inst = _instance(32, 2, 6, 4, 3, "fp32_tc", 42)
    plan = inst["plan"]
    ref = plan.collide(inst["f"]).clone()
    plan.set_schedule(1)
    Q = torch.full_like(ref, float("nan"))
    g = B.dgfs_graph_capture([plan._h], [inst["P"]], [inst["f"]], [Q])
    try:
        for _ in range(3):
            B.dgfs_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        B.dgfs_graph_destroy(g)
    plan.check()
    assert torch.equal(Q, ref)


def test_schedule_argument_errors():
    inst = _instance(16, 1, 6, 4, 1, "fp32_tc", 43)
    with pytest.raises(B.DgfsError) as e:
        inst["plan"].set_schedule(1)  # N = 16 runs stage kernels with different pipeline counts
    assert e.value.status == 5
    with pytest.raises(B.DgfsError) as e:
        inst["plan"].set_schedule(2)
    assert e.value.status == 1
    p64 = _instance(24, 1, 6, 4, 1, "fp64", 44)["plan"]
    with pytest.raises(B.DgfsError) as e:
        p64.set_schedule(1)
    assert e.value.status == 5


def test_uneven_batch_worklist_equals_round_launches_and_oracle():
    insts = [
        _instance(24, 3, 6, 4, 2, "fp32_tc", 51),
        _instance(24, 2, 12, 8, 1, "fp32_tc", 52),
        _instance(32, 2, 12, 8, 3, "fp32_tc", 53),
        _instance(32, 3, 6, 4, 2, "fp32_tc", 54),
        _instance(48, 2, 6, 4, 2, "fp32_tc", 55),
        _instance(32, 2, 6, 4, 2, "bf16x3", 56),
    ]
    Q1 = [torch.full((i["P"], i["plan"].S, i["plan"].S) + (i["plan"].N,) * 3, float("nan"),
                     device="cuda", dtype=torch.float32) for i in insts]
    Q0 = [torch.full_like(q, float("nan")) for q in Q1]
    b1 = B.Batch([i["plan"] for i in insts], [i["f"] for i in insts], Q1)
    try:
        b1.set_schedule(1)
        for _ in range(2):
            b1.launch()
        torch.cuda.synchronize()
    finally:
        b1.close()
    b0 = B.Batch([i["plan"] for i in insts], [i["f"] for i in insts], Q0)
    try:
        b0.launch()  # default: per-stage launches per round
        torch.cuda.synchronize()
    finally:
        b0.close()
    for inst, a, b in zip(insts, Q1, Q0):
        inst["plan"].check()
        assert torch.equal(a, b)
    # one sampled point of the N = 24, S = 3 instance against the oracle
    pb = insts[0]["pb"]
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(insts[0]["fnp"][1:2])
    Qg = Q1[0][1:2].double().cpu().numpy()
    for p in range(3):
        for q in range(3):
            err = np.abs(Qg[0, p, q] - Qo[0, p, q]).max() / np.abs(Qo[0, p, q]).max()
            assert err < 1e-5, (p, q, err)
