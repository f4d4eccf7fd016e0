"""Batching and scheduling: one CUDA graph over uneven instances (different N,
S, M, N_rho, precision and point counts) equals separate calls bit for bit, and
so does the batched work list (one launch per stage over the jobs of every
instance with the same N and operand format); the homogeneous relaxation step;
the autotuner keeps results within bounds."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instance(N, S, M, Nrho, P, prec, seed, vhs=False):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.0, 4.0][:S]
    alpha = [1.0, 1.0, 1.0] if vhs else [1.0, 1.4, 1.2]
    pairs = W.pair_params([0.81, 0.75, 0.7][:S], alpha[:S], [1.0, 1.2, 0.9][:S])
    L = N / 3.2
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    plan = B.Plan(N, L, M, Nrho, masses, pairs, prec, P)
    dt = torch.float64 if prec == "fp64" else torch.float32
    fd = torch.from_numpy(f).to("cuda", dt)
    return dict(plan=plan, f=fd, fnp=f, P=P, pb=dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs))


@pytest.fixture(scope="module")
def batch():
    return [
        _instance(8, 3, 12, 4, 3, "fp32_tc", 1),
        _instance(16, 2, 6, 8, 2, "fp32_tc", 2),
        _instance(24, 2, 6, 3, 1, "fp32_tc", 3),
        _instance(16, 1, 12, 4, 2, "fp64", 4),
    ]


def test_graph_of_uneven_batch_equals_separate_calls(batch):
    refs = []
    for inst in batch:
        refs.append(inst["plan"].collide(inst["f"]).clone())
    torch.cuda.synchronize()
    Qs = [torch.full_like(r, float("nan")) for r in refs]
    g = B.dgfs_graph_capture([i["plan"]._h for i in batch], [i["P"] for i in batch], [i["f"] for i in batch], Qs)
    try:
        assert B.dgfs_graph_kernel_count(g) > len(batch)
        for _ in range(2):
            B.dgfs_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        B.dgfs_graph_destroy(g)
    for inst, Q, ref in zip(batch, Qs, refs):
        inst["plan"].check()
        assert torch.equal(Q, ref)


@pytest.fixture(scope="module")
def worklist():
    # three N = 16 FP32 tensor-core plans with different job counts (S^2
    # pairs), one of them VHS on the sigma-collapsed path; an N = 8 plan whose
    # 30 points take two chunks (24 + 6); N = 24 (ragged 5-plane tiles) and
    # N = 32 groups; a BF16 group and an FP64 plan
    return [
        _instance(16, 2, 6, 8, 3, "fp32_tc", 11),
        _instance(16, 3, 12, 4, 2, "fp32_tc", 12),
        _instance(16, 2, 12, 3, 2, "fp32_tc", 13, vhs=True),
        _instance(8, 2, 6, 4, 30, "fp32_tc", 14),
        _instance(24, 3, 6, 4, 2, "fp32_tc", 17),
        _instance(32, 2, 12, 8, 3, "fp32_tc", 18),
        _instance(16, 1, 6, 4, 2, "bf16x3", 15),
        _instance(8, 1, 12, 4, 2, "fp64", 16),
    ]


def test_batched_worklist_equals_separate_calls(worklist):
    assert worklist[2]["plan"].info()["collapse"] == 1
    refs = [inst["plan"].collide(inst["f"]).clone() for inst in worklist]
    torch.cuda.synchronize()
    Qs = [torch.full_like(r, float("nan")) for r in refs]
    b = B.dgfs_batch_create([i["plan"]._h for i in worklist], [i["P"] for i in worklist],
                            [i["f"] for i in worklist], Qs)
    try:
        for _ in range(2):
            B.dgfs_batch_launch(b)
        torch.cuda.synchronize()
    finally:
        B.dgfs_batch_destroy(b)
    for inst, Q, ref in zip(worklist, Qs, refs):
        inst["plan"].check()
        assert torch.equal(Q, ref)


def test_batched_worklist_with_relaxation_matches_graph(worklist):
    sub = [worklist[0], worklist[3], worklist[4]]
    dt = 0.01
    f_b = [i["f"].clone() for i in sub]
    f_g = [i["f"].clone() for i in sub]
    Q_b = [torch.empty(i["P"], i["f"].shape[1], *i["f"].shape[1:], dtype=i["f"].dtype, device="cuda")
           for i in sub]
    Q_g = [torch.empty_like(q) for q in Q_b]
    b = B.dgfs_batch_create([i["plan"]._h for i in sub], [i["P"] for i in sub], f_b, Q_b, dt=dt)
    try:
        B.dgfs_batch_launch(b)
        B.dgfs_batch_launch(b)
        torch.cuda.synchronize()
    finally:
        B.dgfs_batch_destroy(b)
    g = B.dgfs_graph_capture([i["plan"]._h for i in sub], [i["P"] for i in sub], f_g, Q_g, dt=dt, steps=2)
    try:
        B.dgfs_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        B.dgfs_graph_destroy(g)
    for a, c in zip(f_b, f_g):
        assert torch.equal(a, c)


def test_batch_rejects_repeated_plan_and_stale_configuration(worklist):
    inst = worklist[0]
    Q = torch.empty(inst["P"], 2, 2, 16, 16, 16, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_batch_create([inst["plan"]._h] * 2, [inst["P"]] * 2, [inst["f"]] * 2, [Q] * 2)
    assert e.value.status == 1
    b = B.dgfs_batch_create([inst["plan"]._h], [inst["P"]], [inst["f"]], [Q])
    try:
        inst["plan"].set_kernel_variant(0)
        with pytest.raises(B.DgfsError) as e:
            B.dgfs_batch_launch(b)
        assert e.value.status == 1
    finally:
        B.dgfs_batch_destroy(b)


def test_batch_instances_match_oracle(batch):
    for inst in batch:
        Q = inst["plan"].collide(inst["f"]).double().cpu().numpy()
        prob = O.Problem(**{k: inst["pb"][k] for k in ("N", "L", "M", "Nrho", "masses", "pairs")})
        Qo = prob.collide_all(inst["fnp"])
        tol = 1e-12 if inst["plan"].precision == B.FP64 else 1e-5
        assert np.abs(Q - Qo).max() <= tol * np.abs(Qo).max()


def test_relax_step_and_graph_of_relaxation_steps():
    inst = _instance(8, 2, 6, 4, 2, "fp64", 7)
    plan, f0 = inst["plan"], inst["f"]
    dt = 0.05
    # reference: two explicit Euler steps with separate calls
    f = f0.clone()
    for _ in range(2):
        Q = plan.collide(f)
        ref = f + dt * Q.sum(dim=2)
        plan.relax_step(f, Q, dt)
        torch.cuda.synchronize()
        assert torch.allclose(f, ref, rtol=0, atol=1e-15 * float(ref.abs().max()))
    # the same two steps inside one graph
    fg = f0.clone()
    Qg = torch.empty_like(Q)
    g = B.dgfs_graph_capture([plan._h], [2], [fg], [Qg], dt=dt, steps=2)
    try:
        B.dgfs_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        B.dgfs_graph_destroy(g)
    assert torch.equal(fg, f)


def test_relaxation_mass_change_equals_moment_of_q():
    """f_p <- f_p + dt sum_q Q^(pq): the change of h^3 sum f_p over one step is
    dt times the mass moment of sum_q Q^(pq) reported by dgfs_moments."""
    inst = _instance(16, 2, 12, 8, 1, "fp64", 9)
    plan, f = inst["plan"], inst["f"].clone()
    h3 = (2 * inst["pb"]["L"] / 16) ** 3
    dt = 0.02
    m0 = f.sum(dim=(2, 3, 4)) * h3
    Q = plan.collide(f)
    mom = plan.moments(Q)  # [P][S][S][5]
    plan.relax_step(f, Q, dt)
    torch.cuda.synchronize()
    m1 = f.sum(dim=(2, 3, 4)) * h3
    expect = dt * mom[..., 0].sum(dim=2)
    assert torch.allclose(m1 - m0, expect, rtol=1e-9, atol=1e-13)


def test_autotune_keeps_results():
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 1)
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float32)
    best = plan.autotune(f)
    assert best > 0
    info = plan.info()
    assert info["tuned"] == 1
    Q = plan.collide(f).double().cpu().numpy()
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(pb["f"])
    assert np.abs(Q - Qo).max() <= 1e-5 * np.abs(Qo).max()


def test_autotune_rejects_fp64_plans():
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    f = torch.from_numpy(pb["f"]).cuda()
    with pytest.raises(B.DgfsError) as e:
        plan.autotune(f)
    assert e.value.status == 5


@pytest.mark.parametrize("N,S,M,P", [(8, 1, 6, 24), (8, 2, 12, 24), (16, 2, 6, 6), (24, 2, 6, 4)])
def test_batch_on_fresh_plans_matches_oracle(N, S, M, P):
    """The work list run first, on plans that never ran a plain call (so no
    workspace contents from an earlier call can stand in for a missing write),
    against the oracle."""
    inst = _instance(N, S, M, 4, P, "fp32_tc", 40 + N)
    Q = torch.full((P, S, S, N, N, N), float("nan"), dtype=torch.float32, device="cuda")
    b = B.dgfs_batch_create([inst["plan"]._h], [P], [inst["f"]], [Q])
    try:
        B.dgfs_batch_launch(b)
        torch.cuda.synchronize()
    finally:
        B.dgfs_batch_destroy(b)
    inst["plan"].check()
    pb = inst["pb"]
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(inst["f"].double().cpu().numpy())
    assert np.abs(Q.double().cpu().numpy() - Qo).max() <= 1e-5 * np.abs(Qo).max()
