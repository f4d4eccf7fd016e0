"""GPU parity at the full sizes of the paper-shaped workloads, against the FP64
oracle.

* The 1-D slab workload (24 points x 4 pairs, N = 32, M = 12, N_rho = 8, VSS)
  in the benchmark's launch configuration (autotuned): every (point, pair) of
  the 3xTF32 and split-BF16 forms.
* The adjoint workload (64 points x 2 species x 32^3, float32) through
  torch.autograd: df at four spread points against the oracle adjoint, and
  dL/d omega against the per-point sum of the FP64 plan's adjoint, whose
  per-point values are checked against the oracle at those points.
* The uneven relaxation workload (256 problems, N in {24, 32, 48}, S in
  {2, 3}, M in {6, 12}, N_rho in {8, 16}) through the batched work list replayed
  from a CUDA graph: one problem of every (N, S, M, N_rho) group against the
  oracle; and the benchmark's own uneven-batch code path on a reduced set.
* The trace-halo split of the DG slab (Sec. 3.3's linear domain
  decomposition) against the DG oracle with halos, and its collisional
  SSP-RK3 step against the oracle's step of the whole slab.
* The heat-transfer slab (48 points) in full: every stage of one collisional
  SSP-RK3 step against the DG oracle plus the collision oracle at sampled
  points, given the GPU's input to that stage.

Bounds as in test_gpu_tc.py: per (point, pair)
  ||Q_gpu - Q_orc||_inf <= tol ||Q^pq_orc||_inf + 0.1 tol ||gain^pq||_inf,
tol = 1e-5 (3xTF32) or 1e-3 (split BF16); over a batch, tol ||Q_orc||_inf.
"""
import concurrent.futures
import os
import sys

import numpy as np
import pytest
import torch

import oracle as O
from oracle import dg as ODG
from paper_1903_04670_gb300 import autograd as AG
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORES = len(os.sched_getaffinity(0))
TOL = {"fp32_tc": 1e-5, "bf16x3": 1e-3}


def _pool(fn, jobs):
    """Run oracle calls in parallel threads (the oracle's C calls release the GIL)."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=CORES) as ex:
        return list(ex.map(lambda j: fn(*j), jobs))


def _collide(pair, fp, fq):
    return pair.collide(fp, fq)


def _check_pair(Qg, Qo, d, tol, where):
    err = float(np.abs(Qg - Qo).max())
    bound = tol * float(np.abs(Qo).max()) + 0.1 * tol * d["gain_max"]
    assert err <= bound, (where, err, float(np.abs(Qo).max()), d["gain_max"])
    return err


# ----------------------------------------------------------- slab workload
@pytest.fixture(scope="module")
def c2_oracle():
    pb = W.make_problem("c2_slab_n32")
    O.set_threads(CORES)
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    O.set_threads(1)
    f = pb["f"]
    P, S = f.shape[0], f.shape[1]
    jobs = [(prob.pair(p, q), f[pt, p], f[pt, q]) for pt in range(P) for p in range(S) for q in range(S)]
    res = _pool(_collide, jobs)
    O.set_threads(CORES)
    N = pb["N"]
    Qo = np.stack([r[0] for r in res]).reshape(P, S, S, N, N, N)
    diag = [r[1] for r in res]
    return pb, Qo, diag


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x3"])
def test_slab_workload_every_point_and_pair(c2_oracle, prec):
    pb, Qo, diag = c2_oracle
    f = pb["f"]
    P, S = f.shape[0], f.shape[1]
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P)
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    Q = plan.collide(fd)
    plan.autotune(fd, Q)  # the benchmark's launch configuration
    plan.collide(fd, Q)
    plan.check()
    Qg = Q.double().cpu().numpy()
    tol = TOL[prec]
    k = 0
    for pt in range(P):
        for p in range(S):
            for q in range(S):
                _check_pair(Qg[pt, p, q], Qo[pt, p, q], diag[k], tol, (prec, pt, p, q))
                k += 1
    batch = float(np.abs(Qg - Qo).max() / np.abs(Qo).max())
    assert batch < tol
    print("slab workload %s: batch rel. max-norm error %.3e over %d evaluations" % (prec, batch, P * S * S))


# --------------------------------------------------------- adjoint workload
def _adjoint(pair, fp, fq, g):
    return pair.adjoint(fp, fq, g)


def test_adjoint_workload_full_size_through_autograd():
    pb = W.make_problem("c4_adjoint_n32", dtype=np.float32)
    N, L, P = pb["N"], pb["L"], pb["f"].shape[0]
    S = len(pb["masses"])
    assert P == 64
    op = AG.CollisionOperator(N, L, pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", P)
    c = torch.from_numpy(W.velocity_grid(N, L)).cuda()
    cx, cy, cz = torch.meshgrid(c, c, c, indexing="ij")
    rng = np.random.default_rng(4)
    wts = torch.from_numpy(rng.normal(size=(S, S, 4))).cuda()
    basis = torch.stack([torch.ones_like(cx), cx, cx ** 2 + cy ** 2 + cz ** 2, cx * cy])
    wgt = torch.einsum("pqk,kxyz->pqxyz", wts, basis)  # [S, S, N, N, N] FP64
    f = torch.from_numpy(pb["f"]).cuda().requires_grad_(True)
    omega = op.omega.clone().requires_grad_(True)
    Q = op(f, omega)
    loss = (Q.double() * wgt[None]).sum()
    loss.backward()
    torch.cuda.synchronize()

    # an omega other than the plan's is refused (the tables are built for it)
    with pytest.raises(ValueError):
        op(f.detach(), (op.omega + 1e-3).requires_grad_(True))

    f64 = pb["f"].astype(np.float64)
    # Q is float32, so autograd hands the backward dL/dQ = wgt rounded to
    # float32: the references below take exactly that upstream gradient
    gq = wgt.to(torch.float32).to(torch.float64)
    g = gq.cpu().numpy()
    pts = [0, 21, 42, 63]
    O.set_threads(CORES)
    prob = O.Problem(N, L, pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    O.set_threads(1)
    jobs = [(prob.pair(p, q), f64[pt, p], f64[pt, q], g[p, q]) for pt in pts for p in range(S) for q in range(S)]
    res = _pool(_adjoint, jobs)
    O.set_threads(CORES)
    dfo = np.zeros((len(pts), S) + (N, N, N))
    domo = np.zeros((len(pts), S * S))
    k = 0
    for i, pt in enumerate(pts):
        for p in range(S):
            for q in range(S):
                dp, dq, dw = res[k]
                dfo[i, p] += dp
                dfo[i, q] += dq
                domo[i, p * S + q] = dw
                k += 1
    bwd_fp64 = op.bwd.precision == B.FP64
    # the gradient comes back in f's dtype (float32): FP64 adjoint values
    # rounded to float32 are within a few float32 ulps of the largest entry
    tol_df = 4 * float(np.finfo(np.float32).eps) if bwd_fp64 else 1e-5
    got = f.grad.double().cpu().numpy()
    for i, pt in enumerate(pts):
        assert np.abs(got[pt] - dfo[i]).max() <= tol_df * np.abs(dfo[i]).max(), pt

    # dL/d omega: the per-point FP64 adjoint (checked against the oracle at the
    # sampled points) summed over all 64 points equals the autograd result
    plan64 = B.Plan(N, L, pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    fd64 = torch.from_numpy(f64).cuda()
    gd = gq[None].contiguous()
    per_pt = []
    for pt in range(P):
        _, dw = plan64.backward(fd64[pt:pt + 1].contiguous(), gd)
        per_pt.append(dw.cpu().numpy().reshape(S * S))
    per_pt = np.array(per_pt)
    for i, pt in enumerate(pts):
        # dL/d omega sums g dQ/d omega over the grid with cancellation: FP64 to ~1e-10
        assert np.abs(per_pt[pt] - domo[i]).max() <= 1e-9 * np.abs(domo[i]).max(), pt
    tot = per_pt.sum(0)
    got_w = omega.grad.cpu().numpy().reshape(S * S)
    if bwd_fp64:
        assert np.abs(got_w - tot).max() <= 1e-9 * np.abs(tot).max()
    else:
        # dL/d omega sums beta (sum_rs wlog_rs <V_rs, A_rs B_rs> - <g f_p, Re S_w f_q>) and
        # dlnbeta <g, Q>: gain-level terms that cancel against the loss to the
        # size of <g, Q> itself (conservation makes the moment weights nearly
        # orthogonal to Q; on this workload sum |g dQ/domega| is 50-70 times
        # |<g, dQ/domega>| and the gain 25 times Q).  Its tensor-core error is
        # therefore of the order of the tensor-core forward's error in the same
        # functional <g, Q>: bounded here by ten times that error (per pair, against
        # the FP64 forward) plus the form's 1e-5.
        p64P = B.Plan(N, L, pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", P)
        Q64 = p64P.collide(fd64)
        Qt = op.fwd.collide(f.detach())
        gQ64 = (gq[None] * Q64).sum(dim=(0, 3, 4, 5)).reshape(S * S).cpu().numpy()
        gQt = (gq[None] * Qt.double()).sum(dim=(0, 3, 4, 5)).reshape(S * S).cpu().numpy()
        eQ = np.abs(gQt - gQ64) / np.abs(gQ64)
        ew = np.abs(got_w - tot) / np.abs(tot)
        assert np.all(ew <= 10 * eQ + 1e-5), (ew.tolist(), eQ.tolist())


# ------------------------------------------------------------ uneven batch
def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


SAMPLED_PAIRS = {2: [(0, 0), (0, 1), (1, 0), (1, 1)], 3: [(0, 1), (1, 2), (2, 0), (2, 2)]}


def test_uneven_relaxation_batch_matches_oracle():
    """All 256 problems (86 plans) through the batched work list, replayed from
    a CUDA graph; one problem of each of the 24 (N, S, M, N_rho) groups is
    compared with the oracle (all pairs for S = 2, four of nine for S = 3)."""
    bench = _bench()
    groups, plans, fs, Qs = bench.uneven_plans(B, W, torch, np, "fp32_tc", 0)
    assert sum(len(g) for g in groups) == 256
    bt = B.Batch(plans, fs, Qs)
    try:
        bt.launch()  # eager once (warm-up), then the captured pass
        torch.cuda.synchronize()
        for Q in Qs:
            Q.zero_()
        cg = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(cg, stream=cs):
            bt.launch(cs)
        cg.replay()
        torch.cuda.synchronize()
    finally:
        bt.close()
    for pl in plans:
        pl.check()
    seen = {}
    for i, xs in enumerate(groups):
        x = xs[0]
        key = (x["N"], len(x["masses"]), x["M"], x["Nrho"])
        if key not in seen:
            seen[key] = (i, 0, x)
    assert len(seen) == 24
    O.set_threads(CORES)
    jobs, where = [], []
    for key, (i, j, x) in sorted(seen.items()):
        S = len(x["masses"])
        for (p, q) in SAMPLED_PAIRS[S]:
            pr = x["pairs"][p * S + q]
            pair = O.Pair(x["N"], x["L"], x["M"], x["Nrho"], x["masses"][p], x["masses"][q],
                          pr["omega"], pr["alpha"], pr["d"])
            jobs.append((pair, x["f"][0, p], x["f"][0, q]))
            where.append((key, i, j, p, q))
    O.set_threads(1)
    res = _pool(_collide, jobs)
    O.set_threads(CORES)
    for (key, i, j, p, q), (Qo, d) in zip(where, res):
        Qg = Qs[i][j, p, q].double().cpu().numpy()
        _check_pair(Qg, Qo, d, TOL["fp32_tc"], (key, p, q))


def test_benchmark_uneven_batch_code_path_reduced():
    """The benchmark's uneven-batch section on a reduced set: it must run
    without error (the benchmark only reports an error in its JSON)."""
    bench = _bench()
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 1)
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float32)
    Q = plan.collide(f)
    flush = torch.empty(1 << 20, dtype=torch.float32, device="cuda")
    res = bench.uneven_batch(B, W, torch, np, "fp32_tc", 0, flush, torch.cuda.current_stream(), plan,
                             {"f": f, "Q": Q}, count=12, reps=1)
    for k in ("separate_calls", "graph_of_calls", "batch", "batch_graph", "one_instance"):
        assert k in res, k
    assert res["instances"] == 12 and res["evals_per_pass"] > 0
    assert res["batch"]["evals_per_s"] > 0


# ------------------------------------------------- DG slab split by traces
WALLS = ((1.0, (0.0, -0.2, 0.0)), (2.0, (0.0, 0.2, 0.1)))


def _flat(a):
    return a.reshape(a.shape[0], a.shape[1], -1)


@pytest.mark.parametrize("prec,tol_rhs,tol_step", [("fp64", 1e-13, 1e-11), ("fp32_tc", 1e-6, 2e-5)])
def test_split_slab_with_trace_halos_matches_oracle(prec, tol_rhs, tol_step):
    from paper_1903_04670_gb300 import distributed as D

    N, L, M, Nrho, K = 8, 5.0, 6, 4, 3
    masses = [1.0, 2.0]
    pairs = W.pair_params([0.81, 0.75], [1.0, 1.4], [1.0, 1.2])
    plan = B.Plan(N, L, M, Nrho, masses, pairs, prec, 2 * K)
    halves = [B.Slab(plan, 2, K, 0.0, 0.5, WALLS), B.Slab(plan, 2, K, 0.5, 1.0, WALLS)]
    rng = np.random.default_rng(31)
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(4 * K)])
    fd = torch.from_numpy(f).to("cuda", plan.dtype)
    f0 = fd.double().cpu().numpy()
    parts = [fd[: 2 * K].clone(), fd[2 * K:].clone()]
    oh = [ODG.Slab(2, K, 0.0, 0.5, N, L, masses, WALLS), ODG.Slab(2, K, 0.5, 1.0, N, L, masses, WALLS)]

    # right-hand side of each half with the neighbour's trace as its halo
    tr = [h.traces(x) for h, x in zip(halves, parts)]
    got = [halves[0].rhs_halo(parts[0], None, None, tr[1][0]), halves[1].rhs_halo(parts[1], None, tr[0][1], None)]
    fo = [_flat(f0[: 2 * K]), _flat(f0[2 * K:])]
    otr = [o.traces(x) for o, x in zip(oh, fo)]
    ref = [oh[0].streaming(fo[0], None, otr[1][0]), oh[1].streaming(fo[1], otr[0][1], None)]
    for gh, rh in zip(got, ref):
        assert np.abs(_flat(gh.double().cpu().numpy()) - rh).max() <= tol_rhs * np.abs(rh).max()

    # one collisional SSP-RK3 step of the split slab against the oracle's
    # step of the whole slab (oracle collisions)
    dt = 0.01
    work = [(torch.empty_like(x), torch.empty_like(x)) for x in parts]
    for k, (src, a0, a1) in enumerate(D.SSP_RK3):
        bufs = [(x, w[0], w[1]) for x, w in zip(parts, work)]
        fins = [b[src] for b in bufs]
        tr = [h.traces(x) for h, x in zip(halves, fins)]
        hal = [(None, tr[1][0]), (tr[0][1], None)]
        for i, h in enumerate(halves):
            out = (bufs[i][1], bufs[i][2], bufs[i][0])[k]
            h.stage(fins[i], parts[i] if a0 != 0.0 else None, out, a0, a1, dt, True, *hal[i])
    got = _flat(torch.cat(parts).double().cpu().numpy())
    whole = ODG.Slab(4, K, 0.0, 1.0, N, L, masses, WALLS)
    prob = O.Problem(N, L, M, Nrho, masses, pairs)

    def col(g):
        Q = prob.collide_all(g.reshape(f.shape))
        return Q.reshape(Q.shape[0], Q.shape[1], Q.shape[2], -1)

    fo_new = whole.ssp_rk3(_flat(f0), dt, col)
    d_orc = fo_new - _flat(f0)
    assert np.abs((got - _flat(f0)) - d_orc).max() <= tol_step * np.abs(d_orc).max()


# --------------------------------------------- heat slab, full collisional
def test_heat_slab_full_size_collisional_stages_sampled():
    """The DG benchmark workload (16 elements x 3 points = 48 points, N = 32,
    M = 12, N_rho = 8, walls at T = 1 and 2) in its launch configuration: each
    SSP-RK3 stage's output at sampled points equals a0 f0 + a1 (f_in + dt
    (streaming(f_in) + sum_q Q(f_in))) with the DG oracle's streaming and the
    collision oracle, given the GPU's input f_in to that stage."""
    from paper_1903_04670_gb300 import distributed as D

    pb = W.make_problem("c5_heat_slab_n32")
    N, P = pb["N"], pb["f"].shape[0]
    S = len(pb["masses"])
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", P)
    slab = B.Slab(plan, pb["elements"], pb["order"], 0.0, 1.0, pb["walls"])
    ref = ODG.Slab(pb["elements"], pb["order"], 0.0, 1.0, N, pb["L"], pb["masses"], pb["walls"])
    O.set_threads(CORES)
    prob = O.Problem(N, pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float32)
    f1, f2 = torch.empty_like(f), torch.empty_like(f)
    bufs, outs = (f, f1, f2), (f1, f2, f)
    f0 = _flat(f.double().cpu().numpy())
    dt = 1e-3
    pts = [0, 23, 47]
    for k, (src, a0, a1) in enumerate(D.SSP_RK3):
        fin = _flat(bufs[src].double().cpu().numpy())
        slab.stage(bufs[src], f if a0 != 0.0 else None, outs[k], a0, a1, dt, True)
        out = _flat(outs[k].double().cpu().numpy())
        stream = ref.streaming(fin)
        Qo = prob.collide_all(fin.reshape(pb["f"].shape), points=pts).reshape(len(pts), S, S, -1)
        for i, pt in enumerate(pts):
            inc = a1 * dt * (stream[pt] + Qo[i].sum(axis=1))
            expect = a0 * f0[pt] + a1 * fin[pt] + inc
            # FP32 operator and transport on the increment, plus float32 storage of the stage output
            bound = 2e-5 * np.abs(inc).max() + 4 * np.finfo(np.float32).eps * np.abs(expect).max()
            assert np.abs(out[pt] - expect).max() <= bound, (k, pt)
    plan.check()
