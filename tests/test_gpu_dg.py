"""1-D DG transport around the operator on the GPU (dgfs_dg_*) against the
DG oracle (oracle/dg.py) and the collision oracle: right-hand sides, mass
conservation with zero-flux walls, SSP-RK3 steps with and without collisions,
graph capture, argument errors."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import dg as ODG
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WALLS = ((1.0, (0.0, -0.2, 0.0)), (2.0, (0.0, 0.2, 0.1)))


def _setup(prec, N=8, L=5.0, M=6, Nrho=4, Ne=4, K=3, masses=(1.0, 2.0), seed=3):
    pairs = W.pair_params([0.81, 0.75][: len(masses)], [1.0, 1.4][: len(masses)], [1.0, 1.2][: len(masses)])
    P = Ne * K
    plan = B.Plan(N, L, M, Nrho, list(masses), pairs, prec, P)
    slab = B.Slab(plan, Ne, K, 0.0, 1.0, WALLS)
    rng = np.random.default_rng(seed)
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    ref = ODG.Slab(Ne, K, 0.0, 1.0, N, L, masses, WALLS)
    prob = O.Problem(N, L, M, Nrho, list(masses), pairs)
    return plan, slab, f, ref, prob


def _flat(a):
    return a.reshape(a.shape[0], a.shape[1], -1)


def test_nodes_match_oracle():
    plan, slab, f, ref, _ = _setup("fp64")
    assert np.abs(slab.x - ref.x).max() < 1e-15


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_transport_rhs_fp64_matches_oracle(K):
    plan, slab, f, ref, _ = _setup("fp64", Ne=3, K=K)
    fd = torch.from_numpy(f).cuda()
    r = slab.rhs(fd).cpu().numpy()
    ro = ref.streaming(_flat(f))
    assert np.abs(_flat(r) - ro).max() <= 1e-13 * np.abs(ro).max()


def test_rhs_with_collisions_fp64_matches_oracle():
    plan, slab, f, ref, prob = _setup("fp64")
    fd = torch.from_numpy(f).cuda()
    Q = plan.collide(fd)
    r = slab.rhs(fd, Q).cpu().numpy()
    Qn = Q.cpu().numpy()
    ro = ref.rhs(_flat(f), Qn.reshape(Qn.shape[0], Qn.shape[1], Qn.shape[2], -1))
    assert np.abs(_flat(r) - ro).max() <= 1e-13 * np.abs(ro).max()
    # and the collision part itself is the oracle's
    Qo = prob.collide_all(f)
    assert np.abs(Q.cpu().numpy() - Qo).max() <= 1e-12 * np.abs(Qo).max()


def test_transport_rhs_fp32_matches_oracle():
    plan, slab, f, ref, _ = _setup("fp32_tc")
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    r = slab.rhs(fd).double().cpu().numpy()
    ro = ref.streaming(_flat(fd.double().cpu().numpy()))
    assert np.abs(_flat(r) - ro).max() <= 1e-6 * np.abs(ro).max()


def test_transport_conserves_mass_with_zero_flux_walls():
    plan, slab, f, ref, _ = _setup("fp64", Ne=5, K=3)
    r = _flat(slab.rhs(torch.from_numpy(f).cuda()).cpu().numpy())
    rate, scale = ref.mass_rate(r), ref.mass_rate(np.abs(r))
    assert np.all(np.abs(rate) <= 1e-13 * scale)


def test_transport_step_fp64_matches_oracle():
    plan, slab, f, ref, _ = _setup("fp64")
    fd = torch.from_numpy(f).cuda()
    dt = 0.01
    slab.step(fd, dt, with_collisions=False)
    fo = ref.ssp_rk3(_flat(f), dt)
    d_gpu, d_orc = _flat(fd.cpu().numpy()) - _flat(f), fo - _flat(f)
    assert np.abs(d_gpu - d_orc).max() <= 1e-12 * np.abs(d_orc).max()


def _oracle_collide(prob, shape):
    def col(g):
        Q = prob.collide_all(g.reshape(shape))
        return Q.reshape(Q.shape[0], Q.shape[1], Q.shape[2], -1)
    return col


def test_collisional_step_fp64_matches_oracle():
    plan, slab, f, ref, prob = _setup("fp64")
    fd = torch.from_numpy(f).cuda()
    dt = 0.01
    slab.step(fd, dt)
    fo = ref.ssp_rk3(_flat(f), dt, _oracle_collide(prob, f.shape))
    d_gpu, d_orc = _flat(fd.cpu().numpy()) - _flat(f), fo - _flat(f)
    assert np.abs(d_gpu - d_orc).max() <= 1e-11 * np.abs(d_orc).max()


def test_collisional_step_tensor_cores_matches_oracle():
    plan, slab, f, ref, prob = _setup("fp32_tc")
    f32 = torch.from_numpy(f).to("cuda", torch.float32)
    f0 = f32.double().cpu().numpy()
    dt = 0.01
    slab.step(f32, dt)
    fo = ref.ssp_rk3(_flat(f0), dt, _oracle_collide(prob, f.shape))
    d_gpu, d_orc = _flat(f32.double().cpu().numpy()) - _flat(f0), fo - _flat(f0)
    assert np.abs(d_gpu - d_orc).max() <= 2e-5 * np.abs(d_orc).max()


def test_step_replays_from_a_cuda_graph():
    plan, slab, f, ref, _ = _setup("fp64")
    fe = torch.from_numpy(f).cuda()
    fg = fe.clone()
    slab.step(fe, 0.01)
    slab.step(fe, 0.01)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        slab.step(fg.clone(), 0.01)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        slab.step(fg, 0.01)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(fg, fe)


def test_bad_arguments_are_status_codes():
    pairs = W.pair_params([0.81], [1.0], [1.0])
    plan = B.Plan(8, 5.0, 6, 4, [1.0], pairs, "fp64", 6)
    with pytest.raises(B.DgfsError) as e:
        B.Slab(plan, 2, 6, 0.0, 1.0, WALLS)  # K > 5
    assert e.value.status == 1
    with pytest.raises(B.DgfsError) as e:
        B.Slab(plan, 3, 3, 0.0, 1.0, WALLS)  # Ne K = 9 > max_points = 6
    assert e.value.status == 1
    with pytest.raises(B.DgfsError) as e:
        B.Slab(plan, 2, 3, 0.0, 1.0, ((0.0, (0, 0, 0)), (1.0, (0, 0, 0))))  # T = 0
    assert e.value.status == 1


def test_heat_slab_full_size_transport():
    """The benchmark's DG workload (16 elements x 3 points, N = 32, M = 12,
    N_rho = 8, walls at T = 1 and T = 2) in its launch configuration: the
    transport right-hand side at every point against the DG oracle."""
    pb = W.make_problem("c5_heat_slab_n32")
    P = pb["f"].shape[0]
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", P)
    slab = B.Slab(plan, pb["elements"], pb["order"], 0.0, 1.0, pb["walls"])
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float32)
    r = slab.rhs(f).double().cpu().numpy()
    ref = ODG.Slab(pb["elements"], pb["order"], 0.0, 1.0, pb["N"], pb["L"], pb["masses"], pb["walls"])
    ro = ref.streaming(_flat(f.double().cpu().numpy()))
    assert np.abs(_flat(r) - ro).max() <= 1e-6 * np.abs(ro).max()
    rate, scale = ref.mass_rate(_flat(r)), ref.mass_rate(np.abs(_flat(r)))
    assert np.all(np.abs(rate) <= 1e-6 * scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32_tc", 1e-6)])
def test_split_slab_with_trace_halos_equals_whole_slab(prec, tol):
    """Two halves of the slab on one GPU, run one after the other (no kernel
    waits on another), with the boundary traces handed across before every
    stage: the right-hand side and one collisional SSP-RK3 step equal those
    of the whole slab."""
    from paper_1903_04670_gb300 import distributed as D

    plan, slab, f, ref, prob = _setup(prec, Ne=4, K=3)
    K = 3
    halves = [B.Slab(plan, 2, K, 0.0, 0.5, WALLS), B.Slab(plan, 2, K, 0.5, 1.0, WALLS)]
    fd = torch.from_numpy(f).to("cuda", plan.dtype)
    parts = [fd[: 2 * K].clone(), fd[2 * K:].clone()]

    def exchange(fs):
        tr = [h.traces(x) for h, x in zip(halves, fs)]
        return [(None, tr[1][0]), (tr[0][1], None)]  # (halo_left, halo_right) per half

    full = slab.rhs(fd).double()
    hal = exchange(parts)
    got = torch.cat([h.rhs_halo(x, None, *hl) for h, x, hl in zip(halves, parts, hal)]).double()
    assert (got - full).abs().max() <= tol * full.abs().max()

    dt = 0.01
    whole = fd.clone()
    slab.step(whole, dt)
    work = [(torch.empty_like(x), torch.empty_like(x)) for x in parts]
    for k, (src, a0, a1) in enumerate(D.SSP_RK3):
        bufs = [(x, w[0], w[1]) for x, w in zip(parts, work)]
        fins = [b[src] for b in bufs]
        hal = exchange(fins)
        for i, h in enumerate(halves):
            out = (bufs[i][1], bufs[i][2], bufs[i][0])[k]
            h.stage(fins[i], parts[i] if a0 != 0.0 else None, out, a0, a1, dt, True, *hal[i])
    got = torch.cat(parts).double()
    d_ref = (whole.double() - fd.double())
    assert (got - whole.double()).abs().max() <= max(tol, 1e-12) * d_ref.abs().max() * 10
