"""The declared Hermitian form (dgfs_plan_set_hermitian: Algorithm 2 with the
Nyquist planes removed, two spatial points per complex grid slot) against the
oracle's orc_collide_hermitian, for the FP64 path (1e-12) and the tensor-core
forms (3xTF32: 1e-5 with the gain-scaled floor; split BF16: 1e-3), with odd
point counts (a slot whose second point is absent), the sigma collapse, the
switch back to the literal form, and the paths that refuse the form."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(N, M, Nrho, S, P, seed, alpha=(1.4, 1.0, 1.2)):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.0, 4.0][:S]
    pairs = W.pair_params([0.81, 0.75, 0.7][:S], list(alpha[:S]), [1.0, 1.2, 0.9][:S])
    L = N / 3.2
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    return dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs), f


def _gpu(pb, f, prec, herm=True, collapse=None):
    P = f.shape[0]
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P)
    if collapse is not None:
        plan.set_collapse(collapse)
    if herm:
        plan.set_hermitian(True)
    fd = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", plan.dtype)
    Q = plan.collide(fd)
    plan.check()
    return Q.double().cpu().numpy(), plan, fd


def _oracle(pb, f):
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    return prob, prob.collide_all_hermitian(f)


@pytest.mark.parametrize("N,M,Nrho,S,P", [(8, 12, 3, 2, 3), (16, 6, 4, 2, 4), (12, 6, 2, 3, 1), (24, 6, 2, 2, 2)])
def test_fp64_hermitian_matches_oracle(N, M, Nrho, S, P):
    pb, f = _problem(N, M, Nrho, S, P, seed=N + P)
    Qg, _, _ = _gpu(pb, f, "fp64")
    _, Qo = _oracle(pb, f)
    assert np.abs(Qg - Qo).max() <= 1e-12 * np.abs(Qo).max()


@pytest.mark.parametrize("prec,tol", [("fp32_tc", 1e-5), ("bf16x3", 1e-3)])
@pytest.mark.parametrize("N,M,Nrho,S,P", [(8, 12, 3, 3, 3), (16, 6, 4, 2, 5), (24, 6, 3, 2, 2), (32, 12, 2, 2, 3)])
def test_tensor_core_hermitian_matches_oracle(prec, tol, N, M, Nrho, S, P):
    pb, f = _problem(N, M, Nrho, S, P, seed=7 * N + P)
    Qg, _, fd = _gpu(pb, f, prec)
    f32 = fd.double().cpu().numpy()
    prob, Qo = _oracle(pb, f32)
    for pt in range(P):
        for p in range(S):
            for q in range(S):
                _, d = prob.pair(p, q).collide(f32[pt, p], f32[pt, q])
                err = np.abs(Qg[pt, p, q] - Qo[pt, p, q]).max()
                assert err <= tol * np.abs(Qo[pt, p, q]).max() + 0.1 * tol * d["gain_max"], (pt, p, q, err)
    assert np.abs(Qg - Qo).max() <= tol * np.abs(Qo).max()


def test_slab_workload_hermitian_sampled():
    """The benchmark's slab workload (24 points, N = 32, M = 12, N_rho = 8, VSS)
    in the Hermitian form, autotuned, against the oracle at sampled points of
    both parities (real and imaginary halves of a slot)."""
    pb = W.make_problem("c2_slab_n32")
    f = pb["f"]
    P = f.shape[0]
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", P)
    plan.set_hermitian(True)
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    Q = plan.collide(fd)
    plan.autotune(fd, Q)
    plan.collide(fd, Q)
    plan.check()
    Qg = Q.double().cpu().numpy()
    f32 = fd.double().cpu().numpy()
    pts = [0, 7, 12, 23]
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all_hermitian(f32, points=pts)
    assert np.abs(Qg[pts] - Qo).max() <= 1e-5 * np.abs(Qo).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_tc", 1e-5)])
def test_hermitian_with_sigma_collapse(prec, tol):
    pb, f = _problem(16, 12, 3, 2, 3, seed=99, alpha=(1.0, 1.0, 1.0))
    Qg, plan, fd = _gpu(pb, f, prec, collapse=True)
    assert plan.info()["collapse"] == 1
    _, Qo = _oracle(pb, fd.double().cpu().numpy())
    assert np.abs(Qg - Qo).max() <= tol * np.abs(Qo).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc"])
def test_switching_back_gives_the_literal_form(prec):
    pb, f = _problem(16, 6, 3, 2, 2, seed=3)
    Ql, plan, fd = _gpu(pb, f, prec, herm=False)
    plan.set_hermitian(True)
    Qh = plan.collide(fd).double().cpu().numpy()
    plan.set_hermitian(False)
    Ql2 = plan.collide(fd).double().cpu().numpy()
    plan.check()
    assert np.array_equal(Ql, Ql2)
    assert not np.array_equal(Ql, Qh)


def test_paths_that_refuse_the_hermitian_form():
    pb, f = _problem(16, 6, 3, 2, 2, seed=4)
    _, plan, fd = _gpu(pb, f, "fp64")
    Q = torch.empty((2, 2, 2, 16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        plan.backward(fd, Q)
    assert e.value.status == 5
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_collide_noalloc(plan._h, 2, fd, Q)
    assert e.value.status == 5
    _, tplan, tfd = _gpu(pb, f, "fp32_tc")
    Qt = torch.empty((2, 2, 2, 16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.Batch([tplan], [tfd], [Qt])
    assert e.value.status == 5
    big = B.Plan(48, 15.0, 6, 2, [1.0, 2.0], W.pair_params([0.81, 0.81], [1.0, 1.0], [1.0, 1.2]), "fp32_tc", 1)
    with pytest.raises(B.DgfsError) as e:
        big.set_hermitian(True)
    assert e.value.status == 5
