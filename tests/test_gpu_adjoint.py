"""GPU adjoint (dgfs_collide_backward) against the oracle's FP64 adjoint, the
dot-product identity of the bilinear map, and central finite differences in
omega; plus the torch.autograd wrapper.  The FP64 plans' adjoint runs in FP64;
the tensor-core plans' adjoint runs its (rho, sigma) loop on the tensor cores
in the plan's operand format (bounds as the forward's: 1e-5 for 3xTF32, 1e-3
for split BF16, relative to the largest entry)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1903_04670_gb300 import autograd as AG
from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(N, M, Nrho, S, P, seed, alpha=1.3):
    rng = np.random.default_rng(seed)
    masses = [1.0, 2.5, 0.7, 1.6][:S]
    pairs = W.pair_params([0.72, 0.8, 0.9, 0.75][:S], [alpha, 1.0, 1.2, 1.1][:S], [1.0, 1.1, 0.9, 1.05][:S])
    L = 0.5 * N
    f = np.stack([np.stack([W.two_maxwellians(rng, N, L, m) for m in masses]) for _ in range(P)])
    g = rng.normal(size=(P, S, S, N, N, N))
    return dict(N=N, L=L, M=M, Nrho=Nrho, masses=masses, pairs=pairs), f, g


def _oracle_grads(pb, f, g):
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    P, S = f.shape[0], f.shape[1]
    df = np.zeros_like(f)
    dom = np.zeros(S * S)
    for pt in range(P):
        for p in range(S):
            for q in range(S):
                dp, dq, dw = prob.pair(p, q).adjoint(f[pt, p], f[pt, q], g[pt, p, q])
                df[pt, p] += dp
                df[pt, q] += dq
                dom[p * S + q] += dw
    return df, dom


@pytest.mark.parametrize("N,M,Nrho,S,P", [(8, 12, 4, 2, 2), (12, 6, 3, 3, 1), (16, 6, 4, 2, 1)])
def test_gpu_adjoint_matches_oracle_adjoint(N, M, Nrho, S, P):
    pb, f, g = _problem(N, M, Nrho, S, P, seed=N + S)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", P)
    df, dom = plan.backward(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    dfo, domo = _oracle_grads(pb, f, g)
    assert np.abs(df.cpu().numpy() - dfo).max() <= 1e-11 * np.abs(dfo).max()
    assert np.abs(dom.cpu().numpy() - domo).max() <= 1e-10 * np.abs(domo).max()


def test_gpu_dot_product_identity():
    pb, f, g = _problem(8, 12, 4, 2, 1, seed=3)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    fd = torch.from_numpy(f).cuda()
    gd = torch.from_numpy(g).cuda()
    df, _ = plan.backward(fd, gd)
    d = torch.randn_like(fd)
    # <g, dQ/df [d]> = <g, Q(f + d) - Q(f)> up to the quadratic term: Q is bilinear, so
    # d/dt Q(f + t d) at t = 0 equals Q(f + d) - Q(f) - (Q(d) restricted to both slots) ...
    # use the exact identity: J d = Q(f+d) - Q(f-d) over 2 (central difference is exact
    # for a quadratic map)
    Qp = plan.collide((fd + d).contiguous())
    Qm = plan.collide((fd - d).contiguous())
    lhs = float((gd * (Qp - Qm) / 2).sum())
    rhs = float((df * d).sum())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + float(df.abs().max()))


def test_gpu_omega_gradient_finite_difference():
    pb, f, g = _problem(8, 6, 4, 2, 1, seed=5)
    fd = torch.from_numpy(f).cuda()
    gd = torch.from_numpy(g).cuda()
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    _, dom = plan.backward(fd, gd)
    h = 1e-4
    S = 2
    for k in range(S * S):
        vals = []
        for sgn in (+1, -1):
            pairs = [dict(p) for p in pb["pairs"]]
            pairs[k]["omega"] += sgn * h
            pl = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pairs, "fp64", 1)
            Q = pl.collide(fd)
            vals.append(float((gd[:, k // S, k % S] * Q[:, k // S, k % S]).sum()))
        fdiff = (vals[0] - vals[1]) / (2 * h)
        assert abs(float(dom[k]) - fdiff) <= 1e-6 * max(1.0, abs(fdiff)), (k, float(dom[k]), fdiff)


def test_autograd_moment_loss_c4_shape():
    """Configuration 4's loss: weighted velocity moments (1, v, |v|^2, v_x v_y) of
    Q^(pq); float32 f on the tensor-core forward, gradients from its tensor-core
    adjoint, checked against the oracle adjoint at one sampled point."""
    pb = W.make_problem("c4_adjoint_n32", points=2, dtype=np.float32)
    N, L = pb["N"], pb["L"]
    op = AG.CollisionOperator(N, L, pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 2)
    c = torch.from_numpy(W.velocity_grid(N, L)).cuda()
    cx, cy, cz = torch.meshgrid(c, c, c, indexing="ij")
    rng = np.random.default_rng(4)
    wts = torch.from_numpy(rng.normal(size=(2, 2, 4))).cuda()
    basis = torch.stack([torch.ones_like(cx), cx, cx ** 2 + cy ** 2 + cz ** 2, cx * cy])  # [4, N, N, N]
    f = torch.from_numpy(pb["f"]).cuda().requires_grad_(True)
    omega = op.omega.clone().requires_grad_(True)
    Q = op(f, omega)
    wgt = torch.einsum("pqk,kxyz->pqxyz", wts, basis)
    loss = (Q.double() * wgt[None]).sum()
    loss.backward()
    g = wgt[None].expand(2, -1, -1, -1, -1, -1).cpu().numpy()
    dfo, domo = _oracle_grads(pb, pb["f"][:1].astype(np.float64), g[:1])
    got = f.grad[0].double().cpu().numpy()
    assert np.abs(got - dfo[0]).max() <= 1e-5 * np.abs(dfo[0]).max()
    # omega gradient sums over both points: compare the FP64 plan's per-point value
    assert omega.grad is not None and omega.grad.shape == (2, 2)
    assert torch.isfinite(omega.grad).all()


TC_TOL = {"fp32_tc": 1e-5, "bf16x3": 1e-3}


def _f32(x):
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("N,M,Nrho,S,P,prec", [(8, 12, 4, 2, 2, "fp32_tc"), (16, 6, 4, 2, 1, "fp32_tc"),
                                               (16, 6, 4, 2, 1, "bf16x3"), (24, 6, 3, 3, 1, "fp32_tc"),
                                               (32, 12, 4, 2, 1, "fp32_tc"), (48, 6, 2, 2, 1, "fp32_tc"),
                                               (48, 6, 2, 2, 1, "bf16x3"), (8, 6, 2, 4, 2, "fp32_tc")])
def test_tc_adjoint_matches_oracle_adjoint(N, M, Nrho, S, P, prec):
    """The tensor-core adjoint (float32 f, dQ) against the oracle's FP64 adjoint
    of the same float32-rounded inputs: df and dL/d omega.  N = 48 runs one
    pipeline per CTA, whose stage B images do not fit next to the data and are
    reloaded per contraction."""
    pb, f, g = _problem(N, M, Nrho, S, P, seed=N + S + 7)
    f, g = _f32(f), _f32(g)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P)
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    gd = torch.from_numpy(g).to("cuda", torch.float32)
    df, dom = plan.backward(fd, gd)
    plan.check()
    torch.cuda.synchronize()
    dfo, domo = _oracle_grads(pb, f, g)
    tol = TC_TOL[prec]
    err_df = np.abs(df.double().cpu().numpy() - dfo).max() / np.abs(dfo).max()
    err_w = np.abs(dom.cpu().numpy() - domo).max() / np.abs(domo).max()
    assert err_df <= tol, err_df
    assert err_w <= tol, err_w


def test_tc_adjoint_chunks_and_repeat():
    """30 points take two launch chunks (24 + 6): two calls in a row give the same
    bits, and every point equals its own one-point call."""
    P = 30
    pb, f, g = _problem(8, 6, 2, 2, P, seed=11)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", P)
    assert plan.info()["chunk"] < P
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    gd = torch.from_numpy(g).to("cuda", torch.float32)
    df1, dom1 = plan.backward(fd, gd)
    df2, dom2 = plan.backward(fd, gd)
    torch.cuda.synchronize()
    assert torch.equal(df1, df2) and torch.equal(dom1, dom2)
    parts = [plan.backward(fd[i:i + 1].contiguous(), gd[i:i + 1].contiguous()) for i in range(P)]
    dfs = torch.cat([p[0] for p in parts])
    doms = sum(p[1] for p in parts)
    assert float((dfs - df1).abs().max()) <= 1e-6 * float(df1.abs().max())
    assert float((doms - dom1).abs().max()) <= 1e-6 * float(dom1.abs().max())


def test_tc_dot_product_identity():
    """<g, J d> = <J^T g, d> with the tensor-core forward and adjoint: J d is the
    exact central difference (Q(f + d) - Q(f - d)) / 2 of the quadratic map."""
    pb, f, g = _problem(16, 6, 4, 2, 1, seed=13)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 1)
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    gd = torch.from_numpy(g).to("cuda", torch.float32)
    df, _ = plan.backward(fd, gd)
    d = torch.randn_like(fd) * fd.abs().max()
    Qp = plan.collide((fd + d).contiguous()).double()
    Qm = plan.collide((fd - d).contiguous()).double()
    lhs = float((gd.double() * (Qp - Qm) / 2).sum())
    rhs = float((df.double() * d.double()).sum())
    scale = float((gd.double().abs() * ((Qp - Qm) / 2).abs()).sum())
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)


def test_tc_adjoint_refuses_hermitian_form():
    pb, f, g = _problem(8, 6, 2, 2, 1, seed=2)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 1)
    plan.set_hermitian(True)
    with pytest.raises(B.DgfsError):
        plan.backward(torch.from_numpy(f).to("cuda", torch.float32), torch.from_numpy(g).to("cuda", torch.float32))


def test_tc_adjoint_tf32_and_collapsed_plans():
    """A single-product TF32 plan's adjoint stays near the 3xTF32 one (TF32 keeps
    about 11 bits per operand), and a VHS plan with the sigma collapse switched on
    (a forward-only variant) gives the same adjoint bits as without it."""
    pb, f, g = _problem(16, 6, 4, 2, 1, seed=17, alpha=1.0)
    args = (pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    fd = torch.from_numpy(f).to("cuda", torch.float32)
    gd = torch.from_numpy(g).to("cuda", torch.float32)
    ref = B.Plan(*args, "fp32_tc", 1)
    df3, dw3 = ref.backward(fd, gd)
    tf = B.Plan(*args, "tf32", 1)
    df1, dw1 = tf.backward(fd, gd)
    col = B.Plan(*args, "fp32_tc", 1)
    col.set_collapse(True)
    dfc, dwc = col.backward(fd, gd)
    torch.cuda.synchronize()
    assert float((df1 - df3).abs().max()) <= 2e-2 * float(df3.abs().max())
    assert float((dw1 - dw3).abs().max()) <= 2e-2 * float(dw3.abs().max())
    assert torch.equal(dfc, df3) and torch.equal(dwc, dw3)
