"""The allocation-free entry point dgfs_collide_noalloc (for callers that may
not allocate device memory while they evaluate) against dgfs_collide.

Runs last in the suite (file name) and also stands alone in a fresh process.
The two entry points run the same FP64 kernels on different scratch memory, so
they must agree to the FP64 parity bound; two calls in a row check that the
shared static scratch carries no state from one call into the next."""
import numpy as np
import pytest
import torch

from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_matches_collide_on_two_calls():
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float64)
    Qref = plan.collide(f)
    torch.cuda.synchronize()
    ref = Qref.cpu().numpy()
    for _ in range(2):
        Q = torch.full_like(Qref, float("nan"))
        B.dgfs_collide_noalloc(plan._h, 1, f, Q)
        torch.cuda.synchronize()
        assert _rel(Q.cpu().numpy(), ref) <= TOL64


def test_noalloc_second_input_after_first():
    # a different input on the second call: results follow the input, not the
    # previous call's scratch contents
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    f1 = torch.from_numpy(pb["f"]).to("cuda", torch.float64)
    f2 = (0.5 * f1.flip(-1)).contiguous()
    Q = torch.empty((1, 2, 2, 16, 16, 16), dtype=torch.float64, device="cuda")
    B.dgfs_collide_noalloc(plan._h, 1, f1, Q)
    B.dgfs_collide_noalloc(plan._h, 1, f2, Q)
    ref = plan.collide(f2)
    torch.cuda.synchronize()
    assert _rel(Q.cpu().numpy(), ref.cpu().numpy()) <= TOL64


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pb = W.make_problem("c2_slab_n32", points=1)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    f = torch.zeros((1, 2, 32, 32, 32), dtype=torch.float64, device="cuda")
    Q = torch.zeros((1, 2, 2, 32, 32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_collide_noalloc(plan._h, 1, f, Q)
    assert e.value.status == 1
    assert "scratch" in str(e.value)


def test_noalloc_splits_points_over_passes():
    # N = 16, M = 6, N_rho = 8, S = 2, P = 8: the 32 MiB scratch holds five
    # evaluations per pass next to the forward transforms of all eight points,
    # so the points run in passes of 5 and 3 (the size loop's ragged last pass)
    pb = W.make_problem("c1_homog_n16", points=8)
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 8)
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float64)
    ref = plan.collide(f)
    torch.cuda.synchronize()
    for _ in range(2):
        Q = torch.full_like(ref, float("nan"))
        B.dgfs_collide_noalloc(plan._h, 8, f, Q)
        torch.cuda.synchronize()
        assert _rel(Q.cpu().numpy(), ref.cpu().numpy()) <= TOL64


def test_noalloc_rejects_points_beyond_its_scratch():
    # at N = 16, M = 6, N_rho = 8, S = 2 one evaluation per pass fits up to
    # P = 207 (16 B x 4096 x (2 P + 98) <= 32 MiB); P = 208 is refused
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    f = torch.zeros((208, 2, 16, 16, 16), dtype=torch.float64, device="cuda")
    Q = torch.zeros((208, 2, 2, 16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_collide_noalloc(plan._h, 208, f, Q)
    assert e.value.status == 1
    assert "scratch" in str(e.value)
