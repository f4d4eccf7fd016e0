"""Fault handling without faulting the GPU: a bounded device wait that nothing
completes reports DGFS_ETIMEOUT through dgfs_plan_check and leaves the context
usable; argument errors are status codes, not crashes."""
import numpy as np
import pytest
import torch

from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc_plan():
    pb = W.make_problem("c1_homog_n16")
    return pb, B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp32_tc", 1)


def test_expired_wait_reports_timeout_and_context_survives(tc_plan):
    pb, plan = tc_plan
    f = torch.from_numpy(pb["f"]).to("cuda", torch.float32)
    Q0 = plan.collide(f).clone()
    plan.check()
    B.dgfs_plan_selftest_wait(plan._h, expire=True)
    with pytest.raises(B.DgfsError) as e:
        plan.check()
    assert e.value.status == 4  # DGFS_ETIMEOUT
    plan.check()  # flag cleared
    Q1 = plan.collide(f)
    plan.check()
    assert torch.equal(Q0, Q1)


def test_completed_wait_reports_nothing(tc_plan):
    _, plan = tc_plan
    B.dgfs_plan_selftest_wait(plan._h, expire=False)
    plan.check()


def test_fp64_plans_have_no_device_waits():
    pb = W.make_problem("c1_homog_n16")
    plan = B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], "fp64", 1)
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_plan_selftest_wait(plan._h, expire=True)
    assert e.value.status == 5


def test_bad_arguments_are_status_codes(tc_plan):
    pb, plan = tc_plan
    f = torch.zeros((2, 2, 16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        plan.collide(f)  # P = 2 > max_points = 1
    assert e.value.status == 1
    with pytest.raises(ValueError):
        plan.collide(f[:1].double().contiguous())  # wrong dtype is rejected by the binding


def test_misaligned_f_is_rejected_by_tensor_core_plans(tc_plan):
    pb, plan = tc_plan
    buf = torch.zeros(16 ** 3 * 2 + 1, dtype=torch.float32, device="cuda")
    f = buf[1:].view(1, 2, 16, 16, 16)  # 4-byte offset from an aligned allocation
    Q = torch.empty((1, 2, 2, 16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_collide(plan._h, 1, f, Q)
    assert e.value.status == 1
