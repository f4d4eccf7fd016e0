"""Allocation failure, injected on the host (dgfs_debug_fail_alloc): every
creation call of the C ABI returns DGFS_ENOMEM with a NULL handle and releases
what it had allocated, whichever of its allocations fails; the context stays
usable and the next creation works.  No GPU fault is involved: the failing
allocation is refused on the host before the allocation routine would run."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ENOMEM = 2
SENTINEL = 0x5EED


@pytest.fixture(autouse=True)
def _hook_off():
    B.dgfs_debug_fail_alloc(0)
    yield
    B.dgfs_debug_fail_alloc(0)


def _plan_raw(N, L, M, Nrho, masses, pairs, prec, max_points):
    """dgfs_plan_create through ctypes, returning (status, handle) so that the
    handle written on failure can be checked."""
    S = len(masses)
    m = (ctypes.c_double * S)(*masses)
    pr = (B.dgfs_pair * (S * S))()
    for k, p in enumerate(pairs):
        pr[k].omega, pr[k].alpha, pr[k].d = p["omega"], p["alpha"], p["d"]
        pr[k].beta_override = math.nan
    h = ctypes.c_void_p(SENTINEL)
    st = B.lib().dgfs_plan_create(ctypes.byref(h), N, L, M, Nrho, S, ctypes.cast(m, ctypes.c_void_p),
                                  ctypes.cast(pr, ctypes.c_void_p), B.PRECISIONS[prec], max_points, 0)
    return st, h.value


def _sweep(create, destroy):
    """Fail the 1st, 2nd, ... allocation of `create` until it succeeds; returns
    how many allocations it makes."""
    base = B.dgfs_debug_live_allocations()
    n = 1
    while True:
        B.dgfs_debug_fail_alloc(n)
        st, h = create()
        if st == 0:
            B.dgfs_debug_fail_alloc(0)
            destroy(h)
            torch.cuda.synchronize()
            assert B.dgfs_debug_live_allocations() == base
            return n - 1
        assert st == ENOMEM, (n, st, B.dgfs_last_error())
        assert h is None, n  # *out set to NULL
        assert B.dgfs_debug_live_allocations() == base, (n, B.dgfs_debug_live_allocations(), base)
        n += 1
        assert n < 400


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc", "bf16x3"])
def test_plan_create_unwinds_at_every_allocation(prec):
    N, L, M, Nrho = 8, 2.5, 6, 3
    masses = [1.0, 2.0]
    pairs = W.pair_params([0.81, 0.75], [1.0, 1.4], [1.0, 1.2])
    count = _sweep(lambda: _plan_raw(N, L, M, Nrho, masses, pairs, prec, 2),
                   lambda h: B.dgfs_plan_destroy(ctypes.c_void_p(h)))
    # host object, twiddles, overflow flag, quadrature, six tables per pair,
    # masses, workspace, staging (and the tensor-core images and state)
    assert count >= 5 + 6 * 4 + 3
    # the context is usable and a plan built afterwards evaluates normally
    plan = B.Plan(N, L, M, Nrho, masses, pairs, prec, 1)
    rng = np.random.default_rng(7)
    f = np.stack([W.two_maxwellians(rng, N, L, m) for m in masses])[None]
    Q = plan.collide(torch.from_numpy(f).to("cuda", plan.dtype))
    plan.check()
    assert torch.isfinite(Q).all()


def test_dg_batch_and_graph_creation_unwind():
    N, L, M, Nrho = 8, 2.5, 6, 3
    masses = [1.0, 2.0]
    pairs = W.pair_params([0.81, 0.75], [1.0, 1.4], [1.0, 1.2])
    plan = B.Plan(N, L, M, Nrho, masses, pairs, "fp32_tc", 6)
    walls = np.array([1.0, 0.0, 0.0, 0.0, 2.0, 0.0, 0.0, 0.0])

    def dg_create():
        h = ctypes.c_void_p(SENTINEL)
        st = B.lib().dgfs_dg_create(ctypes.byref(h), plan._h, 2, 3, 0.0, 1.0, walls.ctypes.data_as(ctypes.c_void_p))
        return st, h.value

    count = _sweep(dg_create, lambda h: B.dgfs_dg_destroy(ctypes.c_void_p(h)))
    assert count >= 6  # host object, wall tables, flux partials, two stage buffers, Q

    f = torch.zeros((6, 2, N, N, N), dtype=torch.float32, device="cuda")
    Q = torch.zeros((6, 2, 2, N, N, N), dtype=torch.float32, device="cuda")
    ph = (ctypes.c_void_p * 1)(plan._h.value)
    pp = (ctypes.c_int * 1)(6)
    fp = (ctypes.c_void_p * 1)(f.data_ptr())
    qp = (ctypes.c_void_p * 1)(Q.data_ptr())

    def batch_create():
        h = ctypes.c_void_p(SENTINEL)
        st = B.lib().dgfs_batch_create(1, ctypes.cast(ph, ctypes.c_void_p), ctypes.cast(pp, ctypes.c_void_p),
                                       ctypes.cast(fp, ctypes.c_void_p), ctypes.cast(qp, ctypes.c_void_p), 0.0,
                                       ctypes.byref(h))
        return st, h.value

    assert _sweep(batch_create, lambda h: B.dgfs_batch_destroy(ctypes.c_void_p(h))) == 2  # batch + its TC part

    def graph_create():
        h = ctypes.c_void_p(SENTINEL)
        st = B.lib().dgfs_graph_capture(1, ctypes.cast(ph, ctypes.c_void_p), ctypes.cast(pp, ctypes.c_void_p),
                                        ctypes.cast(fp, ctypes.c_void_p), ctypes.cast(qp, ctypes.c_void_p), 0.0, 1,
                                        ctypes.byref(h))
        return st, h.value

    assert _sweep(graph_create, lambda h: B.dgfs_graph_destroy(ctypes.c_void_p(h))) == 1
    plan.collide(f, Q)
    plan.check()


def test_tc_backward_allocation_failure():
    """The tensor-core backward allocates its k-space tables once per plan and its
    FP64 scratch per call: a failure of either returns DGFS_ENOMEM, leaves no
    scratch behind, and the next call gives the same result as an unhindered plan."""
    N, L, M, Nrho = 8, 2.5, 6, 3
    masses = [1.0, 2.0]
    pairs = W.pair_params([0.81, 0.75], [1.0, 1.4], [1.0, 1.2])
    rng = np.random.default_rng(9)
    f = torch.from_numpy(np.stack([W.two_maxwellians(rng, N, L, m) for m in masses])[None]).to("cuda", torch.float32)
    g = torch.from_numpy(rng.normal(size=(1, 2, 2, N, N, N))).to("cuda", torch.float32)
    ref = B.Plan(N, L, M, Nrho, masses, pairs, "fp32_tc", 1)
    df0, dw0 = ref.backward(f, g)
    plan = B.Plan(N, L, M, Nrho, masses, pairs, "fp32_tc", 1)
    torch.cuda.synchronize()
    base = B.dgfs_debug_live_allocations()
    df = torch.empty_like(f)
    dom = torch.zeros(4, dtype=torch.float64, device="cuda")
    # 1st allocation: the plan's conj(phi) tables
    B.dgfs_debug_fail_alloc(1)
    st = B.lib().dgfs_collide_backward(plan._h, 1, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(df.data_ptr()), ctypes.c_void_p(dom.data_ptr()), 0, None)
    B.dgfs_debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert st == ENOMEM, B.dgfs_last_error()
    assert B.dgfs_debug_live_allocations() == base
    # 2nd allocation: the per-call scratch (the tables of the 1st stay with the plan)
    B.dgfs_debug_fail_alloc(2)
    st = B.lib().dgfs_collide_backward(plan._h, 1, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(df.data_ptr()), ctypes.c_void_p(dom.data_ptr()), 0, None)
    B.dgfs_debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert st == ENOMEM, B.dgfs_last_error()
    assert B.dgfs_debug_live_allocations() == base + 1
    df1, dw1 = plan.backward(f, g)
    plan.check()
    torch.cuda.synchronize()
    assert B.dgfs_debug_live_allocations() == base + 1
    assert torch.equal(df1, df0) and torch.equal(dw1, dw0)
