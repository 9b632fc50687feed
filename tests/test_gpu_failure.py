"""Failure paths, made on the host or by bounded waits -- nothing here faults or hangs the GPU.

- An HBM budget too small for a problem gives LBE_OOM on solve and on submit; the context
  keeps working for problems that fit.
- A non-finite value that the device detects: a poisoned starting iterate (NaN in h) and a
  rarefaction so large that the iterates overflow both end in LBE_NAN.
- The tensor-core GEMM's bounded waits: a test hook makes each CTA wait on a barrier that
  nothing completes, with a short limit; the call returns LBE_TIMEOUT after the CTA has
  drained its own copies, and the next call without the hook is correct.
- Request cancellation in the service, queued and admitted.
- Checkpoint / resume: a solve stopped after k iterations and resumed from its iterate and
  flow rates continues bit for bit as the uninterrupted solve.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1612_04488_gb300 import lbe, workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    yield c
    c.close()


def small_plate(**kw):
    base = dict(dim=1, ns=20, grid_kind=0, nv=16, vmax=6.0, M=16, R=4.5, delta=1.0, scheme=lbe.SIS,
                precision=lbe.FP64, eps=1e-9, max_iter=300)
    base.update(kw)
    return lbe.problem(**base)


def test_budget_gives_oom_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0, hbm_budget=48 << 20)
    try:
        big = lbe.problem(**workloads.PLATES_32, delta=1.0, R=4.5, scheme=lbe.SIS, precision=lbe.FP64,
                          eps=1e-8, max_iter=50)
        with pytest.raises(lbe.LbeError) as e:
            c.solve(big)
        assert e.value.status == lbe.OOM
        t = c.submit(big)
        deadline = time.time() + 60
        while True:
            done, r = c.poll(t)
            if done:
                break
            assert time.time() < deadline
            time.sleep(0.01)
        assert r.status == lbe.OOM
        # a problem that fits still solves, and equals the same solve in an unconstrained context
        res, _, _ = c.solve(small_plate())
        assert res.status == lbe.OK
        ref_ctx = lbe.Context(0)
        try:
            ref, _, _ = ref_ctx.solve(small_plate())
        finally:
            ref_ctx.close()
        assert res.mass_flow == ref.mass_flow and res.heat_flow == ref.heat_flow
    finally:
        c.close()


@pytest.mark.parametrize("prec", [lbe.FP64, lbe.FP32])
def test_poisoned_start_gives_nan(ctx, prec):
    pb = small_plate(precision=prec, max_iter=10)
    n = lbe.cells_of(pb)
    h = np.zeros((n, 16, 16, 16))
    h[3, 5, 6, 7] = np.nan
    with pytest.raises(lbe.LbeError) as e:
        ctx.solve_from(pb, h)
    assert e.value.status == lbe.NAN
    res, _, _ = ctx.solve(small_plate(precision=prec, eps=1e-9 if prec == lbe.FP64 else 1e-5))
    assert res.status == lbe.OK


def test_overflowing_iterates_give_nan(ctx):
    with pytest.raises(lbe.LbeError) as e:
        ctx.solve(small_plate(delta=1e300, max_iter=20))
    assert e.value.status == lbe.NAN
    assert ctx.solve(small_plate())[0].status == lbe.OK


def test_gemm_wait_expiry_returns_timeout_and_recovers(ctx):
    nv, M, cells, parity = 16, 16, 64, 2
    h = workloads.random_h(cells, nv, 6.0, seed=9)
    h = np.ascontiguousarray(0.5 * (h + h[:, :, ::-1, :]))
    hd = torch.tensor(h, device="cuda", dtype=torch.float32)
    dd = torch.full((cells,), 2.0, device="cuda", dtype=torch.float64)
    ref = torch.empty_like(hd)
    ctx.apply_L_sym(nv, 6.0, M, 4.5, lbe.BF16_REFINED, parity, cells, dd.data_ptr(), hd.data_ptr(), ref.data_ptr(),
                    None)
    torch.cuda.synchronize()
    out = torch.full_like(hd, float("nan"))
    lbe.debug_expire_waits(True)
    try:
        with pytest.raises(lbe.LbeError) as e:
            ctx.apply_L_sym(nv, 6.0, M, 4.5, lbe.BF16_REFINED, parity, cells, dd.data_ptr(), hd.data_ptr(),
                            out.data_ptr(), None)
        assert e.value.status == lbe.TIMEOUT
        # a solve whose operator is that GEMM reports the expiry as its status
        with pytest.raises(lbe.LbeError) as e:
            ctx.solve(small_plate(precision=lbe.BF16, eps=1e-5))
        assert e.value.status == lbe.TIMEOUT
    finally:
        lbe.debug_expire_waits(False)
    ctx.apply_L_sym(nv, 6.0, M, 4.5, lbe.BF16_REFINED, parity, cells, dd.data_ptr(), hd.data_ptr(), out.data_ptr(),
                    None)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert ctx.solve(small_plate(precision=lbe.BF16, eps=1e-5))[0].status == lbe.OK


def wait_done(c, t, timeout=120):
    deadline = time.time() + timeout
    while True:
        done, r = c.poll(t)
        if done:
            return r
        assert time.time() < deadline, "request did not finish"
        time.sleep(0.005)


def test_cancel_queued_and_admitted():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    try:
        c.set_max_active(1)
        slow = small_plate(scheme=lbe.CIS, delta=30.0, eps=0.0, max_iter=100000)   # runs until cancelled
        quick = small_plate(delta=2.0)
        t_slow = c.submit(slow)
        t_queued = c.submit(quick)   # waits for the single slot
        t_after = c.submit(quick)
        c.cancel(t_queued)
        time.sleep(0.3)              # the slow request is admitted and iterating
        assert not c.poll(t_slow)[0]
        c.cancel(t_slow)
        assert wait_done(c, t_slow).status == lbe.CANCELLED
        assert wait_done(c, t_queued).status == lbe.CANCELLED
        r = wait_done(c, t_after)
        assert r.status == lbe.OK
        ref, _, _ = c.solve(quick)
        assert r.mass_flow == ref.mass_flow and r.heat_flow == ref.heat_flow
        c.cancel(t_after)            # finished: nothing changes
        assert c.poll(t_after)[1].status == lbe.OK
    finally:
        c.close()


@pytest.mark.parametrize("prec", [lbe.FP64, lbe.FP32, lbe.BF16])
def test_resume_is_bitwise(ctx, prec):
    """A solve stopped after k iterations and resumed from its h and flow rates ends exactly where
    the uninterrupted solve ends. BF16 keeps plate iterates in the orbit layout (one value per
    orbit of the v2 and v3 reflections), so its checkpoint round-trips through the full grid."""
    pb = small_plate(precision=prec, delta=10.0, eps=1e-9 if prec == lbe.FP64 else 1e-5)
    full, U_full, h_full = ctx.solve(pb, want_h=True)
    assert full.status == lbe.OK and full.iters > 8
    k = 7
    part_pb = small_plate(precision=prec, delta=10.0, eps=pb.eps, max_iter=k)
    part, _, h_part = ctx.solve(part_pb, want_h=True)
    assert part.iters == k
    res, U_res, h_res = ctx.solve_from(pb, h_part, prev=part, want_h=True)
    assert res.status == lbe.OK
    assert res.iters + k == full.iters
    assert res.mass_flow == full.mass_flow and res.heat_flow == full.heat_flow
    assert np.array_equal(h_res, h_full) and np.array_equal(U_res, U_full)
