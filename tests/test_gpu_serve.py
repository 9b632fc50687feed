"""Continuous-batching service (lbe_submit / lbe_poll): results equal lbe_solve, bitwise the
same alone and in a mix, admission under a slot limit, refined requests reach the FP64
solution."""
import time

import pytest

torch = pytest.importorskip("torch")

from paper_1612_04488_gb300 import lbe  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    yield c
    c.close()


def wait_all(ctx, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout, "service timed out"
        for t in tickets:
            if t not in out:
                done, r = ctx.poll(t)
                if done:
                    out[t] = r
        time.sleep(0.002)
    return [out[t] for t in tickets]


def mix(prec, eps=1e-9):
    base = dict(nv=8, vmax=4.0, M=8, R=3.0, scheme=lbe.SIS, precision=prec, eps=eps, max_iter=300)
    pbs = [lbe.problem(dim=1, ns=ns, grid_kind=1, delta=d, forcing=f, **base)
           for ns, d, f in ((12, 0.1, 0), (30, 1.0, 1), (20, 10.0, 0), (50, 3.0, 1))]
    pbs += [lbe.problem(dim=2, nx=nx, ny=ny, width=nx / ny, delta=d, forcing=f, **base)
            for nx, ny, d, f in ((6, 5, 2.0, 0), (10, 5, 0.5, 1))]
    return pbs


def test_served_equals_solve_and_mix_equals_alone(ctx):
    pbs = mix(lbe.FP64)
    alone = wait_all(ctx, [ctx.submit(pbs[2])])[0]
    mixed = wait_all(ctx, [ctx.submit(p) for p in pbs])
    assert all(r.status == lbe.OK for r in mixed)
    assert mixed[2].mass_flow == alone.mass_flow and mixed[2].heat_flow == alone.heat_flow
    assert mixed[2].iters == alone.iters
    for p, r in zip(pbs, mixed):
        s, _, _ = ctx.solve(p)
        assert r.mass_flow == s.mass_flow and r.heat_flow == s.heat_flow and r.iters == s.iters


def test_admission_with_few_slots_and_arrivals_in_flight(ctx):
    ctx.set_max_active(2)
    try:
        pbs = mix(lbe.FP32, eps=1e-6)  # the relative-change test FP32 arithmetic can meet
        tickets = [ctx.submit(p) for p in pbs[:3]]
        time.sleep(0.01)
        tickets += [ctx.submit(p) for p in pbs[3:]]
        res = wait_all(ctx, tickets)
    finally:
        ctx.set_max_active(64)
    assert all(r.status == lbe.OK for r in res), [(r.status, r.iters, r.last_rel_change) for r in res]


@pytest.mark.parametrize("prec", [lbe.FP32_REFINED, lbe.BF16_REFINED])
def test_refined_requests_reach_fp64(ctx, prec):
    pbs = mix(lbe.FP64)
    ref = [ctx.solve(p)[0] for p in pbs]
    rp = mix(prec)
    got = wait_all(ctx, [ctx.submit(p) for p in rp])
    for r, g in zip(ref, got):
        assert g.status == lbe.OK, (g.status, g.iters, g.refinements, g.mass_flow, r.mass_flow)
        assert abs(g.mass_flow - r.mass_flow) <= 1e-7 * abs(r.mass_flow)
        assert abs(g.heat_flow - r.heat_flow) <= 1e-7 * abs(r.heat_flow)


def test_submit_rejects_bad_problem(ctx):
    with pytest.raises(lbe.LbeError):
        ctx.submit(lbe.problem(dim=1, ns=10, nv=12))


def test_serving_stream_at_workload_sizes(ctx):
    """Requests of the serving stream at their own sizes (velocity grids 24^3 and 32^3, M = 32,
    plates of 50-200 sections and ducts up to 80 x 40 cells, delta log-uniform on [0.01, 100]),
    BF16-refined, submitted while others are on the GPU: every result reaches the FP64 solution
    of its problem to 1e-7, and a request served in the mix agrees with the same request served
    alone to 1e-7 (the tensor-core GEMM's K split depends on the bucket's cells, so the last bits
    may differ)."""
    from paper_1612_04488_gb300 import workloads
    reqs = workloads.serving_requests(n=256, seed=20261203)
    # two of each kind: plates and ducts at 24^3 and 32^3
    pick, seen = [], {}
    for r in reqs:
        k = (r["dim"], r["nv"])
        if seen.get(k, 0) < 2 and (r["dim"] == 1 or r["nx"] * r["ny"] <= 1600):
            seen[k] = seen.get(k, 0) + 1
            pick.append(r)
    assert len(pick) == 8

    def pb(r, prec, eps):
        geo = {k: r[k] for k in ("dim", "ns", "grid_kind", "nx", "ny", "width") if k in r}
        return lbe.problem(**geo, delta=r["delta"], nv=r["nv"], vmax=r["vmax"], M=r["M"], R=4.5, forcing=r["forcing"],
                           scheme=lbe.SIS, precision=prec, eps=eps, max_iter=400)

    ctx.set_max_active(64)
    tickets = []
    for i, r in enumerate(pick):  # arrivals spread while earlier requests run
        tickets.append(ctx.submit(pb(r, lbe.BF16_REFINED, 1e-9)))
        time.sleep(0.02)
    got = wait_all(ctx, tickets, timeout=600.0)
    alone = wait_all(ctx, [ctx.submit(pb(pick[0], lbe.BF16_REFINED, 1e-9))], timeout=600.0)[0]
    for r, g in zip(pick, got):
        ref, _, _ = ctx.solve(pb(r, lbe.FP64, 1e-9))
        info = (r, g.status, g.refinements, g.mass_flow, ref.mass_flow, g.heat_flow, ref.heat_flow)
        assert g.status == lbe.OK and ref.status == lbe.OK, info
        assert abs(g.mass_flow - ref.mass_flow) <= 1e-7 * abs(ref.mass_flow), info
        assert abs(g.heat_flow - ref.heat_flow) <= 1e-7 * abs(ref.heat_flow), info
    assert abs(alone.mass_flow - got[0].mass_flow) <= 1e-7 * abs(got[0].mass_flow)
    assert abs(alone.heat_flow - got[0].heat_flow) <= 1e-7 * abs(got[0].heat_flow)
