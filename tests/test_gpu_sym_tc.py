"""Parity-subspace collision operator (lbe_apply_L_sym): the symmetry-reduced fast-spectral
form in FP64 / FP32 and the dense tcgen05 GEMM form, against the FP64 oracle on seeded h with
the plate (odd v3, even v2) and duct (odd v3) parities; and the BF16-refined solve against
the FP64 solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fsm  # noqa: E402
from paper_1612_04488_gb300 import lbe, workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    yield c
    c.close()


def parity_h(cells, nv, parity, seed):
    h = workloads.random_h(cells, nv, 6.0, seed=seed)          # odd in v3 by construction
    if parity == 2:
        h = 0.5 * (h + h[:, :, ::-1, :])                         # even in v2
    return np.ascontiguousarray(h)


@pytest.mark.parametrize("nv,M,parity,cells,prec,tol", [
    (16, 16, 2, 21, lbe.FP64, 1e-12), (16, 16, 1, 9, lbe.FP64, 1e-12), (32, 32, 2, 3, lbe.FP64, 1e-12),
    (24, 16, 2, 4, lbe.FP64, 1e-12), (32, 32, 1, 3, lbe.FP32, 3e-6), (16, 16, 2, 300, lbe.BF16_REFINED, 1e-4),
    (32, 32, 2, 40, lbe.BF16_REFINED, 1e-4), (16, 16, 1, 70, lbe.BF16_REFINED, 1e-4),
    (8, 8, 2, 33, lbe.BF16_REFINED, 1e-4), (8, 8, 1, 20, lbe.BF16_REFINED, 1e-4),
    (24, 16, 2, 30, lbe.BF16_REFINED, 1e-4), (24, 16, 1, 17, lbe.BF16_REFINED, 1e-4),
    (16, 16, 2, 21, lbe.DF32, 1e-12), (16, 16, 1, 9, lbe.DF32, 1e-12), (32, 32, 2, 3, lbe.DF32, 1e-12),
    (24, 16, 2, 4, lbe.DF32, 1e-12)])
def test_apply_L_sym_matches_oracle(ctx, nv, M, parity, cells, prec, tol):
    h = parity_h(cells, nv, parity, seed=cells + nv)
    deltas = np.linspace(0.3, 30.0, cells)
    dt = torch.float64 if prec in (lbe.FP64, lbe.DF32) else torch.float32
    hd = torch.tensor(h, device="cuda", dtype=dt)
    dd = torch.tensor(deltas, device="cuda")
    lp = torch.full_like(hd, float("nan"))
    L = torch.full_like(hd, float("nan"))
    ctx.apply_L_sym(nv, 6.0, M, 4.5, prec, parity, cells, dd.data_ptr(), hd.data_ptr(), lp.data_ptr(), L.data_ptr())
    torch.cuda.synchronize()
    lp, L = lp.double().cpu().numpy(), L.double().cpu().numpy()
    F = fsm.FSM(nv, 6.0, M, 4.5)
    hh = hd.double().cpu().numpy()
    for c in sorted({0, cells // 2, cells - 1}):
        olp, oL = F.apply(hh[c], deltas[c])
        assert np.max(np.abs(lp[c] - olp)) <= tol * np.max(np.abs(olp)), c
        assert np.max(np.abs(L[c] - oL)) <= tol * np.max(np.abs(oL)), c


@pytest.mark.parametrize("nv,M,cells", [(16, 16, 7), (8, 8, 33), (32, 16, 2)])
def test_apply_L_df32_matches_oracle(ctx, nv, M, cells):
    """The full operator (all M directions, no parity assumed) in double-float arithmetic,
    with the L-moments, against the FP64 oracle."""
    rng = np.random.default_rng(nv + cells)
    h = workloads.random_h(cells, nv, 6.0, seed=nv * cells)
    h = h + 0.1 * rng.standard_normal(h.shape) * np.abs(h).max()   # no parity at all
    deltas = np.linspace(0.5, 50.0, cells)
    nd = 1.25 * deltas
    hd = torch.tensor(h, device="cuda", dtype=torch.float64)
    dd = torch.tensor(deltas, device="cuda")
    ndd = torch.tensor(nd, device="cuda")
    lp = torch.full_like(hd, float("nan"))
    L = torch.full_like(hd, float("nan"))
    G = torch.zeros((cells, 2), device="cuda", dtype=torch.float64)
    ctx.apply_L(nv, 6.0, M, 4.5, lbe.DF32, cells, dd.data_ptr(), hd.data_ptr(), lp.data_ptr(), L.data_ptr(),
                ndd.data_ptr(), G.data_ptr())
    torch.cuda.synchronize()
    lp, L, G = lp.cpu().numpy(), L.cpu().numpy(), G.cpu().numpy()
    F = fsm.FSM(nv, 6.0, M, 4.5)
    V1, V2, V3 = F.V1, F.V2, F.V3
    for c in sorted({0, cells // 2, cells - 1}):
        olp, oL = F.apply(h[c], deltas[c])
        assert np.max(np.abs(lp[c] - olp)) <= 1e-12 * np.max(np.abs(olp)), c
        assert np.max(np.abs(L[c] - oL)) <= 1e-12 * np.max(np.abs(oL)), c
        w = 2.0 * (oL + nd[c] * h[c]) * V3 * F.dv ** 3
        for j, Vj in ((0, V1), (1, V2)):
            ref = np.sum(Vj * w)
            assert abs(G[c, j] - ref) <= 1e-11 * np.sum(np.abs(Vj * w)), (c, j)


def oracle_G(F, Lh, h, nd):
    w = 2.0 * (Lh + nd * h) * F.V3 * F.dv ** 3
    return np.array([np.sum(F.V1 * w), np.sum(F.V2 * w)]), np.sum(np.abs(w) * (np.abs(F.V1) + np.abs(F.V2)))


@pytest.mark.parametrize("case", ["plates808", "duct2048"])
def test_tensor_operator_at_production_size(ctx, case):
    """The tcgen05 operator at the sizes the solves run it: 808 plate cells (column tiles of
    208, the first 152 tiles whole and the rest split four ways in K with the fix-up, the last
    column tile holding cells 624-807 plus padding) and 2048 duct cells (whole waves of
    256-column tiles, then split tiles).  Every output cell takes rows from whole and from
    split tiles.  Sampled cells against the oracle, with the fused L-moments."""
    nv, M = 32, 32
    if case == "plates808":
        cells, parity = 808, 2
        deltas = np.repeat(np.array([0.1, 1.0, 10.0, 100.0] * 2), 101)
        sample = (0, 207, 208, 500, 623, 624, 800, 807)
    else:
        cells, parity = 2048, 1
        deltas = np.full(cells, 10.0) * np.linspace(0.5, 2.0, cells)
        sample = (0, 255, 1024, 1791, 2047)
    base = parity_h(16, nv, parity, seed=cells)
    h = np.ascontiguousarray(np.resize(base, (cells, nv, nv, nv)))
    nd = 1.25 * deltas
    hd = torch.tensor(h, device="cuda", dtype=torch.float32)
    dd = torch.tensor(deltas, device="cuda")
    ndd = torch.tensor(nd, device="cuda")
    lp = torch.full_like(hd, float("nan"))
    L = torch.full_like(hd, float("nan"))
    G = torch.full((cells, 2), float("nan"), device="cuda", dtype=torch.float64)
    ctx.apply_L_sym(nv, 6.0, M, 4.5, lbe.BF16_REFINED, parity, cells, dd.data_ptr(), hd.data_ptr(), lp.data_ptr(),
                    L.data_ptr(), ndd.data_ptr(), G.data_ptr())
    torch.cuda.synchronize()
    assert torch.isfinite(lp).all() and torch.isfinite(L).all() and torch.isfinite(G).all()
    F = fsm.FSM(nv, 6.0, M, 4.5)
    G = G.cpu().numpy()
    for c in sample:
        hc = hd[c].double().cpu().numpy()
        olp, oL = F.apply(hc, deltas[c])
        got_lp, got_L = lp[c].double().cpu().numpy(), L[c].double().cpu().numpy()
        assert np.max(np.abs(got_lp - olp)) <= 1e-4 * np.max(np.abs(olp)), c
        assert np.max(np.abs(got_L - oL)) <= 1e-4 * np.max(np.abs(oL)), c
        oG, scale = oracle_G(F, oL, hc, nd[c])
        assert np.all(np.abs(G[c] - oG) <= 1e-4 * scale), (c, G[c], oG)


@pytest.mark.parametrize("prec,tol", [(lbe.FP64, 1e-11), (lbe.DF32, 1e-11), (lbe.FP32, 2e-5)])
def test_apply_L_sym_moments(ctx, prec, tol):
    """The L-moments of lbe_apply_L_sym in the fast-spectral forms against the oracle."""
    nv, M, cells, parity = 16, 16, 9, 2
    h = parity_h(cells, nv, parity, seed=5)
    deltas = np.linspace(0.5, 20.0, cells)
    nd = 1.25 * deltas
    dt = torch.float32 if prec == lbe.FP32 else torch.float64
    hd = torch.tensor(h, device="cuda", dtype=dt)
    dd, ndd = torch.tensor(deltas, device="cuda"), torch.tensor(nd, device="cuda")
    G = torch.full((cells, 2), float("nan"), device="cuda", dtype=torch.float64)
    ctx.apply_L_sym(nv, 6.0, M, 4.5, prec, parity, cells, dd.data_ptr(), hd.data_ptr(), None, None,
                    ndd.data_ptr(), G.data_ptr())
    torch.cuda.synchronize()
    F = fsm.FSM(nv, 6.0, M, 4.5)
    hh = hd.double().cpu().numpy()
    G = G.cpu().numpy()
    for c in range(cells):
        _, oL = F.apply(hh[c], deltas[c])
        oG, scale = oracle_G(F, oL, hh[c], nd[c])
        assert np.all(np.abs(G[c] - oG) <= tol * scale), (c, G[c], oG)


def test_bf16_unrefined_within_1e4_of_fp64(ctx):
    """The low-precision phase alone (LBE_BF16: tensor-core operator, FP32 sweeps, no
    refinement) on the batched plates workload (808 cells of 32^3, M = 32) gives flow rates
    within 1e-4 of the FP64 solution of the same discrete problem, relative to the larger flow
    rate of each problem (a tiny flow rate, e.g. the heat flow at delta = 100, is resolved only
    to FP32 rounding of that scale)."""
    kw = dict(workloads.PLATES_32, R=4.5, scheme=lbe.SIS, max_iter=400)
    cases = [(d, f) for d in workloads.PLATES_32_DELTAS for f in (0, 1)]
    ref = ctx.solve_batch([lbe.problem(**kw, delta=d, forcing=f, precision=lbe.FP64, eps=1e-10) for d, f in cases])
    got = ctx.solve_batch([lbe.problem(**kw, delta=d, forcing=f, precision=lbe.BF16, eps=1e-6) for d, f in cases])
    for (d, f), r, g in zip(cases, ref, got):
        assert g.status == lbe.OK, (d, f, g.status, g.iters)
        scale = max(abs(r.mass_flow), abs(r.heat_flow))
        assert abs(g.mass_flow - r.mass_flow) <= 1e-4 * scale, (d, f, g.mass_flow, r.mass_flow)
        assert abs(g.heat_flow - r.heat_flow) <= 1e-4 * scale, (d, f, g.heat_flow, r.heat_flow)


def test_bf16_refined_solve_reaches_fp64(ctx):
    base = dict(dim=1, ns=40, grid_kind=1, nv=16, vmax=6.0, M=16, R=4.5, scheme=lbe.SIS, eps=1e-9, max_iter=300)
    pbs = [lbe.problem(**base, delta=d, forcing=f, precision=lbe.FP64) for d in (1.0, 30.0) for f in (0, 1)]
    ref = ctx.solve_batch(pbs)
    got = ctx.solve_batch([lbe.problem(**base, delta=d, forcing=f, precision=lbe.BF16_REFINED)
                           for d in (1.0, 30.0) for f in (0, 1)])
    for r, g in zip(ref, got):
        assert g.status == lbe.OK, (g.status, g.iters, g.refinements)
        assert abs(g.mass_flow - r.mass_flow) <= 1e-7 * abs(r.mass_flow)
        assert abs(g.heat_flow - r.heat_flow) <= 1e-7 * abs(r.heat_flow)


@pytest.mark.parametrize("prec,eps,tol", [(lbe.BF16, 1e-6, 1e-4), (lbe.BF16_REFINED, 1e-9, 1e-6)])
def test_bf16_plate_iterate_symmetric_and_near_fp64(ctx, prec, eps, tol):
    """The plate iterates of the tensor-core paths (the FP32 one, and the FP64 one of the
    refinement) live in the orbit layout; returned on the full grid they are exactly even in v2
    and odd in v3, and near the FP64 iterate (1e-4 of its scale unrefined, 1e-6 refined)."""
    base = dict(dim=1, ns=30, grid_kind=1, nv=16, vmax=6.0, M=16, R=4.5, delta=3.0, scheme=lbe.SIS,
                max_iter=300)
    r64, _, h64 = ctx.solve(lbe.problem(**base, precision=lbe.FP64, eps=1e-10), want_h=True)
    rb, _, hb = ctx.solve(lbe.problem(**base, precision=prec, eps=eps), want_h=True)
    assert rb.status == lbe.OK and r64.status == lbe.OK
    assert np.array_equal(hb[:, :, ::-1, :], hb)
    assert np.array_equal(hb[:, :, :, ::-1], -hb)
    scale = np.abs(h64).max()
    assert np.abs(hb - h64).max() <= tol * scale


@pytest.mark.parametrize("prec,eps,tol", [(lbe.BF16, 1e-6, 1e-4), (lbe.BF16_REFINED, 1e-9, 1e-6)])
def test_bf16_duct_iterate_odd_and_near_fp64(ctx, prec, eps, tol):
    """Duct iterates of the tensor-core paths keep one value per orbit of the v3 reflection (half
    of each cell); returned on the full grid they are exactly odd in v3 and near the FP64 iterate."""
    base = dict(dim=2, nx=10, ny=6, width=1.6, delta=2.0, nv=16, vmax=6.0, M=16, R=4.5, scheme=lbe.SIS,
                max_iter=300)
    r64, _, h64 = ctx.solve(lbe.problem(**base, precision=lbe.FP64, eps=1e-10), want_h=True)
    rb, _, hb = ctx.solve(lbe.problem(**base, precision=prec, eps=eps), want_h=True)
    assert rb.status == lbe.OK and r64.status == lbe.OK
    assert np.array_equal(hb[:, :, :, ::-1], -hb)
    scale = np.abs(h64).max()
    assert np.abs(hb - h64).max() <= tol * scale
