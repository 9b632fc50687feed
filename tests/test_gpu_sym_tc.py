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
    (24, 16, 2, 4, lbe.FP64, 1e-12), (32, 32, 1, 3, lbe.FP32, 3e-6), (16, 16, 2, 300, lbe.BF16_REFINED, 2e-4),
    (32, 32, 2, 40, lbe.BF16_REFINED, 2e-4), (16, 16, 1, 70, lbe.BF16_REFINED, 2e-4),
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
