"""The rectangular-duct workload at its full size: 64 x 32 cells of aspect ratio 2, 32^3
velocities, M = 32, delta = 10 (Sec. 2.4, Table 2 geometry).

- The 2D transport sweep (FP64 and FP32) over all 2048 cells against the oracle's sweep.
- The SIS diffusion solve on the 62 x 30 interior (DST-I on the GPU, dense LU in the oracle).
- A 32^3 duct solve (small cross-section) for fixed iterations against the oracle.
- The mixed-precision solves of the 64 x 32 duct against the FP64 GPU solve: BF16-refined to
  1e-7, the unrefined BF16 phase to 1e-4 of the flow-rate scale.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fsm, solver, transport, velocity  # noqa: E402
from paper_1612_04488_gb300 import lbe, workloads  # noqa: E402

pytestmark = pytest.mark.gpu

R45 = 4.5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def F32():
    return fsm.FSM(32, 6.0, 32, R45)


@pytest.mark.parametrize("prec,tol", [(lbe.FP64, 1e-12), (lbe.FP32, 3e-6)])
def test_sweep_duct64x32_matches_oracle(ctx, F32, prec, tol):
    kw = dict(workloads.DUCT_64x32)
    nx, ny, nv, width, delta = kw["nx"], kw["ny"], kw["nv"], kw["width"], kw["delta"]
    pb = lbe.problem(**kw, R=R45, precision=prec, forcing=lbe.POISEUILLE)
    n = nx * ny
    base = workloads.random_h(32, nv, 6.0, seed=64)
    lplus = np.resize(base, (n, nv, nv, nv)) * np.linspace(0.5, 1.5, n)[:, None, None, None]
    dt = torch.float64 if prec == lbe.FP64 else torch.float32
    r = torch.tensor(lplus, device="cuda", dtype=dt)
    h = torch.empty_like(r)
    mom = torch.empty((n, 5), dtype=torch.float64, device="cuda")
    ctx.sweep(pb, r.data_ptr(), h.data_ptr(), mom.data_ptr())
    torch.cuda.synchronize()
    rin = r.double().cpu().numpy()
    S = velocity.source(F32.V1, F32.V2, F32.V3, 0)
    rq = (rin + S).reshape((nx, ny) + (nv,) * 3)
    oh = transport.sweep_2d(rq, delta * F32.nu, F32.V1, F32.V2, nx, ny, width).reshape(n, nv, nv, nv)
    gh = h.double().cpu().numpy()
    assert np.max(np.abs(gh - oh)) <= tol * np.max(np.abs(oh))
    om = np.stack(solver.cell_moments(F32, oh), -1)
    assert np.max(np.abs(mom.cpu().numpy() - om)) <= 10 * tol * np.max(np.abs(om))


def test_diffusion_duct64x32_matches_oracle(ctx):
    rng = np.random.default_rng(6432)
    nx, ny, width = 64, 32, 2.0
    pb = lbe.problem(dim=2, nx=nx, ny=ny, width=width, delta=10.0, nv=8, vmax=4.0, M=8, R=3.0,
                     forcing=lbe.POISEUILLE)
    Uh, W1, W2, X12, G1, G2 = rng.standard_normal((6, nx, ny))
    got = ctx.diffusion(pb, *[a.reshape(-1) for a in (Uh, W1, W2, X12, G1, G2)])
    ref = solver.poisson_2d(Uh, W1, W2, X12, G1, G2, width, 1.25 * 10.0, 1.0)
    assert np.max(np.abs(got - ref.reshape(-1))) <= 1e-11 * np.max(np.abs(ref))


def test_duct_nv32_fixed_iterations_match_oracle(ctx, F32):
    kw = dict(dim=2, nx=10, ny=8, width=1.25, delta=10.0, nv=32, vmax=6.0, M=32, R=R45, forcing=0)
    opb = solver.Problem(dim=2, nx=10, ny=8, width=1.25, delta=10.0, nv=32, vmax=6.0, M=32, R=R45,
                         forcing=0, scheme="sis", eps=0.0, max_iter=3)
    run = solver.Run(opb, F=F32)
    for _ in range(3):
        run.M, run.Q = run.step()
    pb = lbe.problem(**kw, scheme=lbe.SIS, precision=lbe.FP64, eps=0.0, max_iter=3)
    res, U, h = ctx.solve(pb, want_h=True)
    assert abs(res.mass_flow - run.M) <= 1e-10 * abs(run.M)
    assert abs(res.heat_flow - run.Q) <= 1e-10 * abs(run.Q)
    assert np.max(np.abs(h - run.h.reshape(h.shape))) <= 1e-10 * np.max(np.abs(run.h))


def test_duct64x32_mixed_precision_against_fp64(ctx):
    kw = dict(workloads.DUCT_64x32, R=R45, scheme=lbe.SIS, max_iter=400)
    ref, _, _ = ctx.solve(lbe.problem(**kw, precision=lbe.FP64, eps=1e-9))
    assert ref.status == lbe.OK
    ref_t, _, _ = ctx.solve(lbe.problem(**kw, precision=lbe.FP64, eps=1e-9, forcing=lbe.THERMAL_TRANSPIRATION))
    got = ctx.solve_batch([lbe.problem(**kw, precision=lbe.BF16_REFINED, eps=1e-9),
                           lbe.problem(**kw, precision=lbe.BF16_REFINED, eps=1e-9,
                                       forcing=lbe.THERMAL_TRANSPIRATION)])
    for g, r in zip(got, (ref, ref_t)):
        assert g.status == lbe.OK and g.refinements >= 1, (g.status, g.refinements)
        assert abs(g.mass_flow - r.mass_flow) <= 1e-7 * abs(r.mass_flow), (g.mass_flow, r.mass_flow)
        assert abs(g.heat_flow - r.heat_flow) <= 1e-7 * abs(r.heat_flow), (g.heat_flow, r.heat_flow)
    lo, _, _ = ctx.solve(lbe.problem(**kw, precision=lbe.BF16, eps=1e-6))
    scale = max(abs(ref.mass_flow), abs(ref.heat_flow))
    assert lo.status == lbe.OK
    assert abs(lo.mass_flow - ref.mass_flow) <= 1e-4 * scale and abs(lo.heat_flow - ref.heat_flow) <= 1e-4 * scale
