"""Fourier-mode convergence analysis on the GPU (lbe_fourier_omega, Sec. 2.3): the power
iteration of the CIS and SIS error maps against the oracle's, from the same start vector, and
the paper's findings on the GPU driver (CIS omega -> 1 as delta grows, SIS omega near 0.6,
both small in the free-molecular regime)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import eig, fsm  # noqa: E402
from paper_1612_04488_gb300 import lbe, workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lbe.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def F():
    return fsm.FSM(16, 6.0, 16, 4.5)


@pytest.mark.parametrize("delta", [0.1, 10.0, 100.0])
@pytest.mark.parametrize("scheme", ["cis", "sis"])
def test_ratios_match_oracle(ctx, F, delta, scheme):
    e0 = workloads.fourier_start(16, 6.0, seed=3)
    step = (lambda e: eig.cis_map(F, e, delta)) if scheme == "cis" else (lambda e: eig.sis_map(F, e, delta))
    ref = eig.power_ratios(step, e0, 12)
    got = ctx.fourier_omega(16, 6.0, 16, 4.5, delta, 1.25, lbe.CIS if scheme == "cis" else lbe.SIS, 12, e0)
    assert np.allclose(got, ref, rtol=1e-10, atol=0), (got, ref)


def test_paper_findings_on_gpu(ctx):
    e0 = workloads.fourier_start(16, 6.0, seed=5)
    om = {}
    for d in (0.1, 10.0, 100.0):
        om[d] = tuple(ctx.fourier_omega(16, 6.0, 16, 4.5, d, 1.25, s, 40, e0)[-1] for s in (lbe.CIS, lbe.SIS))
    assert om[0.1][0] < 0.05 and om[0.1][1] < 0.05
    assert om[100.0][0] > 0.99
    assert om[10.0][1] < 0.6 * om[10.0][0]  # SIS well below CIS already at delta = 10
    assert 0.45 < om[100.0][1] < 0.7


def test_bad_arguments(ctx):
    e0 = workloads.fourier_start(8, 6.0, seed=1)
    with pytest.raises(lbe.LbeError):
        ctx.fourier_omega(8, 6.0, 8, 4.5, -1.0, 1.25, lbe.SIS, 3, e0)
    with pytest.raises(lbe.LbeError):
        ctx.fourier_omega(12, 6.0, 8, 4.5, 1.0, 1.25, lbe.SIS, 3, e0)


def test_full_grid_sis_near_continuum(ctx):
    """32^3, M = 32: the SIS factor near the continuum matches the oracle and sits at the
    paper's maximum of about 0.6 while the CIS stalls."""
    F32 = fsm.FSM(32, 6.0, 32, 4.5)
    e0 = workloads.fourier_start(32, 6.0, seed=5)
    ref = eig.power_ratios(lambda e: eig.sis_map(F32, e, 100.0), e0, 30)
    got = ctx.fourier_omega(32, 6.0, 32, 4.5, 100.0, 1.25, lbe.SIS, 30, e0)
    assert np.allclose(got, ref, rtol=1e-9, atol=0)
    assert 0.55 < got[-1] < 0.67
    cis = ctx.fourier_omega(32, 6.0, 32, 4.5, 100.0, 1.25, lbe.CIS, 30, e0)
    assert cis[-1] > 0.99
