"""The allocation-free collision operator (lbe_apply_L_noalloc) against lbe_apply_L.

Callers that cannot allocate device memory (graph capture, latency-critical loops, host
frameworks that own every device byte) get the same operator with scratch taken from a
fixed 32 MiB device array.  Two calls in a row must both reproduce the allocating entry
point bit for bit, including cell counts that need several scratch slices with a ragged
last one."""
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


@pytest.mark.parametrize("nv,M,cells,prec", [(32, 32, 10, lbe.FP32), (16, 16, 70, lbe.FP64), (32, 32, 2, lbe.FP64)])
def test_noalloc_matches_allocating_entry_point(ctx, nv, M, cells, prec):
    dt = torch.float64 if prec == lbe.FP64 else torch.float32
    h = torch.tensor(workloads.random_h(cells, nv, 6.0, seed=cells), device="cuda", dtype=dt)
    d = torch.linspace(0.3, 30.0, cells, device="cuda", dtype=torch.float64)
    ref_p, ref_l = torch.empty_like(h), torch.empty_like(h)
    # the allocating call also builds the operator tables this context needs
    ctx.apply_L(nv, 6.0, M, 4.5, prec, cells, d.data_ptr(), h.data_ptr(), ref_p.data_ptr(), ref_l.data_ptr())
    torch.cuda.synchronize()
    for _ in range(2):
        out_p = torch.full_like(h, float("nan"))
        out_l = torch.full_like(h, float("nan"))
        ctx.apply_L_noalloc(nv, 6.0, M, 4.5, prec, cells, d.data_ptr(), h.data_ptr(), out_p.data_ptr(),
                            out_l.data_ptr())
        torch.cuda.synchronize()
        # the same kernels on the same per-cell data: the slicing of the cells changes nothing
        assert torch.isfinite(out_p).all() and torch.isfinite(out_l).all()
        assert torch.equal(out_p, ref_p) and torch.equal(out_l, ref_l)


def test_noalloc_rejects_oversize_and_unprepared(ctx):
    with pytest.raises(lbe.LbeError) as e:
        ctx.apply_L_noalloc(32, 6.0, 64, 4.5, lbe.FP64, 1, 1, 1, None, None)
    assert e.value.status == lbe.BAD_ARG and "maximum" in str(e.value)
    with pytest.raises(lbe.LbeError) as e:
        ctx.apply_L_noalloc(8, 5.5, 4, 4.0, lbe.FP32, 1, 1, 1, None, None)
    assert e.value.status == lbe.BAD_ARG and "not built" in str(e.value)
