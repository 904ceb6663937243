"""The H_eff entry point that allocates no device memory.

Callers that cannot call cudaMalloc (hosts whose device memory belongs to
another allocator, real-time callers that may not allocate mid-work) use
dmrg3s_apply_heff_noalloc, which keeps its intermediates in static device
arrays of the library instead of a context workspace.  This test calls it
through the C ABI and checks its output against dmrg3s_apply_heff, the
context-based entry point, and against the FP64 oracle, within the FP64
tolerance of the other parity tests, on two calls in a row (the static arrays
keep the first call's contents when the second one runs), and on two calls
with different structures queued back to back on one non-default stream.
The file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import contract, io  # noqa: E402
from parity import FP64_TOL, problem, rel_err, site_to_dense  # noqa: E402


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.lib()
    return binding


def _inputs(b, kind, seed, **kw):
    pb = problem(kind, seed, **kw)
    return (b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]), b.env_from_neutral(pb["R"]),
            b.site_from_neutral(pb["A"]))


def test_noalloc_matches_context_entry_point_twice(b):
    ctx = b.dmrg3s_create(0, 1 << 28)
    cases = [("xxz_l100_m512_u1", 1002, {}), ("u1", 21, {})]
    for kind, seed, kw in cases:      # two calls in a row, different structures
        gL, gW, gR, gA = _inputs(b, kind, seed, **kw)
        ref = b.empty_site_like(gA.qp, gA.left, gA.right)
        out = b.empty_site_like(gA.qp, gA.left, gA.right)
        out.data.fill_(float("nan"))
        b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, ref, "fp64")
        b.dmrg3s_apply_heff_noalloc(gL, gW, gR, gA, out)
        torch.cuda.synchronize()
        got, want = site_to_dense(b, out), site_to_dense(b, ref)
        assert np.all(np.isfinite(got))
        assert rel_err(got, want) < FP64_TOL
        pb = problem(kind, seed, **kw)
        oracle = contract.apply_heff(io.env_dense(pb["L"]), pb["W"]["W"], io.env_dense(pb["R"]),
                                     io.site_dense(pb["A"])[0])
        assert rel_err(got, oracle) < FP64_TOL
    # the same structure again: the arrays hold the previous call's data
    gL, gW, gR, gA = _inputs(b, "u1", 22)
    ref = b.empty_site_like(gA.qp, gA.left, gA.right)
    out = b.empty_site_like(gA.qp, gA.left, gA.right)
    b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, ref, "fp64")
    b.dmrg3s_apply_heff_noalloc(gL, gW, gR, gA, out)
    torch.cuda.synchronize()
    assert rel_err(site_to_dense(b, out), site_to_dense(b, ref)) < FP64_TOL
    ctx.close()


def test_noalloc_two_structures_on_one_stream(b):
    """Two calls with different block structures queued on one side stream
    with no synchronisation between them: stream order keeps them apart."""
    ctx = b.dmrg3s_create(0, 1 << 28)
    side = torch.cuda.Stream()
    probs = [problem("u1u1", 23), problem("u1", 24, m_left=37, m_right=29)]
    ins, outs, refs = [], [], []
    for pb in probs:
        gL, gW, gR, gA = (b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]),
                          b.env_from_neutral(pb["R"]), b.site_from_neutral(pb["A"]))
        ref = b.empty_site_like(gA.qp, gA.left, gA.right)
        b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, ref, "fp64")
        out = b.empty_site_like(gA.qp, gA.left, gA.right)
        out.data.fill_(float("nan"))
        ins.append((gL, gW, gR, gA))
        outs.append(out)
        refs.append(ref)
    torch.cuda.synchronize()
    for (gL, gW, gR, gA), out in zip(ins, outs):
        b.dmrg3s_apply_heff_noalloc(gL, gW, gR, gA, out, stream=side)
    side.synchronize()
    for pb, out, ref in zip(probs, outs, refs):
        got = site_to_dense(b, out)
        assert np.all(np.isfinite(got))
        assert rel_err(got, site_to_dense(b, ref)) < FP64_TOL
        want = contract.apply_heff(io.env_dense(pb["L"]), pb["W"]["W"], io.env_dense(pb["R"]),
                                   io.site_dense(pb["A"])[0])
        assert rel_err(got, want) < FP64_TOL
    ctx.close()


def test_noalloc_rejects_oversized_requests(b):
    gL, gW, gR, gA = _inputs(b, "cylinder_4x16_m2048_u1", 1004)
    out = b.empty_site_like(gA.qp, gA.left, gA.right)
    with pytest.raises(b.Dmrg3sError) as e:
        b.dmrg3s_apply_heff_noalloc(gL, gW, gR, gA, out)
    assert e.value.status == 11
