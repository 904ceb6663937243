"""The bounded waits of the tensor-core kernel reach the caller as an error.

With the wait limit set to zero every wait that is not satisfied at once
runs out: the kernel stops (after its copies and products in flight), the
context's error word is latched and dmrg3s_sync returns DMRG3S_ERR_TIMEOUT.
No fault and no hang is involved: the waits end by their own limit.  The
context stays usable: with the default limit the same product then matches
the oracle.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import contract, io  # noqa: E402
from parity import TF32X3_TOL, problem, rel_err, site_to_dense  # noqa: E402


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.slib()
    return binding


def test_zero_wait_limit_latches_timeout_and_context_recovers(b):
    ctx = b.dmrg3s_create(0, 1 << 30)
    pb = problem("u1", 61, m_left=300, m_right=280)
    gL, gW, gR, gA = (b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]),
                      b.env_from_neutral(pb["R"]), b.site_from_neutral(pb["A"]))
    gH = b.empty_site_like(gA.qp, gA.left, gA.right)
    b.dmrg3s_set_wait_limit(ctx, 0.0)
    b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "tf32x3")
    with pytest.raises(b.Dmrg3sError) as e:
        b.dmrg3s_sync(ctx)
    assert e.value.status == 8                     # DMRG3S_ERR_TIMEOUT
    # the latch is cleared by the report, and the context still works
    b.dmrg3s_set_wait_limit(ctx, 1.0)
    b.dmrg3s_sync(ctx)
    b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "tf32x3")
    b.dmrg3s_sync(ctx)
    ref = contract.apply_heff(io.env_dense(pb["L"]), pb["W"]["W"], io.env_dense(pb["R"]),
                              io.site_dense(pb["A"])[0])
    assert rel_err(site_to_dense(b, gH), ref) < TF32X3_TOL
    ctx.close()


def test_negative_wait_limit_is_an_argument_error(b):
    ctx = b.dmrg3s_create(0, 1 << 26)
    with pytest.raises(b.Dmrg3sError) as e:
        b.dmrg3s_set_wait_limit(ctx, -1.0)
    assert e.value.status == 1
    ctx.close()
