"""GPU parity of the contraction entry points against the FP64 oracle.

Every case calls the C ABI (through the ctypes binding) on seeded inputs and
compares element by element with the oracle's dense result.  FP64 tolerance:
relative Frobenius error <= 1e-12 (summation order is the only difference).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import contract, io  # noqa: E402
from parity import (FP64_BLOCK_TOL, FP64_TOL, block_rel_err, env_parts, env_to_dense,  # noqa: E402
                    fused_permutation, problem, rel_err, site_parts, site_to_dense)

CASES = [("dense", 1, {}), ("dense", 2, {"m_left": 37, "m_right": 71}),
         ("u1", 3, {}), ("u1", 4, {"density": 0.5}), ("u1u1", 5, {}),
         ("u1", 6, {"m_left": 9, "m_right": 7})]


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def ctx(b):
    c = b.dmrg3s_create(0, 1 << 30)
    yield c
    c.close()


def _gpu(b, pb):
    return (b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]), b.env_from_neutral(pb["R"]),
            b.site_from_neutral(pb["A"]))


def _dense(pb):
    return (io.env_dense(pb["L"]), pb["W"]["W"], io.env_dense(pb["R"]), io.site_dense(pb["A"])[0])


@pytest.mark.parametrize("kind,seed,kw", CASES)
def test_apply_heff_fp64(b, ctx, kind, seed, kw):
    pb = problem(kind, seed, **kw)
    gL, gW, gR, gA = _gpu(b, pb)
    gH = b.empty_site_like(gA.qp, gA.left, gA.right)
    b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "fp64")
    torch.cuda.synchronize()
    L, W, R, A = _dense(pb)
    ref = contract.apply_heff(L, W, R, A)
    got = site_to_dense(b, gH)
    assert rel_err(got, ref) < FP64_TOL
    assert block_rel_err(got, ref, site_parts(A.shape[0], pb["left"], pb["right"])) < FP64_BLOCK_TOL


def test_apply_heff_fp64_repeated_calls_reuse_plan(b, ctx):
    pb = problem("u1", 11)
    gL, gW, gR, gA = _gpu(b, pb)
    gH = b.empty_site_like(gA.qp, gA.left, gA.right)
    L, W, R, A = _dense(pb)
    for k in range(3):
        gA.data.mul_(-0.5)
        A = A * -0.5
        b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "fp64")
        torch.cuda.synchronize()
        assert rel_err(site_to_dense(b, gH), contract.apply_heff(L, W, R, A)) < FP64_TOL


@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("kind,seed,kw", CASES[:5])
def test_expand_fp64(b, ctx, kind, seed, kw, direction):
    pb = problem(kind, seed, **kw)
    gL, gW, gR, gA = _gpu(b, pb)
    L, W, R, A = _dense(pb)
    alpha = 0.37
    if direction == 1:
        fused = b.expanded_bond(gA.right, pb["t"], False)
        gP = b.empty_site_like(gA.qp, gA.left, fused)
        b.dmrg3s_expand(ctx, 1, gL, gW, gA, alpha, gP, "fp64")
        ref = contract.expansion_term_lr(L, W, A, alpha)
        perm = fused_permutation(pb["right"], pb["t"], fused.q.astype(np.int64))
        ref = ref[:, :, perm]
        parts = site_parts(A.shape[0], pb["left"], fused)
    else:
        fused = b.expanded_bond(gA.left, pb["t"], False)
        gP = b.empty_site_like(gA.qp, fused, gA.right)
        b.dmrg3s_expand(ctx, -1, gR, gW, gA, alpha, gP, "fp64")
        ref = contract.expansion_term_rl(R, W, A, alpha)
        perm = fused_permutation(pb["left"], pb["t"], fused.q.astype(np.int64))
        ref = ref[:, perm, :]
        parts = site_parts(A.shape[0], fused, pb["right"])
    torch.cuda.synchronize()
    got = site_to_dense(b, gP)
    assert rel_err(got, ref) < FP64_TOL
    assert block_rel_err(got, ref, parts) < FP64_BLOCK_TOL


@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("kind,seed,kw", CASES)
def test_update_env_fp64(b, ctx, kind, seed, kw, direction):
    pb = problem(kind, seed, **kw)
    gL, gW, gR, gA = _gpu(b, pb)
    L, W, R, A = _dense(pb)
    if direction == 1:
        gO = b.empty_env(gW.tr, gA.right)
        b.dmrg3s_update_env(ctx, 1, gL, gW, gA, gO, "fp64")
        ref = contract.left_env(L, W, A)
        parts = env_parts(W.shape[3], pb["right"])
    else:
        gO = b.empty_env(gW.tl, gA.left)
        b.dmrg3s_update_env(ctx, -1, gR, gW, gA, gO, "fp64")
        ref = contract.right_env(R, W, A)
        parts = env_parts(W.shape[2], pb["left"])
    torch.cuda.synchronize()
    got = env_to_dense(b, gO)
    assert rel_err(got, ref) < FP64_TOL
    assert block_rel_err(got, ref, parts) < FP64_BLOCK_TOL


def test_apply_heff_fp64_full_size_xxz_m512(b, ctx):
    """Central-site shapes of the L=100, m=512 XXZ workload, whole output compared."""
    pb = problem("xxz_l100_m512_u1", 1002)
    gL, gW, gR, gA = _gpu(b, pb)
    gH = b.empty_site_like(gA.qp, gA.left, gA.right)
    b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "fp64")
    torch.cuda.synchronize()
    L, W, R, A = _dense(pb)
    ref = contract.apply_heff(L, W, R, A)
    got = site_to_dense(b, gH)
    assert rel_err(got, ref) < FP64_TOL
    assert block_rel_err(got, ref, site_parts(A.shape[0], pb["left"], pb["right"])) < FP64_BLOCK_TOL


def test_structure_mismatch_is_an_error(b, ctx):
    pb = problem("u1", 7)
    gL, gW, gR, gA = _gpu(b, pb)
    gH = b.empty_site_like(gA.qp, gA.right, gA.left)     # bonds swapped
    with pytest.raises(b.Dmrg3sError) as e:
        b.dmrg3s_apply_heff(ctx, gL, gW, gR, gA, gH, "fp64")
    assert e.value.status == 2
