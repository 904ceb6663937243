"""H_eff parity at the full sizes of the Hubbard (L=64, m=1024, U(1)xU(1)) and
4x16 cylinder (m=2048, w=14, U(1)) workloads, on sampled output rows.

The dense oracle product is too slow at these sizes, so the oracle evaluates
the definition of H_eff for 16 sampled left bra indices (apply_heff_rows)
and the device result is compared on those rows: FP64 within 1e-12, 3xTF32
within 1e-6 (relative Frobenius), in the launch configuration of
bench.py --heff-only --workload.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
from oracle import contract, io  # noqa: E402
from parity import FP64_TOL, TF32X3_TOL, rel_err, site_to_dense  # noqa: E402


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.slib()
    return binding


@pytest.fixture(scope="module")
def ctx(b):
    c = b.dmrg3s_create(0, 4 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["hubbard_l64_m1024_u1u1", "cylinder_4x16_m2048_u1"])
def test_full_size_heff_on_sampled_rows(b, ctx, name):
    W, Le, Re, M = bench.heff_problem_specs(b, name)
    gL, gR, gM = b.env_from_neutral(Le), b.env_from_neutral(Re), b.site_from_neutral(M)
    L, R, A = io.env_dense(Le), io.env_dense(Re), io.site_dense(M)[0]
    rows = np.sort(np.random.default_rng(11).choice(A.shape[1], 16, replace=False))
    ref = contract.apply_heff_rows(L, W.W, R, A, rows)
    for prec, tol in (("fp64", FP64_TOL), ("tf32x3", TF32X3_TOL)):
        gH = b.empty_site_like(gM.qp, gM.left, gM.right)
        b.dmrg3s_apply_heff(ctx, gL, W, gR, gM, gH, prec)
        b.dmrg3s_sync(ctx)
        got = site_to_dense(b, gH)[:, rows, :]
        assert rel_err(got, ref) < tol, prec
