"""The truncation's FP64 SVD (QR, then one-sided Jacobi on R^T) through the C ABI.

Pins: the singular values of numpy's LAPACK SVD of the same matrix (within
1e-13 of the largest), orthonormal singular vectors (1e-12), reconstruction
A = U S V^T (1e-13 of the largest singular value), descending order; shapes
from a single element to the largest charge sector of the m = 512 XXZ update
(762 x 245), graded spectra down to 1e-14, rank deficiency, the zero matrix
and repeated singular values, each alone and all in one batch.  Sweeps with
this SVD reach the energy of sweeps with cuSOLVER gesvd.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import seeded_inputs as si  # noqa: E402


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.slib()
    return binding


@pytest.fixture(scope="module")
def ctx(b):
    c = b.dmrg3s_create(0, 1 << 30)
    yield c
    c.close()


# (rows, cols, log10 of the smallest singular value, rank)
SHAPES = [(1, 1, 0, 1), (5, 1, 0, 1), (2, 2, 0, 2), (7, 3, -3, 3), (30, 30, -8, 30),
          (64, 17, -13, 17), (60, 20, -13, 12), (10, 4, 0, 0), (200, 65, -13, 65),
          (351, 165, -14, 165), (762, 245, -13, 245)]


def _matrix(rng, m, n, lo, rank):
    qa, _ = np.linalg.qr(rng.standard_normal((m, n)))
    qb, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, lo, n)
    s[rank:] = 0.0
    return (qa * s) @ qb.T


def _repeated(rng):
    qa, _ = np.linalg.qr(rng.standard_normal((40, 10)))
    qb, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    return (qa * np.array([1, 1, 1, .5, .5, .25, .25, .25, 1e-3, 0.0])) @ qb.T


def _check(X, res):
    u, s, vt = (None if t is None else t.cpu().numpy() for t in res)
    ref = np.linalg.svd(X, compute_uv=False)
    s0 = max(ref[0], 1e-300)
    assert np.all(np.diff(s) <= 0.0)
    assert np.abs(s - ref).max() <= 1e-13 * s0
    nz = s > 0
    if nz.any():
        V = vt[nz]
        assert np.abs(V @ V.T - np.eye(V.shape[0])).max() < 1e-12
    assert np.all(vt[~nz] == 0.0)
    if u is not None:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < 1e-12
        assert np.abs((u * s) @ vt - X).max() <= 1e-13 * s0


def test_svd_each_shape(b, ctx):
    rng = si.rng_for(41)
    for (m, n, lo, rk) in SHAPES:
        X = _matrix(rng, m, n, lo, rk)
        res = b.dmrg3s_svd(ctx, [torch.from_numpy(X).cuda()])[0]
        _check(X, res)
    X = _repeated(rng)
    _check(X, b.dmrg3s_svd(ctx, [torch.from_numpy(X).cuda()])[0])


def test_svd_one_batch_and_right_vectors_only(b, ctx):
    rng = si.rng_for(42)
    mats = [_matrix(rng, *sh) for sh in SHAPES] + [_repeated(rng)]
    for want_u in (True, False):
        out = b.dmrg3s_svd(ctx, [torch.from_numpy(X).cuda() for X in mats], want_u=want_u)
        for X, res in zip(mats, out):
            _check(X, res)


def test_svd_shape_errors(b, ctx):
    with pytest.raises(RuntimeError):
        b.dmrg3s_svd(ctx, [torch.zeros(3, 5, dtype=torch.float64, device="cuda")])


def test_sweeps_jacobi_vs_gesvd(b, ctx):
    """Sweeps of the XXZ chain with each SVD reach the same energy.  (The
    trajectories from the Neel state differ at intermediate sweeps: equal
    singular values of symmetry-related sectors may be cut differently.  The
    same-input comparison of one update is the oracle parity test, run with
    both methods.)"""
    L = 24
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    out = {}
    for method in ("gesvd", "jacobi"):
        st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (L // 2)), None, None,
                                   L - 1)
        rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 4, 1e-14, b.update_opts(64, svd=method))
        info = b.dmrg3s_local_update(st, -1, 1e-3, b.update_opts(48, svd=method))
        out[method] = (rep["energies"][-1], info)
        st.close()
    eg, ig = out["gesvd"]
    ej, ij = out["jacobi"]
    assert abs(eg - ej) < 1e-9 * abs(eg)
    assert ig["new_bond_dim"] == ij["new_bond_dim"]
    assert abs(ig["energy_after"] - ij["energy_after"]) < 1e-9 * abs(ig["energy_after"])


def test_sweep_limit_reports_not_converged(b, ctx, monkeypatch):
    """With the sweep limit at one sweep a graded 30 x 30 matrix is not done:
    dmrg3s_svd reports NOT_CONVERGED (status 6) instead of a result."""
    rng = si.rng_for(43)
    X = _matrix(rng, 30, 30, -8, 30)
    monkeypatch.setenv("DMRG3S_JACOBI_SWEEPS", "1")
    with pytest.raises(b.Dmrg3sError) as e:
        b.dmrg3s_svd(ctx, [torch.from_numpy(X).cuda()])
    assert e.value.status == 6
    monkeypatch.delenv("DMRG3S_JACOBI_SWEEPS")
    _check(X, b.dmrg3s_svd(ctx, [torch.from_numpy(X).cuda()])[0])


def test_local_update_falls_back_to_gesvd(b, ctx, monkeypatch):
    """An update whose Jacobi sweeps stop unconverged (limit forced to one
    sweep) redoes its SVD with gesvd on the restored matrix: it reports the
    fallback and matches the gesvd update of the same state."""
    L = 16
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 0.6)).sites()
    res = {}
    for method, limit in (("gesvd", None), ("jacobi", "1")):
        st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (L // 2)), None, None,
                                   L - 1)
        b.dmrg3s_sweep(st, b.alpha_rule(1e-2, fixed=True), 2, 1e-14,
                       b.update_opts(32, svd="gesvd"))
        for _ in range(L // 2 - 1):   # centre to the middle, where the sectors are largest
            b.dmrg3s_local_update(st, -1, 1e-2, b.update_opts(32, svd="gesvd"))
        if limit:
            monkeypatch.setenv("DMRG3S_JACOBI_SWEEPS", limit)
        res[method] = b.dmrg3s_local_update(st, -1, 1e-2, b.update_opts(32, svd=method))
        monkeypatch.delenv("DMRG3S_JACOBI_SWEEPS", raising=False)
        st.close()
    assert res["jacobi"]["svd_fallback"] and not res["gesvd"]["svd_fallback"]
    for k in ("energy_after", "discarded_weight", "new_bond_dim", "lambda"):
        assert res["jacobi"][k] == res["gesvd"][k], k
