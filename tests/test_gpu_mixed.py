"""Mixed precision at the energy tolerance, the small dense Heisenberg benchmark,
and the alpha rule against the oracle (all on the GPU, through the C ABI).

* Sweeps with 3xTF32 block products throughout, and the precision ladder of
  dmrg3s_sweep (3xTF32 until the sweep-to-sweep energy change drops below
  1e-7, FP64 afterwards), reach the exact ground energy to <= 1e-9 relative
  (the energy tolerance of the mixed-precision path) on the U(1) XXZ chain
  L = 10 (Neel start), the dense (no symmetry blocks) Heisenberg chain L = 10
  from a random MPS, and the Hubbard chain L = 4, U = 8 (Sec. VII B sets the
  convergence criterion; exact diagonalisation is the pin).
* The dense Heisenberg benchmark as specified: J = 1, open chain, L = 20,
  d = 2, w = 5, one block, m_max = 64, random N(0, 1) MPS (seed 1001)
  left-normalised, alpha0 = 1e-2 with the adaptive rule, 6 sweeps, against
  sparse exact diagonalisation of L = 20 (S^z = 0; -8.682473334399) and the
  oracle's own run from the same start; the L = 12 chain against dense ED
  (-5.14209063284).
* The mixing factor after every local update (Sec. VI) equals the oracle's
  trajectory (SweepLog.alphas) from the same start with the same rule.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import seeded_inputs as si  # noqa: E402
from oracle import dmrg3s as odm, exact, models  # noqa: E402

E_TOL = 1e-9          # relative energy tolerance of the mixed-precision path


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


def _dense_mpo(b, L):
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    for s in W:     # the dense problem drops the charges
        s.qp = np.zeros((2, 0), np.int32)
        s.tl = np.zeros((s.tl.shape[0], 0), np.int32)
        s.tr = np.zeros((s.tr.shape[0], 0), np.int32)
    return W


def _random_dense_state(b, ctx, L, m, seed):
    """Random N(0, 1) MPS, left-normalised on the device by gauge moves (no
    eigensolver, no expansion, nothing truncated), centre on the last site."""
    W = _dense_mpo(b, L)
    Ms = si.random_dense_mps(si.rng_for(seed), L, 2, m)
    st = b.dmrg3s_state_create(ctx, W, [b.site_from_neutral(x) for x in si.dense_mps_sites(Ms)],
                               None, None, 0)
    gauge = b.update_opts(10 ** 6, skip_eigensolver=True)
    for _ in range(L - 1):
        b.dmrg3s_local_update(st, 1, 0.0, gauge)
    return st


def _neel(b, ctx, L, params=(1.0, 1.0)):
    W = b.Mpo(b.MODEL_XXZ, L, params).sites()
    return b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (L // 2)), None, None,
                                 L - 1)


def _hubbard(b, ctx, L, U):
    W = b.Mpo(b.MODEL_HUBBARD, L, (1.0, U)).sites()
    return b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [2, 1] * (L // 2)), None, None,
                                 L - 1)


def _ed(case):
    if case == "xxz_u1_l10":
        return exact.ed_ground_energy(models.dense_xxz(10, 1.0, 1.0),
                                      models.dense_charges(models.SPIN_HALF_Q, 10), [0])
    if case == "dense_l10":
        return exact.ed_ground_energy(models.dense_xxz(10, 1.0, 1.0))
    return exact.ed_ground_energy(models.dense_hubbard(4, 1.0, 8.0),
                                  models.dense_charges(models.HUB_Q, 4), [4, 0])


def _state(b, ctx, case):
    if case == "xxz_u1_l10":
        return _neel(b, ctx, 10), 32
    if case == "dense_l10":
        return _random_dense_state(b, ctx, 10, 32, 1001), 32
    return _hubbard(b, ctx, 4, 8.0), 64


@pytest.mark.parametrize("ladder", [False, True])
@pytest.mark.parametrize("case", ["xxz_u1_l10", "dense_l10", "hubbard_l4"])
def test_mixed_precision_sweeps_reach_ed(b, ctx, case, ladder):
    st, m = _state(b, ctx, case)
    opts = b.update_opts(m, tol=1e-10, prec="tf32x3")
    if ladder:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 16, 1e-11, opts, final_prec="fp64",
                             switch_tol=1e-7)
        assert 1 <= rep["bulk_sweeps"] < rep["sweeps"]
    else:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 16, 1e-11, opts)
    st.close()
    e0 = _ed(case)
    assert rep["energy"] >= e0 - 1e-12 * abs(e0)          # variational
    assert abs(rep["energy"] - e0) <= E_TOL * abs(e0), (rep["energies"], e0)


def _oracle_dense_run(L, m, seed, sweeps):
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    nos = np.zeros((2, 0), dtype=np.int64)
    mpo_d = models.MPO(mpo.W, nos, [np.zeros((t.shape[0], 0), dtype=np.int64) for t in mpo.t])
    As = odm.left_normalise(si.random_dense_mps(si.rng_for(seed), L, 2, m))
    mps = odm.MPS(As, [np.zeros((A.shape[1], 0), dtype=np.int64) for A in As]
                  + [np.zeros((1, 0), dtype=np.int64)], nos)
    o = odm.SweepOptions(m_max=m, max_sweeps=sweeps, conv_tol=0.0)
    return odm.DMRG3S(mpo_d, mps, o).run()


@pytest.mark.parametrize("ladder", [False, True])
def test_dense_heisenberg_l20_m64_benchmark(b, ctx, ladder):
    """L = 20, dense, m_max = 64, random start (seed 1001), 6 sweeps."""
    L, m = 20, 64
    st = _random_dense_state(b, ctx, L, m, 1001)
    if ladder:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 6, 0.0, b.update_opts(m, prec="tf32x3"),
                             final_prec="fp64", switch_tol=1e-7)
    else:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 6, 0.0, b.update_opts(m))
    st.close()
    assert rep["sweeps"] == 6
    e_ed = exact.ed_sparse_spin(L, [(i, i + 1, 1.0, 1.0) for i in range(L - 1)])
    assert abs(e_ed - (-8.682473334399)) < 1e-11
    assert rep["energy"] >= e_ed - 1e-12 * abs(e_ed)
    assert abs(rep["energy"] - e_ed) <= E_TOL * abs(e_ed), (rep["energies"], e_ed)
    if not ladder:
        # the oracle from the same start with the same rule, sweep by sweep
        log = _oracle_dense_run(L, m, 1001, 6)
        for eg, eo in zip(rep["energies"], log.energies):
            assert abs(eg - eo) <= E_TOL * abs(eo)


def test_dense_heisenberg_l12_reaches_ed(b, ctx):
    L, m = 12, 64
    st = _random_dense_state(b, ctx, L, m, 1001)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 6, 1e-12, b.update_opts(m, tol=1e-12))
    st.close()
    e0 = exact.ed_ground_energy(models.dense_xxz(L, 1.0, 1.0))
    assert abs(e0 - (-5.14209063284)) < 1e-10
    assert abs(rep["energy"] - e0) <= 1e-10 * abs(e0)


def test_alpha_trajectory_matches_oracle(b, ctx):
    """alpha after each of the 36 updates of two sweeps (U(1) XXZ L = 10, Neel start)."""
    L, m, sweeps = 10, 32, 2
    st = _neel(b, ctx, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), sweeps, 0.0, b.update_opts(m, tol=1e-12))
    st.close()
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    o = odm.SweepOptions(m_max=m, max_sweeps=sweeps, conv_tol=0.0, lanczos_tol=1e-12)
    log = odm.DMRG3S(mpo, odm.product_state(mpo.qphys, [0, 1] * (L // 2)), o).run()
    got, want = np.array(rep["alphas"]), np.array(log.alphas)
    assert got.shape == want.shape == (sweeps * 2 * (L - 1),)
    # the rule grows and shrinks alpha: the trajectory is not constant
    assert len(set(np.round(np.log(want) / np.log(1.25), 6))) > 3
    assert np.abs(got - want).max() <= 1e-12 * want.max()
    for eg, eo in zip(rep["energies"], log.energies):
        assert abs(eg - eo) <= 1e-10 * abs(eo)
