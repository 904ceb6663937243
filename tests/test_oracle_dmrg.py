"""Pins of the oracle's eigensolver and of full DMRG3S runs (CPU only).

Full runs are pinned by exact diagonalisation and by the free-fermion closed
forms; the stuck-state behaviour at alpha = 0 follows Sec. VII A; the alpha
rule is checked branch by branch against its stated reading of Sec. VI.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import dmrg3s, exact, models


def test_lanczos_matches_dense_eigensolver():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((300, 300))
    H = X + X.T
    lam, x, it = dmrg3s.lanczos_ground(lambda v: H @ v, rng.standard_normal(300), kmax=300, tol=1e-12)
    assert abs(lam - np.linalg.eigvalsh(H)[0]) < 1e-9
    assert np.linalg.norm(H @ x - lam * x) < 1e-6


def test_lanczos_invariant_subspace_stops_early():
    H = np.diag([1.0, 2.0, 3.0, 4.0])
    v = np.array([1.0, 1.0, 0.0, 0.0])
    lam, x, it = dmrg3s.lanczos_ground(lambda y: H @ y, v, kmax=40)
    assert it == 2 and abs(lam - 1.0) < 1e-14


def _xxz(L, Delta, m, sweeps=8):
    mpo = models.mpo_xxz(L, 1.0, Delta)
    mps = dmrg3s.product_state(mpo.qphys, [0, 1] * (L // 2))
    drv = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=m, max_sweeps=sweeps))
    return drv, drv.run()


def test_dmrg3s_u1_reaches_exact_diagonalisation():
    L = 10
    drv, log = _xxz(L, 1.0, 32)
    H = models.dense_xxz(L, 1.0, 1.0)
    e0 = exact.ed_ground_energy(H, models.dense_charges(models.SPIN_HALF_Q, L), [0])
    assert log.converged
    assert abs(log.energies[-1] - e0) < 1e-10 * abs(e0)


def test_dmrg3s_xx_chain_closed_form():
    drv, log = _xxz(10, 0.0, 32)
    assert abs(log.energies[-1] - exact.xx_chain_energy(10)) < 1e-10 * 4


def test_dmrg3s_dense_random_start_reaches_ed():
    L = 10
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    nos = np.zeros((2, 0), dtype=np.int64)
    mpo.qphys = nos
    mpo.t = [np.zeros((t.shape[0], 0), dtype=np.int64) for t in mpo.t]
    Ms = dmrg3s.left_normalise(si.random_dense_mps(si.rng_for(1001), L, 2, 32))
    mps = dmrg3s.MPS(Ms, [np.zeros((T.shape[1], 0), dtype=np.int64) for T in Ms]
                     + [np.zeros((1, 0), dtype=np.int64)], nos)
    log = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=32, max_sweeps=8)).run()
    e0 = exact.ed_ground_energy(models.dense_xxz(L, 1.0, 1.0))
    assert abs(log.energies[-1] - e0) < 1e-10 * abs(e0)


def test_dmrg3s_free_fermions_closed_form():
    L = 4
    mpo = models.mpo_hubbard(L, 1.0, 0.0)
    mps = dmrg3s.product_state(mpo.qphys, [2, 1] * (L // 2))
    log = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=64, max_sweeps=8)).run()
    assert abs(log.energies[-1] - exact.free_fermion_energy(L, 2, 2)) < 1e-10


def test_dmrg3s_hubbard_matches_ed():
    L, U = 4, 8.0
    mpo = models.mpo_hubbard(L, 1.0, U)
    mps = dmrg3s.product_state(mpo.qphys, [2, 1] * (L // 2))
    log = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=64, max_sweeps=10)).run()
    H = models.dense_hubbard(L, 1.0, U)
    e0 = exact.ed_ground_energy(H, models.dense_charges(models.HUB_Q, L), [L, 0])
    assert abs(log.energies[-1] - e0) < 1e-9 * abs(e0)


def test_alpha_zero_is_stuck_and_expansion_escapes():
    """Sec. VII A: without enrichment a U(1) product state cannot grow its bonds."""
    L = 10
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    o0 = dmrg3s.SweepOptions(m_max=32, max_sweeps=3)
    o0.alpha = dmrg3s.AlphaRule(alpha0=0.0, fixed=True)
    log0 = dmrg3s.DMRG3S(mpo, dmrg3s.product_state(mpo.qphys, [0, 1] * 5), o0).run()
    assert max(log0.bond_dims[-1]) == 1
    assert abs(log0.energies[-1] - (-(L - 1) / 4.0)) < 1e-12      # Neel energy
    drv, log1 = _xxz(L, 1.0, 32)
    assert log1.energies[-1] < log0.energies[-1] - 1.0


def test_energy_monotone_at_alpha_zero_after_warmup():
    drv, _ = _xxz(10, 1.0, 8, sweeps=1)
    drv.opts.alpha = dmrg3s.AlphaRule(alpha0=0.0, fixed=True)
    drv.alpha = 0.0
    log = dmrg3s.SweepLog()
    for _ in range(2):
        drv.sweep(log)
    lam = np.array(log.lambdas)
    assert np.all(np.diff(lam) <= 1e-11)


def test_variational_bound():
    L = 10
    drv, log = _xxz(L, 1.0, 6, sweeps=3)
    e0 = exact.ed_ground_energy(models.dense_xxz(L, 1.0, 1.0),
                                models.dense_charges(models.SPIN_HALF_Q, L), [0])
    assert min(log.lambdas) >= e0 - 1e-12


@pytest.mark.parametrize("e_in,lam,e_f,factor", [
    (-1.0, -1.0 - 1e-15, -1.0, 0.8),          # |dE_O| tiny: shrink
    (-1.0, -2.0, -2.1, 1.25),                 # dE_T < 0: grow
    (-1.0, -2.0, -1.9, 1.25),                 # r = 0.1 < 0.3: grow
    (-1.0, -2.0, -1.5, 0.8),                  # 0.3 < r = 0.5 <= 1: shrink
    (-1.0, -2.0, -0.5, 0.64),                 # r = 1.5 > 1: shrink twice
])
def test_alpha_rule_branches(e_in, lam, e_f, factor):
    rule = dmrg3s.AlphaRule()
    assert abs(rule.update(1e-3, e_in, lam, e_f) - 1e-3 * factor) < 1e-18
    assert dmrg3s.AlphaRule(fixed=True).update(1e-3, e_in, lam, e_f) == 1e-3
    assert dmrg3s.AlphaRule(alpha_max=1e-3).update(1e-3, -1.0, -2.0, -2.1) == 1e-3
