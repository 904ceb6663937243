"""Pins of the oracle's Hamiltonians and exact energies (CPU only).

The MPO route (Sec. II: H = W_1 ... W_l) is compared entry by entry with the
Hamiltonian built independently from Kronecker products; exact
diagonalisation is pinned by the Jordan-Wigner closed forms of the open XX
chain and of free fermions.
"""
import numpy as np
import pytest

from oracle import exact, labels, models


@pytest.mark.parametrize("L", [2, 3, 5, 7])
def test_xxz_mpo_equals_kron(L):
    rng = np.random.default_rng(L)
    J, D = rng.uniform(0.5, 1.5), rng.uniform(0.0, 2.0)
    H_mpo = models.mpo_to_dense(models.mpo_xxz(L, J, D))
    H_dir = models.dense_xxz(L, J, D)
    assert np.abs(H_mpo - H_dir).max() < 1e-13


@pytest.mark.parametrize("L", [2, 3])
def test_hubbard_mpo_equals_jordan_wigner(L):
    rng = np.random.default_rng(10 + L)
    t, U = rng.uniform(0.5, 1.5), rng.uniform(0.0, 8.0)
    H_mpo = models.mpo_to_dense(models.mpo_hubbard(L, t, U))
    H_dir = models.dense_hubbard(L, t, U)
    assert np.abs(H_mpo - H_dir).max() < 1e-13


@pytest.mark.parametrize("Lx,Ly", [(2, 3), (3, 2), (2, 4)])
def test_cylinder_mpo_equals_kron(Lx, Ly):
    bonds = models.cylinder_bonds(Lx, Ly)
    L = Lx * Ly
    H_mpo = models.mpo_to_dense(models.mpo_spin_bonds(L, bonds))
    H_dir = models.dense_spin_bonds(L, bonds)
    assert np.abs(H_mpo - H_dir).max() < 1e-13


def test_bond_builder_reproduces_xxz_chain():
    L = 6
    bonds = [(i, i + 1, 1.0, 0.7) for i in range(L - 1)]
    a, b = models.mpo_spin_bonds(L, bonds), models.mpo_xxz(L, 1.0, 0.7)
    assert [W.shape for W in a.W] == [W.shape for W in b.W]
    assert np.abs(models.mpo_to_dense(a) - models.mpo_to_dense(b)).max() < 1e-14


def test_cylinder_bond_dimension():
    mpo = models.mpo_spin_bonds(64, models.cylinder_bonds(16, 4))
    assert max(W.shape[3] for W in mpo.W) == 14


@pytest.mark.parametrize("build", [lambda: models.mpo_xxz(5, 1.0, 0.3),
                                   lambda: models.mpo_hubbard(4, 1.0, 2.0),
                                   lambda: models.mpo_spin_bonds(8, models.cylinder_bonds(2, 4))])
def test_mpo_conserves_charge(build):
    mpo = build()
    for i, W in enumerate(mpo.W):
        mask = labels.mpo_mask(mpo.qphys, mpo.t[i], mpo.t[i + 1])
        assert np.all(W[~mask] == 0.0)


@pytest.mark.parametrize("L", [6, 8, 10])
def test_ed_matches_xx_closed_form(L):
    H = models.dense_xxz(L, 1.0, 0.0)
    q = models.dense_charges(models.SPIN_HALF_Q, L)
    e = exact.ed_ground_energy(H, q, [0])
    assert abs(e - exact.xx_chain_energy(L)) < 1e-12


def test_xx_closed_form_value_l12():
    # closed form sum_{cos<0} cos(pi k / 13), evaluated independently of the ED
    k = np.arange(1, 13)
    ref = sum(np.cos(np.pi * kk / 13) for kk in k if np.cos(np.pi * kk / 13) < 0)
    assert abs(exact.xx_chain_energy(12) - ref) < 1e-14
    assert abs(exact.xx_chain_energy(12) - (-3.6481149053)) < 1e-9


@pytest.mark.parametrize("L", [2, 3, 4])
def test_ed_matches_free_fermions(L):
    H = models.dense_hubbard(L, 1.0, 0.0)
    q = models.dense_charges(models.HUB_Q, L)
    n_up, n_dn = (L + 1) // 2, L // 2
    e = exact.ed_ground_energy(H, q, [L, n_up - n_dn])
    assert abs(e - exact.free_fermion_energy(L, n_up, n_dn)) < 1e-12


def test_sparse_ed_matches_dense():
    L = 10
    bonds = [(i, i + 1, 1.0, 1.0) for i in range(L - 1)]
    H = models.dense_xxz(L, 1.0, 1.0)
    q = models.dense_charges(models.SPIN_HALF_Q, L)
    assert abs(exact.ed_sparse_spin(L, bonds, 0) - exact.ed_ground_energy(H, q, [0])) < 1e-10
    bonds0 = [(i, i + 1, 1.0, 0.0) for i in range(14 - 1)]
    assert abs(exact.ed_sparse_spin(14, bonds0, 0) - exact.xx_chain_energy(14)) < 1e-10
