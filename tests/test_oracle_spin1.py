"""Pins of the spin-S operators and of the S = 1 Heisenberg ring (the first
workload of Sec. VII B 1), oracle side (CPU only).

The spin matrices are pinned by their algebra ([S+, S-] = 2 Sz, Casimir
S(S+1)); the Hamiltonians by closed forms: the spectrum of one bond S_1.S_2,
(J(J+1) - 2 S(S+1)) / 2 with multiplicity 2J+1, and the four-site ring,
H = (S_1 + S_3).(S_2 + S_4), whose ground energy is -2S(2S+1).  The MPO with
the periodic link equals the Kronecker-product Hamiltonian, the library's C++
builder equals the oracle's MPO, and the oracle's DMRG3S reaches exact
diagonalisation on a six-site ring.
"""
import os

import numpy as np
import pytest

from oracle import dmrg3s, exact, labels, models


@pytest.mark.parametrize("two_s", [1, 2, 3, 4])
def test_spin_algebra(two_s):
    sp, sm, sz, eye, q = models.spin_ops(two_s)
    S = two_s / 2.0
    assert np.abs(sp @ sm - sm @ sp - 2 * sz).max() < 1e-13
    sx, sy_im = 0.5 * (sp + sm), 0.5 * (sp - sm)
    casimir = sx @ sx - sy_im @ sy_im + sz @ sz
    assert np.abs(casimir - S * (S + 1) * eye).max() < 1e-13
    assert np.array_equal(q.ravel(), np.rint(2 * np.diag(sz)).astype(int))
    if two_s == 1:
        assert np.array_equal(sp, models.SP) and np.array_equal(sz, models.SZ)


@pytest.mark.parametrize("two_s", [1, 2, 3])
def test_bond_spectrum(two_s):
    S = two_s / 2.0
    H = models.dense_spin_bonds(2, [(0, 1, 1.0, 1.0)], two_s)
    ev = np.sort(np.linalg.eigvalsh(H))
    ref = []
    for J2 in range(0, 2 * two_s + 1, 2):            # total spin J = 0 .. 2S
        J = J2 / 2.0
        ref += [(J * (J + 1) - 2 * S * (S + 1)) / 2] * int(2 * J + 1)
    assert np.abs(ev - np.sort(ref)).max() < 1e-12


@pytest.mark.parametrize("two_s", [1, 2])
def test_four_site_ring_closed_form(two_s):
    S = two_s / 2.0
    bonds = models.ring_bonds(4)
    H_mpo = models.mpo_to_dense(models.mpo_spin_bonds(4, bonds, two_s))
    H_dir = models.dense_spin_bonds(4, bonds, two_s)
    assert np.abs(H_mpo - H_dir).max() < 1e-13
    assert abs(np.linalg.eigvalsh(H_dir)[0] + 2 * S * (2 * S + 1)) < 1e-12


@pytest.mark.parametrize("L", [3, 5])
def test_spin1_ring_mpo_equals_kron(L):
    bonds = models.ring_bonds(L)
    H_mpo = models.mpo_to_dense(models.mpo_spin_bonds(L, bonds, 2))
    assert np.abs(H_mpo - models.dense_spin_bonds(L, bonds, 2)).max() < 1e-13


def test_spin1_ring_mpo_structure():
    mpo = models.mpo_spin_bonds(100, models.ring_bonds(100), 2)
    # the periodic link keeps site 0's three operators open across the chain
    assert max(W.shape[3] for W in mpo.W) == 8
    for i, W in enumerate(mpo.W):
        assert W.shape[:2] == (3, 3)
        mask = labels.mpo_mask(mpo.qphys, mpo.t[i], mpo.t[i + 1])
        assert np.all(W[~mask] == 0.0)


def test_library_builder_equals_oracle_spin1_ring():
    from paper_1501_05504_gb300 import _build, binding as b
    if not os.path.exists(b.LIB_PATH):
        _build.build()
    for L in (4, 7, 100):
        bonds = models.ring_bonds(L)
        ij = np.array([[i, j] for (i, j, _, _) in bonds])
        cp = np.array([[jx, jz] for (_, _, jx, jz) in bonds])
        sites = b.Mpo(b.MODEL_SPIN_BONDS, L, (2.0,), ij, cp).sites()
        mpo = models.mpo_spin_bonds(L, bonds, 2)
        for i, s in enumerate(sites):
            assert np.array_equal(s.W, mpo.W[i])
            assert np.array_equal(s.qp.astype(np.int64), mpo.qphys)
            assert np.array_equal(s.tl.astype(np.int64), mpo.t[i])
            assert np.array_equal(s.tr.astype(np.int64), mpo.t[i + 1])
    with pytest.raises(b.Dmrg3sError):
        b.Mpo(b.MODEL_SPIN_BONDS, 4, (1.5,), ij[:1], cp[:1])


def test_dmrg3s_spin1_ring_reaches_ed():
    L = 6
    bonds = models.ring_bonds(L)
    mpo = models.mpo_spin_bonds(L, bonds, 2)
    mps = dmrg3s.product_state(mpo.qphys, [0, 2] * (L // 2))     # m = +1, -1, ...: S^z = 0
    log = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=64, max_sweeps=10)).run()
    H = models.dense_spin_bonds(L, bonds, 2)
    e0 = exact.ed_ground_energy(H, models.dense_charges(mpo.qphys, L), [0])
    assert abs(log.energies[-1] - e0) < 1e-9 * abs(e0)


@pytest.mark.parametrize("two_s,L", [(1, 8), (2, 6), (3, 4)])
def test_sparse_ed_matches_dense(two_s, L):
    bonds = models.ring_bonds(L)
    H = models.dense_spin_bonds(L, bonds, two_s)
    _, _, _, _, q = models.spin_ops(two_s)
    e_dense = exact.ed_ground_energy(H, models.dense_charges(q, L), [0 if (L * two_s) % 2 == 0 else 1])
    tz = 0 if (L * two_s) % 2 == 0 else 1
    assert abs(exact.ed_sparse_spin_s(L, bonds, two_s, tz) - e_dense) < 1e-10 * abs(e_dense)


def test_sparse_ed_closed_forms():
    # four-site rings: -2S(2S+1); spin-1/2 chains: the existing spin-1/2 routine
    for two_s in (1, 2, 3):
        S = two_s / 2.0
        assert abs(exact.ed_sparse_spin_s(4, models.ring_bonds(4), two_s) + 2 * S * (2 * S + 1)) < 1e-10
    bonds = [(i, i + 1, 1.0, 0.6) for i in range(11)]
    assert abs(exact.ed_sparse_spin_s(12, bonds, 1) - exact.ed_sparse_spin(12, bonds)) < 1e-10
