"""The library's model MPOs equal the oracle's, entry by entry (host functions, CPU only).

The oracle's MPOs are themselves pinned against Kronecker-product
Hamiltonians (test_oracle_models.py); here the product's builders (C++) are
compared with them, and contracted into dense matrices that must equal the
directly built Hamiltonians.
"""
import os

import numpy as np
import pytest

from oracle import models


@pytest.fixture(scope="module")
def b():
    from paper_1501_05504_gb300 import _build, binding
    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    return binding


def _compare(prod_sites, mpo):
    assert len(prod_sites) == mpo.L
    for i, s in enumerate(prod_sites):
        assert s.W.shape == mpo.W[i].shape
        assert np.array_equal(s.W, mpo.W[i])
        assert np.array_equal(s.qp.astype(np.int64), mpo.qphys)
        assert np.array_equal(s.tl.astype(np.int64), mpo.t[i])
        assert np.array_equal(s.tr.astype(np.int64), mpo.t[i + 1])


@pytest.mark.parametrize("L,J,D", [(2, 1.0, 1.0), (7, 0.8, 0.3), (20, 1.0, 1.0)])
def test_xxz(b, L, J, D):
    _compare(b.Mpo(b.MODEL_XXZ, L, (J, D)).sites(), models.mpo_xxz(L, J, D))


@pytest.mark.parametrize("L,t,U", [(2, 1.0, 8.0), (5, 0.7, 2.5)])
def test_hubbard(b, L, t, U):
    _compare(b.Mpo(b.MODEL_HUBBARD, L, (t, U)).sites(), models.mpo_hubbard(L, t, U))


@pytest.mark.parametrize("Lx,Ly", [(2, 3), (4, 4), (16, 4)])
def test_cylinder(b, Lx, Ly):
    bonds = models.cylinder_bonds(Lx, Ly)
    ij = np.array([[i, j] for (i, j, _, _) in bonds])
    cp = np.array([[jx, jz] for (_, _, jx, jz) in bonds])
    _compare(b.Mpo(b.MODEL_SPIN_BONDS, Lx * Ly, (), ij, cp).sites(),
             models.mpo_spin_bonds(Lx * Ly, bonds))


def test_product_mpo_contracts_to_kron_hamiltonian(b):
    L = 5
    sites = b.Mpo(b.MODEL_XXZ, L, (1.0, 0.4)).sites()
    mpo = models.MPO([s.W for s in sites], models.SPIN_HALF_Q, None)
    assert np.abs(models.mpo_to_dense(mpo) - models.dense_xxz(L, 1.0, 0.4)).max() < 1e-14
    sites = b.Mpo(b.MODEL_HUBBARD, 3, (1.0, 4.0)).sites()
    mpo = models.MPO([s.W for s in sites], models.HUB_Q, None)
    assert np.abs(models.mpo_to_dense(mpo) - models.dense_hubbard(3, 1.0, 4.0)).max() < 1e-14
