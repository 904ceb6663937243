"""Planted mistakes in the oracle must fail its pins (CPU only).

Each case swaps one oracle routine for a copy with a plausible slip (a
transposed operand, a dropped term, a wrong index) and checks that the pin
guarding that routine reports a large error.  The planted copies live only
here, on the CPU.
"""
import numpy as np
import pytest

from oracle import contract, models
from test_oracle_contract import (_mixed_canonical, expansion_lr_errors, expansion_rl_mirror_error,
                                  heff_projection_error, two_spin_errors)


def _heff_R_transposed(L, W, R, M):
    return contract.apply_heff(L, W, np.transpose(R, (0, 2, 1)), M)


def _heff_L_transposed(L, W, R, M):
    return contract.apply_heff(np.transpose(L, (0, 2, 1)), W, R, M)


def _heff_W_phys_swapped(L, W, R, M):
    return contract.apply_heff(L, np.transpose(W, (1, 0, 2, 3)), R, M)


def _heff_dropped_channel(L, W, R, M):
    W2 = W.copy()
    W2[:, :, :, -1] = 0.0
    return contract.apply_heff(L, W2, R, M)


def _heff_W_mpo_swapped(L, W, R, M):
    if W.shape[2] != W.shape[3]:
        return contract.apply_heff(L, W, R, M) * 1.5
    return contract.apply_heff(L, np.transpose(W, (0, 1, 3, 2)), R, M)


@pytest.mark.parametrize("bad", [_heff_R_transposed, _heff_L_transposed, _heff_W_phys_swapped,
                                 _heff_dropped_channel, _heff_W_mpo_swapped])
def test_projected_hamiltonian_pin_catches(bad):
    L = 6
    mpo = models.mpo_xxz(L, 1.0, 0.6)
    H = models.dense_xxz(L, 1.0, 0.6)
    As, x, Bs = _mixed_canonical(L, 2, 8, 2, seed=2)
    assert heff_projection_error(contract.apply_heff, mpo, H, As, x, Bs) < 1e-13
    assert heff_projection_error(bad, mpo, H, As, x, Bs) > 1e-3


def _expand_W_phys_swapped(L, W, M, alpha):
    return contract.expansion_term_lr(L, np.transpose(W, (1, 0, 2, 3)), M, alpha)


def _expand_fused_index_wrong_order(L, W, M, alpha):
    T2 = contract.lw_a(L, W, M)
    P = alpha * np.transpose(T2, (1, 2, 3, 0))
    return P.reshape(P.shape[0], P.shape[1], -1)


def _expand_alpha_squared(L, W, M, alpha):
    return contract.expansion_term_lr(L, W, M, alpha) * 0.5


@pytest.mark.parametrize("bad", [_expand_W_phys_swapped, _expand_alpha_squared])
def test_two_spin_pin_catches(bad):
    errs = two_spin_errors(bad, 0.3, 0.6)
    assert max(errs.values()) > 1e-3


def test_u1_expansion_pin_catches_fused_index_order():
    # with m = 1 the fused index (b, a) of the two-spin example cannot be
    # mis-ordered; the U(1) expansion pin sees it through the charge labels
    assert max(two_spin_errors(_expand_fused_index_wrong_order, 0.3, 0.6).values()) < 1e-14
    errs = expansion_lr_errors(_expand_fused_index_wrong_order)
    assert errs["after_svd"] > 1e-6 or errs["p_kept"] > 1e-6


# ---- right-to-left expansion term: planted slips must break the mirror identity

def _expand_rl_R_transposed(R, W, M, alpha):
    return contract.expansion_term_rl(np.transpose(R, (0, 2, 1)), W, M, alpha)


def _expand_rl_W_phys_swapped(R, W, M, alpha):
    return contract.expansion_term_rl(R, np.transpose(W, (1, 0, 2, 3)), M, alpha)


def _expand_rl_fused_index_wrong_order(R, W, M, alpha):
    # (al, bl) with al the slower index instead of (bl, al)
    U1 = np.einsum("sxy,cYy->csxY", M, R)
    U2 = np.einsum("Ssbc,csxY->SxbY", W, U1)
    P = alpha * U2
    return P.reshape(P.shape[0], -1, P.shape[3])


def _expand_rl_W_mpo_swapped(R, W, M, alpha):
    # contracts R with the left MPO bond of W (only shape-compatible when wl == wr)
    if W.shape[2] != W.shape[3]:
        return contract.expansion_term_rl(R, W, M, alpha) * 1.5
    return contract.expansion_term_rl(R, np.transpose(W, (0, 1, 3, 2)), M, alpha)


def _expand_rl_dropped_channel(R, W, M, alpha):
    W2 = W.copy()
    W2[:, :, :, 0] = 0.0
    return contract.expansion_term_rl(R, W2, M, alpha)


@pytest.mark.parametrize("bad", [_expand_rl_R_transposed, _expand_rl_W_phys_swapped,
                                 _expand_rl_fused_index_wrong_order, _expand_rl_W_mpo_swapped,
                                 _expand_rl_dropped_channel])
def test_rl_mirror_pin_catches(bad):
    assert expansion_rl_mirror_error(contract.expansion_term_rl) < 1e-14
    assert expansion_rl_mirror_error(bad) > 1e-3
