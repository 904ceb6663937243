"""Whole-run checks on the GPU with exact answers (workloads beyond the hot-path table).

* Stuck spins (Sec. VII A): from the Neel state of the L=20 Heisenberg chain
  with U(1) blocks, single-site updates without expansion (alpha = 0) cannot
  leave the m = 1 product state, so the energy stays at <Neel|H|Neel> =
  -(L-1)/4; with the adaptive expansion term the sweeps reach the exact
  ground energy (sparse exact diagonalisation in the S^z = 0 sector).
* Free fermions at full length: the open XX chain with L = 100 (the XXZ MPO
  at Delta = 0) against the closed-form energy of the filled single-particle
  levels, and the half-filled U = 0 Hubbard chain (d = 4, U(1)xU(1) blocks,
  Jordan-Wigner MPO) against its closed form.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import exact  # noqa: E402


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


def _neel(b, ctx, W, L):
    return b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (L // 2)), None, None,
                                 L - 1)


def test_stuck_spins_l20(b, ctx):
    L = 20
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    st = _neel(b, ctx, W, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(0.0, fixed=True), 2, 1e-12, b.update_opts(512))
    assert abs(rep["energy"] + (L - 1) / 4.0) < 1e-12
    st.close()
    st = _neel(b, ctx, W, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 20, 1e-12, b.update_opts(512, tol=1e-12))
    st.close()
    e0 = exact.ed_sparse_spin(L, [(i, i + 1, 1.0, 1.0) for i in range(L - 1)])
    assert abs(rep["energy"] - e0) < 1e-9 * abs(e0)


@pytest.mark.parametrize("svd", ["gesvd", "jacobi"])
def test_xx_chain_l100_closed_form(b, ctx, svd):
    """(Free fermions: Schmidt spectra with many equal singular values, the
    hardest case met for the Jacobi SVD.)"""
    L = 100
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 0.0)).sites()
    st = _neel(b, ctx, W, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 12, 1e-11, b.update_opts(256, svd=svd))
    st.close()
    e0 = exact.xx_chain_energy(L, 1.0)
    print("XX chain L=100 (%s): %d updates of %d fell back to gesvd" % (
        svd, rep["svd_fallbacks"], 2 * (L - 1) * rep["sweeps"]))
    assert abs(rep["energy"] - e0) < 1e-8 * abs(e0)


def test_hubbard_u0_closed_form(b, ctx):
    L = 32
    W = b.Mpo(b.MODEL_HUBBARD, L, (1.0, 0.0)).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [2, 1] * (L // 2)), None, None,
                               L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 12, 1e-11, b.update_opts(512))
    st.close()
    e0 = exact.free_fermion_energy(L, L // 2, L // 2)
    assert abs(rep["energy"] - e0) < 1e-8 * abs(e0)


def test_spin1_ring_l6_matches_ed(b, ctx):
    """S = 1 Heisenberg ring (Sec. VII B 1 at L = 6; d = 3, periodic link
    (0, 5), w = 8): sweeps reach the exact ground energy of the S^z = 0 sector."""
    from oracle import models
    L = 6
    bonds = models.ring_bonds(L)
    ij = [[i, j] for (i, j, _, _) in bonds]
    cp = [[jx, jz] for (_, _, jx, jz) in bonds]
    W = b.Mpo(b.MODEL_SPIN_BONDS, L, (2.0,), ij, cp).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 2] * (L // 2)), None, None,
                               L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 12, 1e-13, b.update_opts(64, tol=1e-12))
    st.close()
    mpo = models.mpo_spin_bonds(L, bonds, 2)
    e0 = exact.ed_ground_energy(models.dense_spin_bonds(L, bonds, 2),
                                models.dense_charges(mpo.qphys, L), [0])
    assert abs(rep["energy"] - e0) < 1e-9 * abs(e0)


def test_spin1_ring_l100_paper_energy(b, ctx):
    """S = 1 Heisenberg chain with periodic boundary conditions, L = 100 (Sec.
    VII B 1: d = 3, the periodic link (0, 99) in the MPO, w = 8, U(1) S^z = 0),
    against the ground-state energy the paper reports, E0 = -140.148404.
    The precision ladder (3xTF32, then FP64) at m_max = 256: a periodic chain
    needs a larger bond dimension than the paper's open-chain runs for the
    same accuracy, so the bound is the variational one plus the relative
    deviation this m reaches (1.2e-6 measured on the GB300)."""
    from oracle import models
    L, m = 100, 256
    bonds = models.ring_bonds(L)
    ij = [[i, j] for (i, j, _, _) in bonds]
    cp = [[jx, jz] for (_, _, jx, jz) in bonds]
    W = b.Mpo(b.MODEL_SPIN_BONDS, L, (2.0,), ij, cp).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 2] * (L // 2)), None, None,
                               L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 14, 1e-9, b.update_opts(m, prec="tf32x3"),
                         final_prec="fp64", switch_tol=1e-6)
    st.close()
    e_paper = -140.148404
    rel = (rep["energy"] - e_paper) / abs(e_paper)
    print("S=1 ring L=100 m=%d: E = %.9f (%d sweeps, %.1f s), rel. deviation from the paper %.2e"
          % (m, rep["energy"], rep["sweeps"], rep["seconds"][-1], rel))
    assert rep["energy"] >= e_paper - 5e-7          # the paper's value is rounded to 1e-6
    assert rel < 5e-6                               # measured: 1.2e-6 at m = 256


def test_hubbard_u0_l100_closed_form(b, ctx):
    """Half-filled U = 0 Hubbard chain (free fermions), L = 100, N = 100
    (Sec. VII B 4): the closed form of the filled single-particle levels,
    -126.6023783108, and the paper's converged DMRG value -126.602376 (the
    paper's m = 1200 run lies 1.8e-8 above the closed form; this m = 512 run
    reached 8.3e-7 on the GB300)."""
    L, m = 100, 512
    W = b.Mpo(b.MODEL_HUBBARD, L, (1.0, 0.0)).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [2, 1] * (L // 2)), None, None,
                               L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 14, 1e-10, b.update_opts(m, prec="tf32x3"),
                         final_prec="fp64", switch_tol=1e-7)
    st.close()
    e0 = exact.free_fermion_energy(L, L // 2, L // 2)
    assert abs(e0 - (-126.6023783108)) < 1e-9
    rel = (rep["energy"] - e0) / abs(e0)
    print("U=0 Hubbard L=100 m=%d: E = %.10f (%d sweeps, %.1f s), rel. error %.2e; paper %.2e"
          % (m, rep["energy"], rep["sweeps"], rep["seconds"][-1], rel,
             (-126.602376 - e0) / abs(e0)))
    assert rep["energy"] >= e0 - 1e-10 * abs(e0)
    assert rel < 2e-6                               # measured: 8.3e-7 at m = 512
