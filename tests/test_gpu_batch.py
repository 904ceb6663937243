"""Batched chains on the GPU: several independent XXZ chains solved together,
every contraction stage of their local updates one launch over all of them
(dmrg3s_local_update_batch, dmrg3s_sweep_batch), Sec. V applied per chain.

* One batched step equals one dmrg3s_local_update per chain (twin states,
  mixed directions and lengths): to rounding in FP64, over 16 steps, and the
  whole states at the end (overlap 1 to 1e-10); in 3xTF32 to the product's
  own tolerance (1e-6) over the first 6 steps (the merged launch groups the
  split-K partial sums of stage 3 differently, and later steps amplify such
  differences through the choice among nearly degenerate states at the
  truncation).
* The chains of the batched-chain workload (seed 1005) that exact
  diagonalisation reaches (L <= 20), with three short chains beside them,
  swept as one batch: every energy within 1e-9 of sparse exact
  diagonalisation, in FP64 and with the 3xTF32 -> FP64 precision ladder.
* dE/dJ and dE/dDelta of every batched chain (dmrg3s_energy_grad): the
  homogeneity identity J dE/dJ = E, central finite differences (h = 1e-4) of
  the exact energies, and the Hellmann-Feynman value of the oracle's MPO-entry
  gradients on the chain's own MPS.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import seeded_inputs as si  # noqa: E402
from oracle import contract, exact  # noqa: E402
from parity import site_to_dense  # noqa: E402

E_TOL = 1e-9
FD_H = 1e-4


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


def _neel(b, ctx, L, J, delta):
    W = b.Mpo(b.MODEL_XXZ, L, (J, delta)).sites()
    spec = si.product_state_sites(si.XXZ_QP, [0, 1] * (L // 2))
    return b.dmrg3s_state_create(ctx, W, [b.site_from_neutral(x) for x in spec], None, None, L - 1)


def _ed(L, J, delta):
    return exact.ed_sparse_spin(L, [(i, i + 1, J, J * delta) for i in range(L - 1)])


def _chains():
    """The ED-sized chains of the batched workload and three short ones."""
    sub = [c for c in si.batch_xxz_chains() if c["L"] <= 20]
    extra = [{"L": 8, "J": 1.0, "Delta": 0.6, "m_max": 16},
             {"L": 10, "J": 1.0, "Delta": 1.4, "m_max": 32},
             {"L": 12, "J": 1.0, "Delta": 1.0, "m_max": 64}]
    return sub + extra


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 1e-6)])
def test_batch_step_equals_single_updates(b, ctx, prec, tol):
    specs = [(8, 0.7, 16), (10, 1.2, 32), (12, 0.9, 24), (6, 1.0, 8)]
    A = [_neel(b, ctx, L, 1.0, d) for L, d, _ in specs]
    B = [_neel(b, ctx, L, 1.0, d) for L, d, _ in specs]
    opts = [b.update_opts(m, tol=1e-12, prec=prec) for _, _, m in specs]
    pos = [L - 1 for L, _, _ in specs]
    dirs = [-1] * len(specs)
    for step in range(16 if prec == "fp64" else 6):
        alphas = [1e-2 * (k + 1) * 0.9 ** step for k in range(len(specs))]
        ia = [b.dmrg3s_local_update(A[k], dirs[k], alphas[k], opts[k]) for k in range(len(specs))]
        ib = b.dmrg3s_local_update_batch(B, dirs, alphas, opts)
        for k in range(len(specs)):
            for key in ("lambda", "energy_after"):
                assert abs(ia[k][key] - ib[k][key]) <= tol * abs(ia[k][key]), (step, k, key)
            assert ia[k]["new_bond_dim"] == ib[k]["new_bond_dim"], (step, k)
            assert abs(ia[k]["lanczos_iters"] - ib[k]["lanczos_iters"]) <= 1, (step, k)
        for k, (L, _, _) in enumerate(specs):   # bounce between the chain's ends
            pos[k] += dirs[k]
            if pos[k] == 0 or pos[k] == L - 1:
                dirs[k] = -dirs[k]
    # the wavefunctions agree (the singular vectors of a truncation are fixed
    # up to sign, a gauge freedom on the bond, so the states are compared,
    # not the tensors)
    for k, (L, _, _) in enumerate(specs if prec == "fp64" else []):
        assert A[k].centre()[0] == B[k].centre()[0]
        pa, pb = _dense_state(b, A[k], L), _dense_state(b, B[k], L)
        ov = abs(float(pa @ pb)) / (np.linalg.norm(pa) * np.linalg.norm(pb))
        assert 1.0 - ov <= 1e-10, (k, ov)
    for st in A + B:
        st.close()


def _dense_state(b, st, L):
    """The MPS of a state contracted into one vector (small chains only)."""
    psi = np.ones((1, 1))
    for i in range(L):
        A = site_to_dense(b, st.site(i))           # (d, left, right)
        psi = np.einsum("pa,sab->psb", psi, A).reshape(-1, A.shape[2])
    return psi.reshape(-1)


def _oracle_dE_ddelta(b, st, L, J, delta):
    """Hellmann-Feynman dE/dDelta from the oracle's MPO-entry gradients on the
    MPS read back from the device."""
    W = b.Mpo(b.MODEL_XXZ, L, (J, delta)).sites()
    W1 = b.Mpo(b.MODEL_XXZ, L, (J, delta + 1.0)).sites()
    A = [site_to_dense(b, st.site(i)) for i in range(L)]
    one = np.ones((1, 1, 1))
    Ls, Rs = [one], [one]
    for i in range(L - 1):
        Ls.append(contract.left_env(Ls[-1], W[i].W, A[i]))
    for i in range(L - 1, 0, -1):
        Rs.append(contract.right_env(Rs[-1], W[i].W, A[i]))
    Rs = Rs[::-1]
    idw = np.eye(2).reshape(2, 2, 1, 1)
    N = one
    for i in range(L):
        N = contract.left_env(N, idw, A[i])
    num = sum(float(np.sum(contract.mpo_gradient(Ls[i], Rs[i], A[i]) * (W1[i].W - W[i].W)))
              for i in range(L))
    return num / float(N[0, 0, 0])


@pytest.fixture(scope="module")
def reference():
    """Exact energies of every test chain at Delta and Delta +- h."""
    out = []
    for c in _chains():
        L, J, d = c["L"], c["J"], c["Delta"]
        out.append({"E": _ed(L, J, d), "Ep": _ed(L, J, d + FD_H), "Em": _ed(L, J, d - FD_H)})
    return out


def test_sweep_batch_reaches_exact_energies_with_gradients(b, ctx, reference):
    chains = _chains()
    states = [_neel(b, ctx, c["L"], c["J"], c["Delta"]) for c in chains]
    opts = [b.update_opts(c["m_max"], tol=1e-12) for c in chains]
    reps = b.dmrg3s_sweep_batch(states, b.alpha_rule(1e-2), 14, 1e-12, opts)
    for k, (c, r, ref) in enumerate(zip(chains, reps, reference)):
        assert r["converged"], (k, c)
        assert abs(r["energy"] - ref["E"]) <= E_TOL * abs(ref["E"]), (k, c, r["energy"], ref["E"])
        E, dE = b.dmrg3s_energy_grad(states[k], b.MODEL_XXZ, (c["J"], c["Delta"]))
        assert abs(E - ref["E"]) <= E_TOL * abs(ref["E"]), k
        # E is homogeneous of degree one in J at fixed Delta
        assert abs(c["J"] * dE[0] - E) <= 1e-10 * abs(E), k
        fd = (ref["Ep"] - ref["Em"]) / (2 * FD_H)
        assert abs(dE[1] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, dE[1], fd)
    # Hellmann-Feynman from the oracle's gradients on two of the chains' MPS
    for k in (0, len(chains) - 1):
        c = chains[k]
        _, dE = b.dmrg3s_energy_grad(states[k], b.MODEL_XXZ, (c["J"], c["Delta"]))
        hf = _oracle_dE_ddelta(b, states[k], c["L"], c["J"], c["Delta"])
        assert abs(dE[1] - hf) <= 1e-10 * abs(hf), (k, dE[1], hf)
    for st in states:
        st.close()


def test_sweep_batch_matches_single_sweeps(b, ctx):
    chains = _chains()[-3:] + _chains()[:1]
    sa = [_neel(b, ctx, c["L"], c["J"], c["Delta"]) for c in chains]
    sb = [_neel(b, ctx, c["L"], c["J"], c["Delta"]) for c in chains]
    opts = [b.update_opts(c["m_max"], tol=1e-12) for c in chains]
    single = [b.dmrg3s_sweep(sa[k], b.alpha_rule(1e-2), 10, 1e-11, opts[k]) for k in range(len(chains))]
    batch = b.dmrg3s_sweep_batch(sb, b.alpha_rule(1e-2), 10, 1e-11, opts)
    for k, c in enumerate(chains):
        s1, s2 = single[k], batch[k]
        assert s1["converged"] and s2["converged"], k
        # once converged, the sweep-to-sweep change and the alpha rule's
        # branches are decided by rounding: compare the first sweep exactly
        # and the end point to the energy tolerance
        assert abs(s1["sweeps"] - s2["sweeps"]) <= 1, k
        assert abs(s2["energies"][0] - s1["energies"][0]) <= 1e-10 * abs(s1["energies"][0]), k
        assert abs(s2["energy"] - s1["energy"]) <= 1e-10 * abs(s1["energy"]), k
        n1 = 2 * (c["L"] - 1)
        np.testing.assert_allclose(s2["alphas"][:n1 // 2], s1["alphas"][:n1 // 2], rtol=1e-9, atol=0)
    for st in sa + sb:
        st.close()


def test_sweep_batch_mixed_precision_ladder(b, ctx, reference):
    chains = _chains()
    states = [_neel(b, ctx, c["L"], c["J"], c["Delta"]) for c in chains]
    opts = [b.update_opts(c["m_max"], tol=1e-12, prec="tf32x3") for c in chains]
    reps = b.dmrg3s_sweep_batch(states, b.alpha_rule(1e-2), 16, 1e-12, opts, final_prec="fp64",
                                switch_tol=1e-7)
    for k, (c, r, ref) in enumerate(zip(chains, reps, reference)):
        assert r["converged"], (k, c)
        assert r["bulk_sweeps"] >= 1, k
        assert abs(r["energy"] - ref["E"]) <= E_TOL * abs(ref["E"]), (k, c, r["energy"], ref["E"])
    for st in states:
        st.close()


def test_batch_rejects_bad_batches(b, ctx):
    s1 = _neel(b, ctx, 6, 1.0, 1.0)
    s2 = _neel(b, ctx, 6, 1.0, 1.0)
    o = b.update_opts(8, svd="gesvd")
    with pytest.raises(b.Dmrg3sError):       # a state twice
        b.dmrg3s_local_update_batch([s1, s1], [-1, -1], [0.01, 0.01], o)
    with pytest.raises(b.Dmrg3sError):       # different SVD methods
        b.dmrg3s_local_update_batch([s1, s2], [-1, -1], [0.01, 0.01],
                                    [o, b.update_opts(8, svd="jacobi")])
    other = b.dmrg3s_create(0, 1 << 26)
    s3 = _neel(b, other, 6, 1.0, 1.0)
    with pytest.raises(b.Dmrg3sError):       # two contexts
        b.dmrg3s_local_update_batch([s1, s3], [-1, -1], [0.01, 0.01], o)
    for st in (s1, s2, s3):
        st.close()
    other.close()
