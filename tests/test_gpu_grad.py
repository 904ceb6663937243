"""GPU parity of the MPO-entry gradient G_i = d<Psi|H|Psi>/dW_i against the FP64 oracle.

<Psi|H|Psi> is linear in every W_i (the network of Sec. II), so G_i is that
network with W_i taken out, and sum_i <G_i, dW_i/dtheta> / <Psi|Psi> is the
Hellmann-Feynman derivative of the energy.  Checks:
  * one site: element-wise against the oracle's contraction on identical inputs;
  * a whole converged state: the oracle's G_i on the MPS read back from the
    device, <G_i, W_i> = <Psi|H|Psi> at every site, the homogeneity identity
    J dE/dJ = E of the XXZ chain, and the free-fermion value of dE/dDelta at
    Delta = 0 (Wick's theorem).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import seeded_inputs as si  # noqa: E402
from oracle import contract, io  # noqa: E402
from parity import FP64_TOL, problem, rel_err, site_to_dense  # noqa: E402

CASES = [("dense", 51, {}), ("u1", 52, {}), ("u1u1", 53, {}),
         ("u1", 54, {"m_left": 9, "m_right": 7}), ("xxz_l100_m512_u1", 1002, {})]


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


@pytest.mark.parametrize("kind,seed,kw", CASES)
def test_site_gradient_matches_oracle(b, ctx, kind, seed, kw):
    pb = problem(kind, seed, **kw)
    gL, gW, gR = b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]), b.env_from_neutral(pb["R"])
    gM = b.site_from_neutral(pb["A"])
    W = pb["W"]["W"]
    G = torch.full((W.size,), float("nan"), dtype=torch.float64, device="cuda")
    b.dmrg3s_mpo_grad_site(ctx, gL, gW, gR, gM, G)
    b.dmrg3s_sync(ctx)
    ref = contract.mpo_gradient(io.env_dense(pb["L"]), io.env_dense(pb["R"]), io.site_dense(pb["A"])[0])
    got = G.cpu().numpy().reshape(W.shape)
    assert np.isfinite(got).all()
    assert rel_err(got, ref) < FP64_TOL
    # linearity of <M|H_eff|M> in W: <G, W> is the expectation value
    L, R, M = io.env_dense(pb["L"]), io.env_dense(pb["R"]), io.site_dense(pb["A"])[0]
    e = contract.expectation(L, W, R, M)
    assert abs(float(np.sum(got * W)) - e) <= 1e-12 * np.abs(got * W).sum()


def test_site_gradient_rejects_mismatched_env(b, ctx):
    pb = problem("u1", 54, m_left=9, m_right=7)
    gL, gW, gR = b.env_from_neutral(pb["L"]), b.mpo_from_neutral(pb["W"]), b.env_from_neutral(pb["R"])
    gM = b.site_from_neutral(pb["A"])
    G = torch.zeros(pb["W"]["W"].size, dtype=torch.float64, device="cuda")
    with pytest.raises(b.Dmrg3sError):
        b.dmrg3s_mpo_grad_site(ctx, gR, gW, gL, gM, G)     # environments swapped


# ---- whole state ----------------------------------------------------------------------


def _xxz_ground_state(b, ctx, L, J, delta, m=64):
    W = b.Mpo(b.MODEL_XXZ, L, (J, delta)).sites()
    spec = si.product_state_sites(si.XXZ_QP, [0, 1] * (L // 2))
    st = b.dmrg3s_state_create(ctx, W, [b.site_from_neutral(x) for x in spec], None, None, L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 12, 1e-12, b.update_opts(m, tol=1e-12))
    return st, W, rep


def _oracle_state_gradients(b, st, W):
    """G_i of the oracle on the MPS read back from the device, and <Psi|Psi>."""
    n = len(W)
    A = [site_to_dense(b, st.site(i)) for i in range(n)]
    one = np.ones((1, 1, 1))
    Ls, Rs = [one], [one]
    for i in range(n - 1):
        Ls.append(contract.left_env(Ls[-1], W[i].W, A[i]))
    for i in range(n - 1, 0, -1):
        Rs.append(contract.right_env(Rs[-1], W[i].W, A[i]))
    Rs = Rs[::-1]
    G = [contract.mpo_gradient(Ls[i], Rs[i], A[i]) for i in range(n)]
    # <Psi|Psi> through the identity MPO
    idw = np.eye(2).reshape(2, 2, 1, 1)
    N = one
    for i in range(n):
        N = contract.left_env(N, idw, A[i])
    return G, float(N[0, 0, 0])


def test_state_gradient_matches_oracle_and_identities(b, ctx):
    L, J, delta = 12, 1.0, 0.7
    st, W, rep = _xxz_ground_state(b, ctx, L, J, delta)
    shapes = [w.W.shape for w in W]
    W1 = b.Mpo(b.MODEL_XXZ, L, (1.0, delta)).sites()
    W0 = b.Mpo(b.MODEL_XXZ, L, (0.0, delta)).sites()
    dW_dJ = [w1.W - w0.W for w1, w0 in zip(W1, W0)]
    G, dE_dJ, norm2 = b.dmrg3s_mpo_grad(st, dW_dJ, shapes)
    Go, norm_o = _oracle_state_gradients(b, st, W)
    assert abs(norm2 - norm_o) < 1e-12 * norm_o
    for i in range(L):
        assert rel_err(G[i], Go[i]) < 1e-11, i
    # <G_i, W_i> = <Psi|H|Psi> at every site (linearity in W_i)
    e_of_site = [float(np.sum(G[i] * W[i].W)) / norm2 for i in range(L)]
    assert max(e_of_site) - min(e_of_site) < 1e-11 * abs(rep["energy"])
    assert abs(e_of_site[0] - rep["energy"]) < 1e-9 * abs(rep["energy"])
    # homogeneity of degree one in J at fixed Delta: J dE/dJ = E
    assert abs(J * dE_dJ - e_of_site[0]) < 1e-11 * abs(e_of_site[0])
    # the same derivative from the oracle's gradients
    dE_o = sum(float(np.sum(g * d)) for g, d in zip(Go, dW_dJ)) / norm_o
    assert abs(dE_dJ - dE_o) < 1e-11 * abs(dE_o)
    st.close()


def test_state_gradient_xx_chain_free_fermions(b, ctx):
    """dE/dDelta at Delta = 0 equals J sum_i <Sz_i Sz_i+1> = -J sum_i G_{i,i+1}^2 (Wick)."""
    L, J = 12, 1.0
    st, W, rep = _xxz_ground_state(b, ctx, L, J, 0.0)
    shapes = [w.W.shape for w in W]
    W1 = b.Mpo(b.MODEL_XXZ, L, (J, 1.0)).sites()
    dW = [w1.W - w0.W for w1, w0 in zip(W1, W)]
    _, dE, _ = b.dmrg3s_mpo_grad(st, dW, shapes)
    # hopping J/2 (c+c + h.c.): modes k with J cos(pi k / (L+1)) < 0 are filled
    k = np.arange(L // 2 + 1, L + 1)
    i = np.arange(1, L + 1)
    phi = np.sqrt(2.0 / (L + 1)) * np.sin(np.pi * np.outer(k, i) / (L + 1))
    Gc = phi.T @ phi
    want = -J * sum(Gc[j, j + 1] ** 2 for j in range(L - 1))
    # first order in the error of the converged state (the same-MPS pin above is exact)
    assert abs(dE - want) < 1e-6 * abs(want)
    st.close()


def test_state_gradient_checks_length(b, ctx):
    st, W, _ = _xxz_ground_state(b, ctx, 4, 1.0, 1.0, m=4)
    shapes = [w.W.shape for w in W]
    with pytest.raises(ValueError):
        b.dmrg3s_mpo_grad(st, [np.zeros(1)] * 4, shapes)
    st.close()
