"""The library's host-side H_eff plan, through dmrg3s_heff_cost (no device
needed): its algorithmic flop count equals an independent count of the block
products and MPO terms written in Python from the selection rules."""
import numpy as np
import pytest

import bench
import seeded_inputs as si


@pytest.fixture(scope="module")
def b():
    from paper_1501_05504_gb300 import binding
    return binding


def _structures(b, W, left, right):
    qp = W.qp
    L = b.Env(W.tl, b.Bond.from_neutral(left))
    R = b.Env(W.tr, b.Bond.from_neutral(right))
    A = b.Site(qp, b.Bond.from_neutral(left), b.Bond.from_neutral(right))
    return L, R, A


@pytest.mark.parametrize("name,model,nsites,params,site,m", [
    ("xxz_l100_m512_u1", "MODEL_XXZ", 100, (1.0, 1.0), 50, 512),
    ("xxz_l100_m512_u1", "MODEL_XXZ", 100, (1.0, 0.3), 50, 96),
    ("hubbard_l64_m1024_u1u1", "MODEL_HUBBARD", 64, (1.0, 8.0), 32, 256),
])
def test_heff_cost_matches_independent_count(b, name, model, nsites, params, site, m):
    W = b.Mpo(getattr(b, model), nsites, params).site(site)
    left, right = si.central_bonds(name, m)
    L, R, A = _structures(b, W, left, right)
    flops, nbytes = b.dmrg3s_heff_cost(L, W, R, A)
    want = bench.heff_flops(W.qp.astype(np.int64), W.tl.astype(np.int64), W.W, left, right)
    assert flops == want
    assert nbytes > 0


def test_heff_cost_rejects_mismatched_structures(b):
    W = b.Mpo(b.MODEL_XXZ, 100, (1.0, 1.0)).site(50)
    left, right = si.central_bonds("xxz_l100_m512_u1", 64)
    L, R, A = _structures(b, W, left, right)
    with pytest.raises(b.Dmrg3sError):
        b.dmrg3s_heff_cost(R, W, L, A)       # environments on the wrong bonds
