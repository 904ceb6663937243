"""The C ABI library loads, exports every declared symbol, and its host-side
layout functions follow the documented canonical order (CPU only, no CUDA call)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(dmrg3s_\w+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def b():
    from paper_1501_05504_gb300 import _build, binding
    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    return binding


def test_library_exports_every_declared_symbol(b):
    names = _declared()
    assert len(names) >= 10
    L = b.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert set(names) <= exported


def test_status_strings(b):
    L = b.lib()
    assert L.dmrg3s_status_string(0) == b"ok"
    assert b"charges" in L.dmrg3s_status_string(3)


def _xxz_site(m_left=30, m_right=34, seed=1):
    rng = si.rng_for(seed)
    left = si.gaussian_bond(m_left, (1,), (2.0,), (2,), (3,))
    right = si.gaussian_bond(m_right, (0,), (2.0,), (2,), (3,))
    return rng, left, right


def test_site_block_table_matches_canonical_order(b):
    rng, left, right = _xxz_site()
    spec = si.random_site(rng, si.XXZ_QP, left, right)
    s = b.Site(spec["qp"], b.Bond.from_neutral(left), b.Bond.from_neutral(right))
    tab = s.blocks()
    keys = si.site_block_keys(si.XXZ_QP, left, right)
    assert [tuple(int(x) for x in r[:3]) for r in tab] == keys
    off = 0
    for r in tab:
        s_, i, j, o, rows, cols = (int(x) for x in r)
        assert o == off and rows == left["dim"][i] and cols == right["dim"][j]
        off += rows * cols
    assert s.size() == off


def test_env_block_table_matches_canonical_order(b):
    rng, left, right = _xxz_site()
    e = b.Env(si.XXZ_T, b.Bond.from_neutral(left))
    tab = e.blocks()
    keys = si.env_block_keys(si.XXZ_T, left, left)
    assert [tuple(int(x) for x in r[:3]) for r in tab] == keys
    assert e.size() == int(sum(r[4] * r[5] for r in tab))


def test_hubbard_two_charges_block_table(b):
    left, right = si.central_bonds("hubbard_l64_m1024_u1u1", m=60)
    # the physical charges move (N, 2Sz) by the local state's charge
    s = b.Site(si.HUB_QP, b.Bond.from_neutral(left), b.Bond.from_neutral(left))
    keys = si.site_block_keys(si.HUB_QP, left, left)
    assert [tuple(int(x) for x in r[:3]) for r in s.blocks()] == keys


def test_expanded_bond_follows_documented_rule(b):
    rng, left, right = _xxz_site()
    bond = b.Bond.from_neutral(right)
    for include_base in (False, True):
        fused = b.expanded_bond(bond, si.XXZ_T, include_base)
        want = {}
        if include_base:
            for q, dm in zip(right["q"], right["dim"]):
                want[tuple(q)] = want.get(tuple(q), 0) + int(dm)
        for t in si.XXZ_T:
            for q, dm in zip(right["q"], right["dim"]):
                k = tuple(q + t)
                want[k] = want.get(k, 0) + int(dm)
        keys = sorted(want)
        assert [tuple(int(x) for x in r) for r in fused.q] == keys
        assert list(fused.dim) == [want[k] for k in keys]


def test_dense_expanded_bond_is_w_times_m(b):
    bond = b.Bond(np.zeros((1, 0), dtype=np.int32), [7])
    fused = b.expanded_bond(bond, np.zeros((5, 0), dtype=np.int32), True)
    assert list(fused.dim) == [42]


@pytest.mark.parametrize("bad", ["unsorted", "zero_dim", "dense_two_sectors"])
def test_malformed_bonds_are_rejected_on_the_host(b, bad):
    if bad == "unsorted":
        bond = b.Bond(np.array([[2], [0]]), [3, 4])
        want = 3
    elif bad == "zero_dim":
        bond = b.Bond(np.array([[0], [2]]), [3, 0])
        want = 1
    else:
        bond = b.Bond(np.zeros((2, 0), dtype=np.int32), [3, 4])
        want = 3
    qp = si.XXZ_QP[:, :bond.nsym] if bond.nsym else np.zeros((2, 0))
    s = b.Site(qp, bond, bond)
    c = s._c()
    n = ctypes.c_int64()
    assert b.lib().dmrg3s_site_size(ctypes.byref(c), ctypes.byref(n)) == want


def test_entry_points_reject_null_context(b):
    assert b.lib().dmrg3s_apply_heff(None, None, None, None, None, None, 0, None) == 1
    assert b.lib().dmrg3s_destroy(None) == 1
