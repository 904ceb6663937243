"""Energies the paper prints, pinned against the oracle's closed forms (CPU)."""
import json
import os

from oracle import exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_free_fermion_reference_energy():
    """Sec. VII B 4: the printed reference energy is a converged DMRG value,
    so the exact open-chain energy lies below it, within the accuracy of an
    m = 1200 MPS (here 2.3e-6 absolute).  A periodic chain (-127.28), spinless
    fermions or another hopping normalisation would miss by far more."""
    with open(os.path.join(GOLDEN, "free_fermions_l100.json")) as f:
        g = json.load(f)
    e = exact.free_fermion_energy(g["L"], g["n_up"], g["n_dn"])
    ref = g["E0_reference"]
    assert e <= ref
    assert ref - e < 1e-7 * abs(ref)
