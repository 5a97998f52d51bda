"""Pins of the oracle's counter-based generator (Philox4x32-10)."""
import os

import numpy as np

import oracle as O
from conftest import GOLDEN


def kat_vectors():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, out in kat_vectors():
        assert list(O.philox(ctr, key)) == out


def test_mv_charge_moments():
    # MV charges: independent Gaussians of variance (g^2 mu a)^2 / Ns per color
    n, ns, g = 64, 4, 0.8
    rho = O.mv_charges(n, ns, g, 99, 1, 2)
    var = g * g / ns
    assert abs(rho.mean()) < 5 * np.sqrt(var / rho.size)
    assert abs(rho.var() / var - 1) < 5 * np.sqrt(2.0 / rho.size)
    c = np.corrcoef(rho.T)
    assert np.abs(c - np.eye(8)).max() < 5 / np.sqrt(n * n)
    # different sheets / nuclei draw from different counters
    assert not np.allclose(rho, O.mv_charges(n, ns, g, 99, 1, 3))
    assert not np.allclose(rho, O.mv_charges(n, ns, g, 99, 0, 2))
