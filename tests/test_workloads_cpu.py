"""The seeded input recipe (no GPU): the unit conversions of the pair-plasma
setups and the properties of the generated inputs that both the oracle and the
CUDA path are fed.

Units are Gaussian with dx = dt = 1: the plasma frequency of the total density
n0 (both species) is omega_p^2 = 4 pi n0 q^2 / m; the magnetisation is
sigma = B0^2 / (4 pi n0 m c^2); the plasma beta is n0 k T / (B0^2 / 8 pi) with
k T = theta m c^2."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_15939_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("ppc,d_e", [(16, 5.0), (32, 5.0), (64, 10.0)])
def test_pair_units_follow_the_definitions(ppc, d_e):
    u = W.PairUnits(0.45, d_e, ppc)
    n0 = 2 * ppc                                  # both species, per unit cell volume
    assert u.omega_p == pytest.approx(0.45 / d_e)  # omega_p = c / d_e
    assert 4 * math.pi * n0 * u.q ** 2 / 1.0 == pytest.approx(u.omega_p ** 2, rel=1e-14)
    for sigma in (0.1, 0.5, 1.0):
        b0 = u.b0_from_sigma(sigma)
        assert b0 ** 2 / (4 * math.pi * n0 * 0.45 ** 2) == pytest.approx(sigma, rel=1e-14)
    for beta, theta in ((1e3, 0.3), (2.0, 0.05)):
        b0 = u.b0_from_beta(beta, theta)
        assert n0 * theta * 0.45 ** 2 / (b0 ** 2 / (8 * math.pi)) == pytest.approx(beta, rel=1e-14)
        assert u.b0_from_sigma(2 * theta / beta) == pytest.approx(b0, rel=1e-14)  # sigma = 2 theta / beta


def test_uniform_plasma_is_seeded_and_well_formed():
    n = (8, 6, 4)
    a = W.uniform_plasma(n, 5, seed=3, uth=0.2, q=0.05)
    b = W.uniform_plasma(n, 5, seed=3, uth=0.2, q=0.05)
    c = W.uniform_plasma(n, 5, seed=4, uth=0.2, q=0.05)
    assert all(np.array_equal(x["x"], y["x"]) and np.array_equal(x["u"], y["u"]) for x, y in zip(a, b))
    assert not np.array_equal(a[0]["x"], c[0]["x"])
    ids = np.concatenate([d["id"] for d in a])
    assert len(a) == 2 and len(ids) == 2 * 5 * 8 * 6 * 4 and len(np.unique(ids)) == len(ids)
    assert [d["q"] for d in a] == [-0.05, 0.05]
    for d in a:
        assert np.all(d["x"] >= 0) and np.all(d["x"] < np.asarray(n, dtype=float))
    flat = W.uniform_plasma((8, 6, 1), 5, seed=3, ignorable=2)
    assert np.all(flat[0]["x"][:, 2] == 0.5)


def test_host_load_into_caller_arrays_matches_the_recipe():
    """The chunked host load fills caller arrays: positions in the box (2D:
    the ignorable coordinate at 0.5), ids id_base + 0..n-1, momenta with the
    recipe's variance theta c^2 per component (no noise here)."""
    w = W.scaled(W.SUITE["keb3d_128_fp32"], (16, 16, 16), ppc=8)
    npart = w.ppc * 16 ** 3
    x = np.empty((npart, 3))
    u = np.empty((npart, 3))
    ids = np.empty(npart, dtype=np.uint32)
    W.host_maxwellian_into(w, 5, x, u, ids, id_base=100, chunk=1000)
    assert np.all(x >= 0) and np.all(x < 16)
    assert np.array_equal(ids, np.arange(100, 100 + npart, dtype=np.uint32))
    var = w.theta * w.c ** 2
    assert abs(u.var() - var) < 5 * var * math.sqrt(2.0 / u.size)
    w2 = W.scaled(W.SUITE["leaky2d_2048_fp32"], (32, 32, 1), ppc=4)
    x2 = np.empty((4 * 32 * 32, 3))
    W.host_maxwellian_into(w2, 5, x2, np.empty_like(x2), np.empty(len(x2), dtype=np.uint32))
    assert np.all(x2[:, 2] == 0.5)


def test_random_phase_perturbation_is_divergence_free_with_the_asked_rms():
    """The leaky box's in-plane dB comes from a vector potential, so its Yee
    divergence vanishes, and its rms is the asked amplitude."""
    n = (64, 64, 1)
    B = W.random_phase_dB(n, seed=2, amplitude=0.7)
    # B_x at (i, j+1/2) and B_y at (i+1/2, j): the divergence sits at the cell centre (i+1/2, j+1/2)
    div = (np.roll(B[0], -1, axis=2) - B[0]) + (np.roll(B[1], -1, axis=1) - B[1])
    assert np.abs(div).max() < 1e-12
    rms = math.sqrt((B[0] ** 2 + B[1] ** 2).mean())
    assert rms == pytest.approx(0.7, rel=1e-12)
