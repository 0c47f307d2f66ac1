"""Pins of the seeded input generators (host code shared by the oracle and the GPU path)."""
import os

import numpy as np
import pytest
from scipy import integrate, stats

import paper_1205_2933_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox-4x32-10 against the published known-answer vectors (SC'11 / Random123)."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert I.philox(w[0:4], w[4:6]) == w[6:10]
        n += 1
    assert n == 3


def test_uniform_and_gauss_moments():
    u = I.uniform(200000, 11, 99)
    assert 0.0 < u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    g = I.gauss_complex((100000,), 12, 99)
    assert abs(g.real.mean()) < 0.01 and abs(g.imag.var() - 1.0) < 0.02
    # deterministic and independent of call order
    assert np.array_equal(I.gauss_complex((10,), 12, 99), g[:10])


@pytest.mark.parametrize("bp", [0.7, 2.5])
def test_kennedy_pendleton_distribution(bp):
    """h0 must follow sqrt(1 - h0^2) exp(bp h0) on [-1, 1] (chi-square, 40 bins)."""
    h = I.kp_samples(200000, bp, 5)
    assert h.min() >= -1.0 and h.max() <= 1.0
    edges = np.linspace(-1, 1, 41)
    obs, _ = np.histogram(h, edges)
    dens = lambda x: np.sqrt(max(0.0, 1 - x * x)) * np.exp(bp * x)
    Z = integrate.quad(dens, -1, 1)[0]
    exp = np.array([integrate.quad(dens, a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) / Z * h.size
    keep = exp > 5
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    p = stats.chi2.sf(chi2, keep.sum() - 1)
    assert p > 1e-4, (chi2, p)


def _unitarity(U):
    return np.abs(np.einsum("...ab,...cb->...ac", U, U.conj()) - np.eye(3)).max()


def test_epsilon_links_su3():
    U = I.epsilon_links((4, 4, 4, 4), 0.3, 1)
    assert U.shape == (4, 4, 4, 4, 4, 3, 3)
    assert _unitarity(U) < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # small eps: U = 1 + O(eps)
    U0 = I.epsilon_links((2, 2, 2, 2), 1e-6, 1)
    assert np.abs(U0 - np.eye(3)).max() < 1e-5


def test_heatbath_plaquette_beta6():
    """Sanity check, not parity: thermalised plaquette near the beta = 6.0 literature value."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "plaquette_beta6.txt")):
        if line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    U = I.heatbath_links((8, 8, 8, 8), vals["beta"], 60, 5, cache=False)
    assert _unitarity(U) < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    assert abs(I.plaquette(U, (8, 8, 8, 8)) - vals["plaquette"]) < vals["tolerance"]


def test_heatbath_deterministic():
    a = I.heatbath_links((4, 4, 4, 4), 5.9, 3, 7, cache=False)
    b = I.heatbath_links((4, 4, 4, 4), 5.9, 3, 7, cache=False)
    assert np.array_equal(a, b)


def test_wall_sources():
    P = I.point_sources((4, 4, 4, 4), 6)
    assert P.shape == (12, 6, 4, 4, 4, 4, 4, 3)
    # spin 0 (chirality +) sits at s = Ls-1, spin 2 (chirality -) at s = 0
    assert P[0, 5, 0, 0, 0, 0, 0, 0] == 1 and np.count_nonzero(P[0]) == 1
    assert P[6, 0, 0, 0, 0, 0, 2, 0] == 1 and np.count_nonzero(P[6]) == 1
    Z = I.z2_source((4, 4, 4, 4), 6, 201)
    assert set(np.unique(np.abs(Z[0, ..., 2:, :]))) == {1.0}
    assert np.count_nonzero(Z[1:5]) == 0
