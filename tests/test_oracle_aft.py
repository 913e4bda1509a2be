"""Pins of the oracle's AFT tables (App. B, App. D, Eq. 13-14) and size logic."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import fse_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


@pytest.mark.parametrize("H", [[3], [7], [31], [1, 1], [2, 3], [7, 7], [1, 2, 1]])
def test_table_covers_harmonic_box_once(H):
    """Rows and their negatives partition the box prod_j [-H_j, H_j] (parity of cos/sin)."""
    tab = O.harmonic_table(H)
    assert tab.shape == ((O.u_tilde(H) + 1) // 2, len(H))
    assert np.all(tab[-1] == 0)
    seen = {}
    for row in tab:
        for sgn in (1, -1):
            key = tuple(int(x) for x in sgn * row)
            seen[key] = seen.get(key, 0) + 1
    box = list(itertools.product(*[range(-h, h + 1) for h in H]))
    assert set(seen) == set(box)
    for key, cnt in seen.items():
        assert cnt == (2 if all(k == 0 for k in key) else 1)


def test_table_d2_order():
    """d = 2: K~^2 = [k_2; 0] (App. B a)."""
    tab = O.harmonic_table([5])
    assert tab[:, 0].tolist() == [1, 2, 3, 4, 5, 0]


def test_table_d3_hand_worked():
    want = np.array([[int(a), int(b)] for a, b in _load("harmonics_d3_H1x1.txt")])
    np.testing.assert_array_equal(O.harmonic_table([1, 1]), want)


def test_unknown_counts_printed_in_paper():
    """2 n U~ reproduces every unknown count printed in Sec. 4."""
    for n, U, count, *_ in _load("unknown_counts.txt"):
        assert 2 * int(n) * int(U) == int(count)
    # U~ from the harmonic sets quoted there
    assert O.u_tilde([5]) == 11 and O.u_tilde([5, 5]) == 121 and O.u_tilde([7]) == 15


def test_sample_grid_phi2_fastest():
    S = [4, 3]
    T = O.sample_grid(S)
    for s in range(12):
        i2, i3 = s % 4, s // 4
        assert T[0, s] == pytest.approx(2 * math.pi * i2 / 4)
        assert T[1, s] == pytest.approx(2 * math.pi * i3 / 3)


@pytest.mark.parametrize("S,H", [([16], [7]), ([15], [7]), ([64], [31]), ([5], [2]),
                                 ([16, 16], [7, 7]), ([7, 5], [3, 2]), ([3, 3, 5], [1, 1, 2])])
def test_discrete_orthogonality(S, H):
    """Gamma^{-1} Gamma = I when S_j >= 2 H_j + 1 (Eq. D2, D3, Sec. 3.1 sampling rule)."""
    tab = O.harmonic_table(H)
    T = O.sample_grid(S)
    G = O.gamma(tab, T)
    Gi = O.gamma_inv(tab, T)
    np.testing.assert_allclose(Gi @ G, np.eye(G.shape[1]), atol=1e-13)


def test_aliasing_detected_below_nyquist():
    tab = O.harmonic_table([7])
    T = O.sample_grid([14])
    G, Gi = O.gamma(tab, T), O.gamma_inv(tab, T)
    assert np.abs(Gi @ G - np.eye(15)).max() > 0.5


@pytest.mark.parametrize("H,rho", [([7], [0.6180339887]), ([3, 2], [math.sqrt(2), math.sqrt(3)])])
def test_rotation_identity(H, rho):
    """H(phi~ - 2 pi rho) = H(phi~) R(rho) (Eq. 13)."""
    tab = O.harmonic_table(H)
    R = O.rotation(tab, np.array(rho))
    rng = np.random.default_rng(1)
    for _ in range(10):
        phi = rng.uniform(0, 2 * math.pi, len(H))
        lhs = O.basis_row(tab, phi - 2 * math.pi * np.array(rho))
        rhs = O.basis_row(tab, phi) @ R
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_round_trip_band_limited():
    """A band-limited function sampled on the grid is recovered exactly by Gamma^{-1}."""
    H, S = [3, 2], [8, 6]
    tab = O.harmonic_table(H)
    T = O.sample_grid(S)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(O.u_tilde(H))
    samples = np.array([O.basis_row(tab, T[:, s]) @ c for s in range(T.shape[1])])
    np.testing.assert_allclose(O.gamma_inv(tab, T) @ samples, c, atol=1e-13)


def test_nyquist_rule_enforced():
    from paper_2508_06302_gb300 import inputs as I
    with pytest.raises(ValueError):
        O.FSEProblem(I.chain(4), [10], [5], 16, [0.5])
