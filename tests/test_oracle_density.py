"""Pins of the oracle's feature density and density loss (Eq. 4-9)."""
import numpy as np
import pytest

from oracle import apmgsrn as ap


def _eye_G(m):
    G = np.zeros((m, 3, 4))
    for d in range(3):
        G[:, d, d] = 1.0
    return G


def test_density_at_centre_with_identity_grids_is_M():
    # Eq. 7 with G_i = I at x = 0: every term is det(I) exp(0) = 1.
    for m in (1, 4, 64):
        assert ap.feature_density(_eye_G(m), np.zeros((1, 3)))[0] == float(m)


def test_density_scales_with_determinant():
    # Sec. 4.2: shrinking a grid by s raises its feature density by det = s^3.
    for s in (0.5, 2.0, 3.0):
        G = _eye_G(3) * s
        assert abs(ap.feature_density(G, np.zeros((1, 3)))[0] - 3 * s ** 3) < 1e-12


def test_flat_top_approaches_box_counts():
    # As p grows, Eq. 7 tends to Eq. 5 (det-weighted box count) and, for identity
    # grids, to Eq. 4 (number of grids containing x).  Points kept off the faces.
    r = np.random.default_rng(0)
    G = r.normal(0, 0.2, size=(6, 3, 4))
    for d in range(3):
        G[:, d, d] += 1.0
    x = r.uniform(-1.3, 1.3, size=(400, 3))
    u = ap.local_coords(G, x)
    keep = np.all(np.abs(np.abs(u) - 1.0) > 0.05, axis=(1, 2))
    keep &= np.all(np.abs(np.abs(x) - 1.0) > 0.05, axis=1)   # identity grids: u = x
    x, u = x[keep], u[keep]
    inside = ap.inside_mask(u)
    det = np.linalg.det(G[:, :, :3])
    box5 = inside @ det
    np.testing.assert_allclose(ap.feature_density(G, x, p=200), box5, atol=1e-6)
    box4 = ap.inside_mask(ap.local_coords(_eye_G(6), x)).sum(axis=1)
    np.testing.assert_allclose(ap.feature_density(_eye_G(6), x, p=200), box4, atol=1e-6)


def test_scaled_density_sums_to_one_and_constant_error_gives_zero_loss():
    r = np.random.default_rng(1)
    G = _eye_G(5) + r.normal(0, 0.05, size=(5, 3, 4))
    x = r.uniform(-1, 1, size=(300, 3))
    rho = ap.feature_density(G, x)
    t = ap.density_terms(rho, np.full(300, 0.37))
    assert abs(t["rho_s"].sum() - 1.0) < 1e-12
    # Sec. 4.2: error equal to the average leaves the target density unchanged
    # (k = hbar/(h+eps) = 1 - O(eps)), so the KL term vanishes.
    np.testing.assert_allclose(t["k"], 1.0, atol=1e-7)
    np.testing.assert_allclose(t["rho_star"], t["rho_s"] + 1e-8, rtol=1e-6)
    assert abs(t["L_den"]) < 1e-9


def test_higher_relative_error_raises_target_density():
    # Sec. 4.2: the target grows where the error is above average.
    rho = np.array([1.0, 1.0, 1.0, 1.0])
    t = ap.density_terms(rho, np.array([0.1, 0.1, 0.1, 10.0]))
    assert t["rho_star"][3] > t["rho_s"][3] > t["rho_star"][0]


def test_brute_force_high_precision_tiny_case():
    # Eq. 7-9 evaluated point by point, grid by grid, at 50 digits with mpmath.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    r = np.random.default_rng(2)
    N, M, p, eps = 4, 2, 10, 1e-8
    G = _eye_G(M) + r.normal(0, 0.15, size=(M, 3, 4))
    x = r.uniform(-1.2, 1.2, size=(N, 3))
    h = r.uniform(0.01, 1.0, size=N)
    rho = []
    for n in range(N):
        acc = mp.mpf(0)
        for i in range(M):
            A = mp.matrix([[mp.mpf(G[i, a, b]) for b in range(3)] for a in range(3)])
            s = mp.mpf(0)
            for d in range(3):
                ud = sum(mp.mpf(G[i, d, e]) * mp.mpf(x[n, e]) for e in range(3)) + mp.mpf(G[i, d, 3])
                s += ud ** (2 * p)
            acc += mp.det(A) * mp.e ** (-s)
        rho.append(acc)
    S = sum(rho)
    hbar = sum(mp.mpf(v) for v in h) / N
    L = mp.mpf(0)
    for n in range(N):
        rs = rho[n] / S
        k = hbar / (mp.mpf(h[n]) + eps)
        star = mp.e ** (k * mp.log(rs + eps))
        L += star * (mp.log(star) - mp.log(rs + eps))
    L /= N
    got = ap.loss_density(G, x, h, p=p, eps=eps)
    assert abs(got - float(L)) <= 1e-12 * max(1.0, abs(float(L)))
    np.testing.assert_allclose(ap.feature_density(G, x), [float(v) for v in rho], rtol=1e-13)
