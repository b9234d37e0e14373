"""Pins of the oracle's encoder (Eq. 1-3) to facts the paper and the mathematics fix."""
import itertools

import numpy as np
import pytest

from oracle import apmgsrn as ap


def _rand_G(m, seed, std=0.05):
    r = np.random.default_rng(seed)
    G = r.normal(0, std, size=(m, 3, 4))
    for d in range(3):
        G[:, d, d] += 1.0
    return G


def test_identity_transform_maps_domain_onto_local_cube():
    # Sec. 4.1.1: local extents are [-1,1]^3; with G = I the global domain is the grid.
    G = np.zeros((3, 3, 4))
    for d in range(3):
        G[:, d, d] = 1.0
    x = np.random.default_rng(0).uniform(-1, 1, size=(50, 3))
    u = ap.local_coords(G, x)
    for i in range(3):
        np.testing.assert_array_equal(u[:, i, :], x)


def test_grid_corners_from_inverse_transform_map_back_to_extents():
    # Sec. 4.1.1: the global corners of grid i are G_i^{-1} applied to the local extents.
    G = _rand_G(4, 1, std=0.2)
    corners = np.array(list(itertools.product((-1.0, 1.0), repeat=3)))
    for i in range(4):
        full = np.eye(4)
        full[:3, :] = G[i]
        inv = np.linalg.inv(full)
        glob = (inv[:3, :3] @ corners.T).T + inv[:3, 3]
        u = ap.local_coords(G[i:i + 1], glob)[:, 0, :]
        np.testing.assert_allclose(u, corners, atol=1e-12)


def test_transform_rows_and_columns():
    # Eq. 1 element by element: u_r = sum_c G[r,c] x_c + G[r,3] (catches a transposed A).
    G = _rand_G(2, 2, std=0.5)
    x = np.array([[0.3, -0.7, 0.11]])
    u = ap.local_coords(G, x)
    for i in range(2):
        for r in range(3):
            ref = G[i, r, 0] * 0.3 + G[i, r, 1] * -0.7 + G[i, r, 2] * 0.11 + G[i, r, 3]
            assert abs(u[0, i, r] - ref) < 1e-15


@pytest.mark.parametrize("res", [2, 3, 5, 16])
def test_interp_exact_at_every_node(res):
    # Corner-aligned vertices (Sec. 4.1.1): node j at -1 + 2j/(R-1) returns the stored value.
    r = np.random.default_rng(res)
    Fi = r.normal(size=(res, res, res, 2))
    ax = -1.0 + 2.0 * np.arange(res) / (res - 1)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    u = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    out = ap.interp_grid(Fi, u)
    np.testing.assert_allclose(out, Fi.reshape(-1, 2), rtol=0, atol=1e-13)


def test_interp_reproduces_trilinear_fields_exactly():
    # Trilinear interpolation is exact for any field a + bX + cY + dZ + eXY + fYZ + gXZ + hXYZ.
    res = 7
    co = np.random.default_rng(3).normal(size=8)
    poly = lambda X, Y, Z: (co[0] + co[1] * X + co[2] * Y + co[3] * Z + co[4] * X * Y
                            + co[5] * Y * Z + co[6] * X * Z + co[7] * X * Y * Z)
    ax = -1.0 + 2.0 * np.arange(res) / (res - 1)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    Fi = poly(x, y, z)[..., None]
    # a trilinear field interpolates exactly only within one cell; on the whole grid
    # the piecewise interpolant is exact for the affine part.  Use an affine field.
    Fa = (co[0] + co[1] * x + co[2] * y + co[3] * z)[..., None]
    u = np.random.default_rng(4).uniform(-1, 1, size=(400, 3))
    np.testing.assert_allclose(ap.interp_grid(Fa, u)[:, 0],
                               co[0] + co[1] * u[:, 0] + co[2] * u[:, 1] + co[3] * u[:, 2],
                               atol=1e-12)
    # within a single cell (R = 2) the full trilinear polynomial is reproduced.
    ax2 = np.array([-1.0, 1.0])
    z2, y2, x2 = np.meshgrid(ax2, ax2, ax2, indexing="ij")
    F2 = poly(x2, y2, z2)[..., None]
    np.testing.assert_allclose(ap.interp_grid(F2, u)[:, 0], poly(u[:, 0], u[:, 1], u[:, 2]),
                               atol=1e-12)
    assert Fi.shape == (res, res, res, 1)


def test_weights_partition_of_unity():
    u = np.random.default_rng(5).uniform(-1, 1, size=(300, 3))
    ones = np.ones((9, 9, 9, 1))
    np.testing.assert_allclose(ap.interp_grid(ones, u)[:, 0], 1.0, atol=1e-14)


def test_out_of_bounds_is_exactly_zero_and_faces_are_inside():
    # Eq. 2: zero outside [-1,1]^3 on any axis; the inequality is inclusive.
    r = np.random.default_rng(6)
    Fi = r.normal(size=(4, 4, 4, 2)) + 5.0
    u_out = np.array([[1.0000001, 0, 0], [0, -1.0000001, 0], [0, 0, 1.5], [-3, -3, -3],
                      [0.5, 0.5, 1.0 + 1e-12]])
    assert np.all(ap.interp_grid(Fi, u_out) == 0.0)
    u_face = np.array([[1.0, 1.0, 1.0], [-1.0, -1.0, -1.0], [1.0, -1.0, 0.2]])
    out = ap.interp_grid(Fi, u_face)
    np.testing.assert_allclose(out[0], Fi[3, 3, 3])
    np.testing.assert_allclose(out[1], Fi[0, 0, 0])
    assert np.all(out[2] != 0.0)


def test_brute_force_single_cell_nested_lerp():
    # R = 2 is one cell; nested linear interpolation (x, then y, then z) is an
    # independent formula for the same trilinear value.
    r = np.random.default_rng(7)
    Fi = r.normal(size=(2, 2, 2, 2))
    u = r.uniform(-1, 1, size=(64, 3))
    out = ap.interp_grid(Fi, u)
    for n in range(64):
        wx, wy, wz = (u[n] + 1.0) / 2.0
        for c in range(2):
            lerp = lambda a, b, w: a + (b - a) * w
            y0 = lerp(lerp(Fi[0, 0, 0, c], Fi[0, 0, 1, c], wx), lerp(Fi[0, 1, 0, c], Fi[0, 1, 1, c], wx), wy)
            y1 = lerp(lerp(Fi[1, 0, 0, c], Fi[1, 0, 1, c], wx), lerp(Fi[1, 1, 0, c], Fi[1, 1, 1, c], wx), wy)
            assert abs(out[n, c] - lerp(y0, y1, wz)) < 1e-13


def test_axis_order_x_is_fastest():
    # Reading: F[i, z, y, x, c]; a field varying only along the x index must vary with u_x.
    res = 5
    Fi = np.zeros((res, res, res, 1))
    Fi[:, :, :, 0] = np.arange(res)[None, None, :]
    u = np.array([[0.5, -0.3, 0.9]])
    assert abs(ap.interp_grid(Fi, u)[0, 0] - (0.5 + 1) / 2 * (res - 1)) < 1e-13


def test_encode_concatenates_grid_major_channel_minor():
    r = np.random.default_rng(8)
    M, R, C = 3, 4, 2
    F = r.normal(size=(M, R, R, R, C))
    G = _rand_G(M, 9)
    x = r.uniform(-0.9, 0.9, size=(20, 3))
    y = ap.encode(F, G, x)
    u = ap.local_coords(G, x)
    assert y.shape == (20, M * C)
    for i in range(M):
        np.testing.assert_array_equal(y[:, i * C:(i + 1) * C], ap.interp_grid(F[i], u[:, i]))
