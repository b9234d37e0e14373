"""Pins of the oracle's analytic gradients against central finite differences in FP64."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from paper_2308_02494_gb300 import synth


def _model(seed, M=4, R=5, C=2, H=8):
    shape = synth.ModelShape(n_grids=M, res=R, channels=C, hidden=H)
    p = synth.parity_model(shape, seed, shrink=0.4)
    return p


def _points_off_faces(p, n, seed, margin=1e-3):
    r = np.random.default_rng(seed)
    x = r.uniform(-1, 1, size=(4 * n, 3))
    u = ap.local_coords(p["G"], x)
    R = p["F"].shape[1]
    s = (np.clip(u, -1, 1) + 1) / 2 * (R - 1)
    frac = s - np.round(s)
    ok = np.all(np.abs(np.abs(u) - 1.0) > margin, axis=(1, 2)) & np.all(np.abs(frac) > margin, axis=(1, 2))
    return x[ok][:n]


def _fd(fun, arr, idx, h):
    a = arr.copy()
    a[idx] += h
    fp = fun(a)
    a[idx] -= 2 * h
    fm = fun(a)
    return (fp - fm) / (2 * h)


def test_grad_rec_matches_finite_differences():
    p = _model(0)
    x = _points_off_faces(p, 40, 1)
    v = np.random.default_rng(2).uniform(0, 1, size=x.shape[0])
    g = ap.grad_rec(p, x, v)

    def L_of(name):
        def f(a):
            q = dict(p)
            q[name] = a
            return ap.loss_rec(ap.query(q, x), v)
        return f

    r = np.random.default_rng(3)
    for name, grad in (("F", g["dF"]), ("W1", g["dW1"]), ("W2", g["dW2"]), ("w3", g["dw3"])):
        arr = np.asarray(p[name], dtype=np.float64)
        flat_nz = np.flatnonzero(np.abs(grad) > 1e-9 * np.abs(grad).max())
        picks = r.choice(flat_nz, size=min(12, flat_nz.size), replace=False)
        for fi in picks:
            idx = np.unravel_index(fi, arr.shape)
            h = 1e-6 * max(1.0, abs(arr[idx]))
            fd = _fd(L_of(name), arr, idx, h)
            assert abs(fd - grad[idx]) <= 1e-6 * np.abs(grad).max() + 1e-7 * abs(grad[idx]), (name, idx)
    # entries untouched by every point have exactly zero gradient
    assert np.any(g["dF"] == 0.0)


def test_grad_density_matches_finite_differences_with_detached_target():
    r = np.random.default_rng(4)
    M = 3
    G = np.zeros((M, 3, 4))
    for d in range(3):
        G[:, d, d] = 1.0
    G += r.normal(0, 0.1, size=G.shape)
    x = r.uniform(-1.1, 1.1, size=(60, 3))
    h = r.uniform(0.0, 0.5, size=60)
    out = ap.grad_density(G, x, h)
    star = out["terms"]["rho_star"]
    L0 = ap.loss_density_fixed_target(G, x, star)
    assert abs(L0 - out["L_den"]) < 1e-12 * max(1, abs(L0))
    f = lambda a: ap.loss_density_fixed_target(a, x, star)
    scale = np.abs(out["dG"]).max()
    for idx in np.ndindex(G.shape):
        fd = _fd(f, G, idx, 1e-6)
        assert abs(fd - out["dG"][idx]) <= 1e-6 * scale, idx


@pytest.mark.parametrize("p", [1, 3, 10])
def test_grad_density_other_flat_top_strengths(p):
    r = np.random.default_rng(5 + p)
    G = np.zeros((2, 3, 4))
    for d in range(3):
        G[:, d, d] = 1.0
    G += r.normal(0, 0.1, size=G.shape)
    x = r.uniform(-1, 1, size=(30, 3))
    h = r.uniform(0.01, 0.5, size=30)
    out = ap.grad_density(G, x, h, p=p)
    star = out["terms"]["rho_star"]
    f = lambda a: ap.loss_density_fixed_target(a, x, star, p=p)
    scale = np.abs(out["dG"]).max()
    for idx in np.ndindex(G.shape):
        assert abs(_fd(f, G, idx, 1e-6) - out["dG"][idx]) <= 1e-6 * scale, idx


def test_transform_gradient_through_features_matches_finite_differences():
    """dL_rec/dG through Eq. 1-2 (the part of the gradient Sec. 4.3.2 leaves out of
    training) against central differences of L_rec in every entry of G."""
    p = _model(5, M=3, R=6)
    x = _points_off_faces(p, 50, 6)
    v = np.random.default_rng(7).uniform(0, 1, size=x.shape[0])
    g = ap.grad_rec(p, x, v)
    dG = ap.grad_transform_through_features(p, x, g["dy"])
    G0 = np.asarray(p["G"], dtype=np.float64)

    def f(a):
        q = dict(p)
        q["G"] = a
        return ap.loss_rec(ap.query(q, x), v)

    scale = np.abs(dG).max()
    assert scale > 0
    for idx in np.ndindex(G0.shape):
        fd = _fd(f, G0, idx, 1e-7)
        assert abs(fd - dG[idx]) <= 1e-6 * scale, (idx, fd, dG[idx])


def test_transform_gradient_of_affine_feature_fields_is_closed_form():
    """Grids whose node values are an affine function a + B u of the node's local
    coordinate interpolate to exactly a + B u inside [-1, 1]^3, so
    dL/dA_i[d, e] = sum_n [u_in inside] sum_c dy_n,c B_i[c, d] x_n,e (and x_n,e -> 1 for t)."""
    r = np.random.default_rng(11)
    M, R, C, n = 3, 7, 2, 200
    G = np.zeros((M, 3, 4))
    for d in range(3):
        G[:, d, d] = 1.3
    G += r.normal(0, 0.2, size=G.shape)
    a = r.normal(size=(M, C))
    B = r.normal(size=(M, C, 3))
    node = -1.0 + 2.0 * np.arange(R) / (R - 1)
    F = np.zeros((M, R, R, R, C))
    for i in range(M):
        for c in range(C):
            F[i, :, :, :, c] = (a[i, c] + B[i, c, 0] * node[None, None, :] + B[i, c, 1] * node[None, :, None]
                                + B[i, c, 2] * node[:, None, None])
    x = r.uniform(-1.2, 1.2, size=(n, 3))
    dy = r.normal(size=(n, M * C))
    got = ap.grad_transform_through_features({"F": F, "G": G}, x, dy)
    u = np.einsum("mde,ne->nmd", G[:, :, :3], x) + G[None, :, :, 3]
    xt = np.concatenate([x, np.ones((n, 1))], axis=1)
    for i in range(M):
        ins = np.all(np.abs(u[:, i, :]) <= 1.0, axis=1)
        assert 0 < ins.sum() < n
        want = np.zeros((3, 4))
        for k in range(n):
            if ins[k]:
                want += np.outer(dy[k, i * C:(i + 1) * C] @ B[i], xt[k])
        assert np.allclose(got[i], want, rtol=1e-12, atol=1e-12), i
    # points outside every grid send nothing back
    far = np.full((5, 3), 9.0)
    assert np.all(ap.grad_transform_through_features({"F": F, "G": G}, far, r.normal(size=(5, M * C))) == 0.0)
