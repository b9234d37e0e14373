"""FP64 CPU oracle of the APMGSRN point query, its training losses and gradients.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product path (the
CUDA library and its binding) never calls it and shares no code with it.

Every function is the plain definition from the paper (Wurster et al.,
"Adaptively Placed Multi-Grid Scene Representation Networks for Large-Scale
Data Visualization"), evaluated in float64 with numpy, vectorised over points
and looped over grids.  Library routines (einsum/matmul, np.add.at) serve as
single steps; there is no blocking, fusion or reordering beyond the definition.

Readings of points the paper leaves open (axis order, the cell used at a node,
the epsilon in Eq. 9, whether the target density is detached, which error h(x)
is) are stated beside the code that takes them.

Array conventions
  x  [N, 3]           global coordinates (x, y, z)
  G  [M, 3, 4]        first three rows of each 4x4 transform G_i = [A_i | t_i]
  F  [M, R, R, R, C]  feature grids indexed [grid, z, y, x, channel]
  W1 [H, K], W2 [H, H], w3 [H]   bias-free decoder (K = M*C)
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------- encoder


def local_coords(G: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 1: u_i = A_i x + t_i for every grid i.  Returns [N, M, 3]."""
    G = np.asarray(G, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    A = G[:, :, :3]
    t = G[:, :, 3]
    return np.einsum("mde,ne->nmd", A, x) + t[None, :, :]


def inside_mask(u: np.ndarray) -> np.ndarray:
    """Eq. 2 condition -1 <= u <= 1 on all three axes (inclusive).  u [..., 3]."""
    return np.all((u >= -1.0) & (u <= 1.0), axis=-1)


def cell_and_weights(u: np.ndarray, res: int):
    """Corner-aligned trilinear set-up for Eq. 2 on an R^3 grid.

    Node j of an axis sits at local coordinate -1 + 2j/(R-1) (vertices at the
    extents, Sec. 4.1.1).  s = (u+1)/2 (R-1); the cell is c = min(floor(s), R-2)
    (reading: at the upper face and at nodes the lower cell is used; the value is
    the same either way) and w = s - c in [0, 1].  Coordinates outside [-1, 1]
    are clipped only so that indices stay valid; their features are masked to 0.
    Returns (c int [..., 3] in (x, y, z) order, w [..., 3])."""
    s = (np.clip(u, -1.0, 1.0) + 1.0) / 2.0 * (res - 1)
    c = np.minimum(np.floor(s), res - 2).astype(np.int64)
    w = s - c
    return c, w


def corner_offsets():
    """The 8 corners of a cell as (dx, dy, dz) in {0,1}^3."""
    return [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]


def corner_weight(w: np.ndarray, dx: int, dy: int, dz: int) -> np.ndarray:
    """Trilinear weight of corner (dx, dy, dz): product over axes of w or 1-w."""
    wx = w[..., 0] if dx else 1.0 - w[..., 0]
    wy = w[..., 1] if dy else 1.0 - w[..., 1]
    wz = w[..., 2] if dz else 1.0 - w[..., 2]
    return wx * wy * wz


def interp_grid(Fi: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. 2 for one grid: e_i(u) = interp(F_i, u) if -1 <= u <= 1 else 0.

    Fi [R, R, R, C] (z, y, x, c); u [N, 3].  Returns [N, C]."""
    res = Fi.shape[0]
    c, w = cell_and_weights(u, res)
    out = np.zeros((u.shape[0], Fi.shape[3]))
    for dx, dy, dz in corner_offsets():
        wt = corner_weight(w, dx, dy, dz)
        out += wt[:, None] * Fi[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx, :]
    out[~inside_mask(u)] = 0.0
    return out


def encode(F: np.ndarray, G: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 3: y = e_0(G_0 x) (+) ... (+) e_{M-1}(G_{M-1} x), grid-major, channel-minor.
    Returns [N, M*C]."""
    F = np.asarray(F, dtype=np.float64)
    u = local_coords(G, x)
    feats = [interp_grid(F[i], u[:, i, :]) for i in range(F.shape[0])]
    return np.concatenate(feats, axis=1)


# ----------------------------------------------------------------------------- decoder


def relu(z):
    return np.maximum(z, 0.0)


def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), as float64.

    Used only as the operand rounding of the mixed-precision reading: a bfloat16
    number is a float32 whose low 16 bits are zero, so rounding keeps the high
    half after adding half an ulp of the kept part (plus the kept lsb for ties)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (bits >> np.uint64(16)) & np.uint64(1)
    bits = ((bits + np.uint64(0x7FFF) + keep_lsb) >> np.uint64(16)) << np.uint64(16)
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def mlp_forward(W1, W2, w3, y, rnd=None):
    """Sec. 4.1.2: two bias-free hidden layers with ReLU, linear scalar output.

    rnd (default none) rounds the activation operand of each hidden-layer matrix
    product (y and ReLU(z1)); with rnd=bf16 this is the mixed-precision reading of
    the decoder (BF16 operands, wide accumulation).  The weights are used as given.
    Returns (m [N], cache) with the pre-activations and activations."""
    rnd = rnd or _ident
    W1, W2, w3 = (np.asarray(a, dtype=np.float64) for a in (W1, W2, w3))
    yq = rnd(y)
    z1 = yq @ W1.T
    h1 = relu(z1)
    h1q = rnd(h1)
    z2 = h1q @ W2.T
    h2 = relu(z2)
    m = h2 @ w3
    return m, {"y": y, "yq": yq, "z1": z1, "h1": h1, "h1q": h1q, "z2": z2, "h2": h2}


def scale_output(m, vmin, vmax):
    """Sec. 4.1.2 "Scaling": d(y) = m(y) (max - min) + min."""
    return m * (vmax - vmin) + vmin


def query(params: dict, x: np.ndarray, rnd=None) -> np.ndarray:
    """f(x) = d(e(x)): Eq. 1-3, the decoder and the output scaling.  Returns [N]."""
    y = encode(params["F"], params["G"], x)
    m, _ = mlp_forward(params["W1"], params["W2"], params["w3"], y, rnd)
    return scale_output(m, params["vmin"], params["vmax"])


# ----------------------------------------------------------------------------- losses


def loss_rec(f, v):
    """Sec. 4.3.1: L_rec = (1/|X|) sum (f(x) - v(x))^2."""
    return float(np.mean((np.asarray(f) - np.asarray(v)) ** 2))


def flat_top_terms(G, x, p: int = 10):
    """Eq. 7 per grid: E_i(x) = exp(-sum_d u_d^(2p)) and det(A_i).
    Returns (E [N, M], det [M], u [N, M, 3])."""
    G = np.asarray(G, dtype=np.float64)
    u = local_coords(G, x)
    E = np.exp(-np.sum(u ** (2 * p), axis=2))
    det = np.linalg.det(G[:, :, :3])
    return E, det, u


def feature_density(G, x, p: int = 10):
    """Eq. 7: rho(x) = sum_i det(A_i) exp(-sum_d (G_i(x)_d)^(2p)).  Returns [N]."""
    E, det, _ = flat_top_terms(G, x, p)
    return E @ det


def density_terms(rho, h, eps: float = 1e-8):
    """Eq. 8 and Eq. 9 from the current density rho [N] and per-point error h [N].

    rho_s = rho / sum(rho) (the set X is the batch);  hbar = mean(h);
    k = hbar / (h + eps);  rho* = exp(k log(rho_s + eps));
    L_den = mean(rho* (log rho* - log(rho_s + eps))).
    Readings: log(rho*) is k log(rho_s + eps) by the definition of rho* (so an
    underflowed rho* never produces log 0); Eq. 9's log(rho_s) takes the same
    eps as Eq. 8, since rho_s can be exactly 0.
    Returns a dict with every intermediate."""
    rho = np.asarray(rho, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    S = rho.sum()
    rho_s = rho / S
    hbar = h.mean()
    k = hbar / (h + eps)
    log_rs = np.log(rho_s + eps)
    log_star = k * log_rs
    rho_star = np.exp(log_star)
    L = float(np.mean(rho_star * (log_star - log_rs)))
    return {"S": S, "rho_s": rho_s, "hbar": hbar, "k": k, "rho_star": rho_star,
            "log_rs": log_rs, "L_den": L}


def loss_density(G, x, h, p: int = 10, eps: float = 1e-8) -> float:
    """L_den (Eq. 7-9) as a function of the transforms, the batch and the error h."""
    return density_terms(feature_density(G, x, p), h, eps)["L_den"]


def loss_density_fixed_target(G, x, rho_star, p: int = 10, eps: float = 1e-8) -> float:
    """Eq. 9 with the target rho* held constant (it is a target the density is steered
    toward, Sec. 4.2, so no gradient flows through it).  Used for finite differences."""
    rho = feature_density(G, x, p)
    rho_s = rho / rho.sum()
    rho_star = np.asarray(rho_star, dtype=np.float64)
    log_star = np.log(np.where(rho_star > 0, rho_star, 1.0))
    return float(np.mean(np.where(rho_star > 0, rho_star * (log_star - np.log(rho_s + eps)), 0.0)))


# ----------------------------------------------------------------------------- gradients


def grad_rec(params: dict, x, v, rnd=None):
    """Analytic gradient of L_rec (Sec. 4.3.1) w.r.t. F, W1, W2, w3 (step (1) of
    Sec. 4.3.2: L_rec updates only the grids' features and the decoder).

    Chain rule written out: f = m (max-min) + min, dL/df = 2 (f - v)/N.
    rnd (see mlp_forward) also rounds the activation-side operand of every
    backward matrix product (dz2, dz1, and the y / ReLU(z1) factors of dW) and
    dL/dy itself, which the mixed-precision reading hands on to the adjoint of
    Eq. 2 in that format.  The ReLU masks are taken from the unrounded
    pre-activations.  Returns dict(L_rec, f, h, dF, dW1, dW2, dw3, dy) where
    h = (f - v)^2 per point and dy = dL/dy [N, M*C]."""
    q = rnd or _ident
    F = np.asarray(params["F"], dtype=np.float64)
    G = np.asarray(params["G"], dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    n = x.shape[0]
    M, R, C = F.shape[0], F.shape[1], F.shape[4]
    y = encode(F, G, x)
    m, c = mlp_forward(params["W1"], params["W2"], params["w3"], y, rnd)
    span = params["vmax"] - params["vmin"]
    f = scale_output(m, params["vmin"], params["vmax"])
    r = f - v
    dm = 2.0 * r * span / n                           # dL/dm
    W1 = np.asarray(params["W1"], dtype=np.float64)
    W2 = np.asarray(params["W2"], dtype=np.float64)
    w3 = np.asarray(params["w3"], dtype=np.float64)
    dw3 = c["h2"].T @ dm
    dz2 = q(dm[:, None] * w3[None, :] * (c["z2"] > 0))
    dW2 = dz2.T @ c["h1q"]
    dz1 = q((dz2 @ W2) * (c["z1"] > 0))
    dW1 = dz1.T @ c["yq"]
    dy = q(dz1 @ W1)                                  # [N, M*C]
    dF = np.zeros_like(F)
    u = local_coords(G, x)
    for i in range(M):
        ui = u[:, i, :]
        ins = inside_mask(ui)
        cc, w = cell_and_weights(ui, R)
        g = dy[:, i * C:(i + 1) * C]
        flat = dF[i].reshape(R * R * R, C)
        for dx, dyy, dz in corner_offsets():
            wt = (corner_weight(w, dx, dyy, dz) * ins)[:, None] * g
            node = ((cc[:, 2] + dz) * R + (cc[:, 1] + dyy)) * R + (cc[:, 0] + dx)
            for ch in range(C):   # scatter-add of each point's share into its corner node
                flat[:, ch] += np.bincount(node, weights=wt[:, ch], minlength=R * R * R)
    return {"L_rec": float(np.mean(r ** 2)), "f": f, "h": r ** 2, "dF": dF,
            "dW1": dW1, "dW2": dW2, "dw3": dw3, "dy": dy}


def interp_grid_du(Fi: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Derivative of Eq. 2 for one grid with respect to the local coordinate u.

    Inside the cell the interpolant is trilinear in w = s - c, so d e / d w_x is the
    sum over corners of (+1 for dx = 1, -1 for dx = 0) times the other two axes'
    weights times the corner value, and likewise for y and z; ds/du = (R-1)/2.
    Outside [-1, 1] the feature is the constant 0, so its derivative is 0.  At a cell
    face the derivative is the one of the cell chosen by cell_and_weights.
    Fi [R, R, R, C]; u [N, 3].  Returns [N, C, 3] (last axis: d/du_x, d/du_y, d/du_z)."""
    res = Fi.shape[0]
    c, w = cell_and_weights(u, res)
    out = np.zeros((u.shape[0], Fi.shape[3], 3))
    for dx, dy, dz in corner_offsets():
        val = Fi[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx, :]          # [N, C]
        fx = w[:, 0] if dx else 1.0 - w[:, 0]
        fy = w[:, 1] if dy else 1.0 - w[:, 1]
        fz = w[:, 2] if dz else 1.0 - w[:, 2]
        out[:, :, 0] += ((1.0 if dx else -1.0) * fy * fz)[:, None] * val
        out[:, :, 1] += ((1.0 if dy else -1.0) * fx * fz)[:, None] * val
        out[:, :, 2] += ((1.0 if dz else -1.0) * fx * fy)[:, None] * val
    out *= (res - 1) / 2.0
    out[~inside_mask(u)] = 0.0
    return out


def grad_transform_through_features(params: dict, x, dy):
    """Gradient that a loss with dL/dy = dy [N, M*C] sends into the transforms G
    through the features (Eq. 1 and Eq. 2), with u_i = A_i x + t_i:
    dL/dA_i = sum_n (dL/du_in) x_n^T and dL/dt_i = sum_n dL/du_in, where
    dL/du_in = sum_c dy_{n,(i,c)} d e_{i,c} / d u.
    Sec. 4.3.2 trains G with L_den alone; this is the L_rec part left out there,
    for diagnostics and for the full gradient of f.  Returns dG [M, 3, 4]."""
    F = np.asarray(params["F"], dtype=np.float64)
    G = np.asarray(params["G"], dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    M, C = F.shape[0], F.shape[4]
    u = local_coords(G, x)
    dG = np.zeros_like(G)
    for i in range(M):
        J = interp_grid_du(F[i], u[:, i, :])                        # [N, C, 3]
        dLdu = np.einsum("nc,ncd->nd", dy[:, i * C:(i + 1) * C], J)   # [N, 3]
        dG[i, :, :3] = dLdu.T @ x
        dG[i, :, 3] = dLdu.sum(axis=0)
    return dG


def grad_density(G, x, h, p: int = 10, eps: float = 1e-8):
    """Analytic gradient of L_den (Eq. 7-9) w.r.t. G with rho* detached (step (2) of
    Sec. 4.3.2: L_den is the only loss that moves the transforms).

    With g_n = dL/d(rho_s,n) = -rho*_n / (N (rho_s,n + eps)) and rho_s = rho/S,
    dL/drho_n = (g_n - sum_m g_m rho_s,m) / S.  For grid i,
    drho_n/dA_i = det_i A_i^{-T} E_in - det_i E_in 2p (u_in^(2p-1)) x_n^T
    (Jacobi's formula d det/dA = det A^{-T}), drho_n/dt_i = -det_i E_in 2p u_in^(2p-1).
    Returns dict(L_den, dG [M, 3, 4], rho, terms)."""
    G = np.asarray(G, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    E, det, u = flat_top_terms(G, x, p)
    rho = E @ det
    t = density_terms(rho, h, eps)
    g = -t["rho_star"] / (n * (t["rho_s"] + eps))
    q = (g - np.sum(g * t["rho_s"])) / t["S"]          # dL/drho_n
    dG = np.zeros_like(G)
    for i in range(G.shape[0]):
        A = G[i, :, :3]
        up = 2 * p * u[:, i, :] ** (2 * p - 1)           # d(sum u^2p)/du
        wq = q * E[:, i] * det[i]                        # [N]
        dA = np.sum(wq) * np.linalg.inv(A).T - (wq[:, None] * up).T @ x
        dt = -(wq[:, None] * up).sum(axis=0)
        dG[i, :, :3] = dA
        dG[i, :, 3] = dt
    return {"L_den": t["L_den"], "dG": dG, "rho": rho, "terms": t}


# ----------------------------------------------------------------------------- optimiser


def adam_update(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.99, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; Sec. 6 "Training" fixes
    beta = (0.9, 0.99) and lr 0.01 (0.001 for the transforms); eps is not given
    (reading: 1e-8).  t is this parameter's 1-based step count.
    Returns (p', m', v')."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------------------------- data side


def volume_sample(vol, x, box=None):
    """v(x) of Sec. 4.3.1: trilinear interpolation of a scalar volume [Vz, Vy, Vx].

    Voxels are corner-aligned: along an axis the box [lo, hi] (inclusive voxel
    indices; default the whole volume) spans local coordinates [-1, 1], so voxel
    lo + j sits at -1 + 2j/(hi - lo).  x [N, 3] must lie in [-1, 1]^3."""
    vol = np.asarray(vol, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if box is None:
        box = [0, 0, 0, vol.shape[2] - 1, vol.shape[1] - 1, vol.shape[0] - 1]
    lo = np.array(box[:3], dtype=np.float64)
    hi = np.array(box[3:], dtype=np.float64)
    s = lo + (np.clip(x, -1, 1) + 1.0) / 2.0 * (hi - lo)
    c = np.minimum(np.floor(s), hi - 1).astype(np.int64)
    w = s - c
    out = np.zeros(x.shape[0])
    for dx, dy, dz in corner_offsets():
        out += corner_weight(w, dx, dy, dz) * vol[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx]
    return out


def brick_index(p, grid):
    """Sec. 5.3 spatial hash: i = floor(I (p_x + 1)/2) (likewise j, k), clamped so that
    i < I (and, reading, i >= 0); flat index i + I j + I J k.  p [N, 3] global."""
    p = np.asarray(p, dtype=np.float64)
    I, J, K = grid
    idx = []
    for d, n in enumerate((I, J, K)):
        i = np.floor(n * (p[:, d] + 1.0) / 2.0).astype(np.int64)
        idx.append(np.clip(i, 0, n - 1))
    return idx[0] + I * idx[1] + I * J * idx[2]


def global_to_brick_local(p, box, vox: int):
    """Map global coordinates (whole volume of `vox` voxels per axis spans [-1, 1])
    into the local [-1, 1]^3 of a brick whose voxel box is `box` (lo xyz, hi xyz)."""
    p = np.asarray(p, dtype=np.float64)
    lo = np.array(box[:3], dtype=np.float64)
    hi = np.array(box[3:], dtype=np.float64)
    s = (p + 1.0) / 2.0 * (vox - 1)
    return (s - lo) / (hi - lo) * 2.0 - 1.0
