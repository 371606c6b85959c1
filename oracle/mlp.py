"""FP64 reference of the learned flux correction (TEST INFRASTRUCTURE ONLY).

The correction is not in the paper; it is the benchmark's addition to the
HLLC flux of Sec. 3.2.  This module is the plain NumPy FP64 statement of what
the CUDA kernels compute, written independently of them:

* features of a face along axis q between cells i-1 and i of a 2D state: the
  six cells i-3 .. i+2 along q; per cell (rho, v_n, v_t, p) with v_n the
  velocity along q and v_t the other component; with rho_bar, p_bar the means
  over the six cells and c_bar = sqrt(gamma p_bar / rho_bar), the 24 features
  are rho/rho_bar - 1, v_n/c_bar, v_t/c_bar, p/p_bar - 1 (cells in order);
* flux scales of the face: (rho_bar c_bar, rho_bar c_bar^2, rho_bar c_bar^2,
  rho_bar c_bar^3) for (mass, normal momentum, transverse momentum, energy);
* network: z1 = W1 x + b1 (64), h1 = silu(z1), z2 = W2 h1 + b2 (64),
  h2 = silu(z2), y = W3 h2 + b3 (4), silu(z) = z / (1 + exp(-z));
* the correction added to the face flux is scale * y, rotated back: mass ->
  D, normal momentum -> S_q, transverse momentum -> the other S, energy -> G;
* loss: mean over samples and the 4 outputs of (y - target)^2;
* Adam (Kingma & Ba) with bias correction.

Parameter vector layout (FP32 on the device, FP64 here), in this order:
W1 [64][24], b1 [64], W2 [64][64], b2 [64], W3 [4][64], b3 [4]  (6020 values).
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 24, 64, 4
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed=0):
    """He-style uniform initialisation; the last layer starts at zero so the
    corrected scheme starts as the plain one."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.uniform(-1, 1, (NH, NIN)) * np.sqrt(3.0 / NIN), "b1": np.zeros(NH),
         "W2": rng.uniform(-1, 1, (NH, NH)) * np.sqrt(3.0 / NH), "b2": np.zeros(NH),
         "W3": np.zeros((NOUT, NH)), "b3": np.zeros(NOUT)}
    return pack(d)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, emulate_bf16=False):
    """X: [N, 24] -> (Y [N, 4], cache).  With emulate_bf16 the inputs, weights
    and hidden activations are rounded to bfloat16 (biases and sums stay
    exact), which is what the tensor-core kernels store."""
    P = unpack(theta)
    r = bf16 if emulate_bf16 else (lambda a: a)
    z1 = r(X) @ r(P["W1"]).T + P["b1"]
    h1 = r(silu(z1))
    z2 = h1 @ r(P["W2"]).T + P["b2"]
    h2 = r(silu(z2))
    Y = h2 @ r(P["W3"]).T + P["b3"]
    return Y, (X, z1, h1, z2, h2)


def loss(theta, X, T):
    Y, _ = forward(theta, X)
    return float(np.mean((Y - T) ** 2))


def grad(theta, X, T):
    """Gradient of `loss` with respect to the packed parameters."""
    P = unpack(theta)
    Y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    dY = 2.0 * (Y - T) / (n * NOUT)
    g = {"W3": dY.T @ h2, "b3": dY.sum(0)}
    dz2 = (dY @ P["W3"]) * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * dsilu(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def face_features(rho, vx, vy, p, gamma, axis):
    """Features and scales of every face of a periodic 2D state.

    rho, vx, vy, p: [ny, nx].  axis 0: x-faces, face (j, i) between cells
    (j, i-1) and (j, i); axis 1: y-faces, face (j, i) between (j-1, i) and (j, i).
    Returns X [ny, nx, 24], scale [ny, nx, 4]."""
    ax = 1 if axis == 0 else 0           # numpy axis along the face normal
    vn, vt = (vx, vy) if axis == 0 else (vy, vx)
    stencil = []
    for k in range(6):                    # cell i - 3 + k
        shift = 3 - k
        stencil.append([np.roll(f, shift, axis=ax) for f in (rho, vn, vt, p)])
    rbar = sum(s[0] for s in stencil) / 6.0
    pbar = sum(s[3] for s in stencil) / 6.0
    cbar = np.sqrt(gamma * pbar / rbar)
    X = np.empty(rho.shape + (24,))
    for k, (r, a, b, q) in enumerate(stencil):
        X[..., 4 * k + 0] = r / rbar - 1.0
        X[..., 4 * k + 1] = a / cbar
        X[..., 4 * k + 2] = b / cbar
        X[..., 4 * k + 3] = q / pbar - 1.0
    scale = np.stack([rbar * cbar, rbar * cbar ** 2, rbar * cbar ** 2, rbar * cbar ** 3], axis=-1)
    return X, scale


def rotate_back(dF_face, axis):
    """Face-frame (mass, normal, transverse, energy) -> conserved order
    (D, S_x, S_y, G) for faces normal to `axis`."""
    out = np.empty_like(dF_face)
    out[..., 0] = dF_face[..., 0]
    out[..., 3] = dF_face[..., 3]
    if axis == 0:
        out[..., 1], out[..., 2] = dF_face[..., 1], dF_face[..., 2]
    else:
        out[..., 1], out[..., 2] = dF_face[..., 2], dF_face[..., 1]
    return out


def corrected_rhs(oracle, grid, U, theta, emulate_bf16=False, plain_faces=None, ylim=np.inf):
    """L[U] of the corrected scheme on a periodic 2D mesh: the oracle's plain
    face fluxes plus scale * network(features), rotated to conserved order.
    plain_faces: optional boolean masks (mx [ny, nx+1], my [ny+1, nx]) of faces
    that keep the plain flux.  Returns (L, Fx, Fy)."""
    Fx, Fy = oracle.face_fluxes_2d(grid, U)
    rho, vel, p = oracle.cons_to_prim(grid, U)
    for axis, F in ((0, Fx), (1, Fy)):
        X, sc = face_features(rho, vel[0], vel[1], p, grid.gamma, axis)
        y, _ = forward(theta, X.reshape(-1, NIN), emulate_bf16)
        y = np.clip(y, -ylim, ylim)
        dF = rotate_back(sc * y.reshape(sc.shape), axis)       # [ny, nx, 4]
        dF = np.moveaxis(dF, -1, 0)                              # [4, ny, nx]
        if axis == 0:
            full = np.concatenate([dF, dF[:, :, :1]], axis=2)    # periodic: face nx = face 0
        else:
            full = np.concatenate([dF, dF[:, :1, :]], axis=1)
        if plain_faces is not None:
            full = np.where(plain_faces[axis][None], 0.0, full)
        F += full
    wx = np.asarray(grid.widths[0])
    wy = np.asarray(grid.widths[1])
    L = -((Fx[:, :, 1:] - Fx[:, :, :-1]) / wx[None, None, :] + (Fy[:, 1:, :] - Fy[:, :-1, :]) / wy[None, :, None])
    return L, Fx, Fy


def _bad_cells(oracle, grid, U):
    rho, vel, p = oracle.cons_to_prim(grid, U, check=False)
    return ~((rho > 0) & (p > 0) & np.isfinite(rho) & np.isfinite(p))


def _plain_masks(bad):
    """Faces touching a flagged cell (periodic neighbours)."""
    mx = np.zeros((bad.shape[0], bad.shape[1] + 1), dtype=bool)
    mx[:, :-1] |= bad
    mx[:, 1:] |= bad
    mx[:, 0] |= bad[:, -1]
    mx[:, -1] |= bad[:, 0]
    my = np.zeros((bad.shape[0] + 1, bad.shape[1]), dtype=bool)
    my[:-1, :] |= bad
    my[1:, :] |= bad
    my[0, :] |= bad[-1, :]
    my[-1, :] |= bad[0, :]
    return mx, my


def corrected_step(oracle, grid, U, dt, theta, emulate_bf16=False, ylim=np.inf):
    """One TVD RK2 step (Eqs. Update, RungeKutta1-3) of the corrected scheme on
    a periodic 2D mesh, with the a-posteriori fallback: after each stage, faces
    touching a cell whose corrected candidate has rho <= 0 or p <= 0 use the
    plain flux, and the stage is recomputed.  Returns (U_new, flagged cells)."""
    flagged = 0
    L1, _, _ = corrected_rhs(oracle, grid, U, theta, emulate_bf16, ylim=ylim)
    bad = _bad_cells(oracle, grid, U + dt * L1)
    if bad.any():
        flagged += int(bad.sum())
        L1, _, _ = corrected_rhs(oracle, grid, U, theta, emulate_bf16, _plain_masks(bad), ylim=ylim)
    K1 = dt * L1
    U1 = U + K1
    L2, _, _ = corrected_rhs(oracle, grid, U1, theta, emulate_bf16, ylim=ylim)
    cand = U + 0.5 * (K1 + dt * L2)
    bad = _bad_cells(oracle, grid, cand)
    if bad.any():
        flagged += int(bad.sum())
        L2, _, _ = corrected_rhs(oracle, grid, U1, theta, emulate_bf16, _plain_masks(bad), ylim=ylim)
    return U + 0.5 * (K1 + dt * L2), flagged


# --------------------------------------------------------------------------
# Flux-corrected transport (Zalesak, J. Comput. Phys. 31, 1979) applied to the
# learned correction: the plain flux is the low-order flux and the network's
# correction the antidiffusive flux.  For a stage U_new = U_b - c dt div(F):
#   U_L      = U_b - c dt div(F_plain)                     (low-order update)
#   bounds   U_max/U_min over the cell and its four face neighbours of
#            U_L and of the stage's input state
#   P+ / P-  sum of the positive / negative antidiffusive contributions
#            (+c dt dF_left/dx - c dt dF_right/dx + same in y)
#   R+ = min(1, (U_max - U_L)/P+), R- = min(1, (U_L - U_min)/P-)  (1 if P = 0)
#   face factor: dF > 0 -> min(R+_right, R-_left), dF < 0 -> min(R-_right, R+_left),
#   taken as the minimum over the conserved variables and applied to all of them.
# --------------------------------------------------------------------------

def _neighbour_extrema(a):
    """Max and min over each cell and its four periodic face neighbours;
    a: [nv, ny, nx]."""
    stack = [a, np.roll(a, 1, 2), np.roll(a, -1, 2), np.roll(a, 1, 1), np.roll(a, -1, 1)]
    return np.max(stack, axis=0), np.min(stack, axis=0)


def fct_factors(U_b, U_in, Fx_plain, Fy_plain, dFx, dFy, cdt, wx, wy):
    """Face factors Cx [ny, nx+1], Cy [ny+1, nx] of the FCT limiter (periodic)."""
    divp = (Fx_plain[:, :, 1:] - Fx_plain[:, :, :-1]) / wx[None, None, :] + (Fy_plain[:, 1:, :] - Fy_plain[:, :-1, :]) / wy[None, :, None]
    UL = U_b - cdt * divp
    umax = _neighbour_extrema(np.maximum(UL, U_in))[0]
    umin = _neighbour_extrema(np.minimum(UL, U_in))[1]
    cl = cdt * dFx[:, :, :-1] / wx[None, None, :]      # from the left face, into the cell
    cr = -cdt * dFx[:, :, 1:] / wx[None, None, :]      # from the right face
    cb = cdt * dFy[:, :-1, :] / wy[None, :, None]
    ct = -cdt * dFy[:, 1:, :] / wy[None, :, None]
    contrib = np.stack([cl, cr, cb, ct])
    Pp = np.sum(np.maximum(contrib, 0.0), axis=0)
    Pm = np.sum(np.maximum(-contrib, 0.0), axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        Rp = np.where(Pp > 0, np.minimum(1.0, (umax - UL) / Pp), 1.0)
        Rm = np.where(Pm > 0, np.minimum(1.0, (UL - umin) / Pm), 1.0)
    # x faces: face i between cells i-1 (left) and i (right), periodic
    Rp_l, Rm_l = np.roll(Rp, 1, 2), np.roll(Rm, 1, 2)
    cxv = np.where(dFx[:, :, :-1] > 0, np.minimum(Rp, Rm_l), np.where(dFx[:, :, :-1] < 0, np.minimum(Rm, Rp_l), 1.0))
    Cx = np.min(cxv, axis=0)
    Cx = np.concatenate([Cx, Cx[:, :1]], axis=1)
    Rp_b, Rm_b = np.roll(Rp, 1, 1), np.roll(Rm, 1, 1)
    cyv = np.where(dFy[:, :-1, :] > 0, np.minimum(Rp, Rm_b), np.where(dFy[:, :-1, :] < 0, np.minimum(Rm, Rp_b), 1.0))
    Cy = np.min(cyv, axis=0)
    Cy = np.concatenate([Cy, Cy[:1, :]], axis=0)
    return Cx, Cy


def _corrections(oracle, grid, U, theta, emulate_bf16, ylim):
    Fx, Fy = oracle.face_fluxes_2d(grid, U)
    rho, vel, p = oracle.cons_to_prim(grid, U)
    d = []
    for axis in (0, 1):
        X, sc = face_features(rho, vel[0], vel[1], p, grid.gamma, axis)
        y, _ = forward(theta, X.reshape(-1, NIN), emulate_bf16)
        y = np.clip(y, -ylim, ylim)
        dF = np.moveaxis(rotate_back(sc * y.reshape(sc.shape), axis), -1, 0)
        d.append(np.concatenate([dF, dF[:, :, :1]], axis=2) if axis == 0 else np.concatenate([dF, dF[:, :1, :]], axis=1))
    return Fx, Fy, d[0], d[1]


def fct_step(oracle, grid, U, dt, theta, emulate_bf16=False, ylim=np.inf):
    """One TVD RK2 step of the FCT-limited corrected scheme on a periodic 2D
    mesh (stage 1: U_b = U^n, c = 1; stage 2: U_b = U^n + dt K/2, c = 1/2)."""
    wx = np.asarray(grid.widths[0])
    wy = np.asarray(grid.widths[1])

    def div(Fx, Fy):
        return (Fx[:, :, 1:] - Fx[:, :, :-1]) / wx[None, None, :] + (Fy[:, 1:, :] - Fy[:, :-1, :]) / wy[None, :, None]

    Fx, Fy, dx_, dy_ = _corrections(oracle, grid, U, theta, emulate_bf16, ylim)
    Cx, Cy = fct_factors(U, U, Fx, Fy, dx_, dy_, dt, wx, wy)
    K = -div(Fx + Cx[None] * dx_, Fy + Cy[None] * dy_)
    U1 = U + dt * K
    Fx, Fy, dx_, dy_ = _corrections(oracle, grid, U1, theta, emulate_bf16, ylim)
    Ub = U + 0.5 * dt * K
    Cx, Cy = fct_factors(Ub, U1, Fx, Fy, dx_, dy_, 0.5 * dt, wx, wy)
    L2 = -div(Fx + Cx[None] * dx_, Fy + Cy[None] * dy_)
    return U + 0.5 * dt * (K + L2)
