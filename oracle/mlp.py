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


def forward(theta, X):
    """X: [N, 24] -> (Y [N, 4], cache)."""
    P = unpack(theta)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = silu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = silu(z2)
    Y = h2 @ P["W3"].T + P["b3"]
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
