"""FP64 CPU oracle of the learned regime switch (TEST INFRASTRUCTURE ONLY).

The paper decides the regime of every cell with the criteria of Sec. 3.1.2
(lambda_A > eta, or kinetic and ||f - M||_1 > delta).  The learned switch is an
addition to the method: a small convolutional network that reads the
macroscopic state of a 5 x 5 neighbourhood of a cell at step n and predicts the
flag the paper's criterion will give the cell at step n + 1.  The criterion
itself stays in charge: the map used for a step is the criterion's map united
with the network's prediction, so a cell the criterion marks kinetic is never
handed to the fluid solver.  This module is the plain reference of every piece
of that addition; it shares nothing with the CUDA path.

Network (3 layers, receptive field 5 x 5 cells):
  x   : (N, H, W, 5) features of each cell (``features``)
  z1  = b1 + conv3x3(x, W1)      a1 = relu(z1)      32 channels
  z2  = b2 + conv3x3(a1, W2)     a2 = relu(z2)      32 channels
  z3  = b3 + a2 . w3                                  1 channel (the logit)
conv3x3(x, W)[n, y, x, o] = sum_{dy, dx in {-1,0,1}} sum_c
    W[o, dy+1, dx+1, c] x[n, y+dy, x+dx, c], zero outside the image ('same'
zero padding).  The predicted flag is z3 > 0 (probability above one half).

Loss: class-weighted binary cross-entropy averaged over cells,
  L = (1/M) sum_i w_i [softplus(z_i) - y_i z_i],  w_i = pos_weight if y_i = 1
  else 1, the usual weighting when the positive class (kinetic) is rare.

Parameter vector (float64, this order): W1 (32,3,3,5), b1 (32), W2 (32,3,3,32),
b2 (32), w3 (32), b3 (1); 10753 values.

Pinned in tests/test_oracle_cnn.py: the forward pass against
torch.nn.functional.conv2d in float64 (an independent library routine), the
gradients against central finite differences of the loss and against torch
autograd, the features against their closed form.
"""

import numpy as np

C_IN, C_HID = 5, 32
SHAPES = (("W1", (C_HID, 3, 3, C_IN)), ("b1", (C_HID,)), ("W2", (C_HID, 3, 3, C_HID)), ("b2", (C_HID,)),
          ("w3", (C_HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Parameter vector -> dict of arrays (views)."""
    theta = np.asarray(theta, np.float64)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed=0):
    """He-style random initialisation (the starting point of training)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(2.0 / (9 * C_IN)), (C_HID, 3, 3, C_IN)),
         "b1": np.zeros(C_HID),
         "W2": rng.normal(0, np.sqrt(2.0 / (9 * C_HID)), (C_HID, 3, 3, C_HID)),
         "b2": np.zeros(C_HID),
         "w3": rng.normal(0, np.sqrt(1.0 / C_HID), C_HID),
         "b3": np.zeros(1)}
    return pack(p)


DX_REF = 1.0 / 128.0


def features(U, eps, dx, dx_ref=DX_REF):
    """Input channels of a cell from the conserved variables U (4, H, W)
    (rho, rho u_x, rho u_y, E with E = rho |u|^2 / 2 + rho T, Sec. 2 with
    d_v = 2), the Knudsen number eps (H, W) and the cell size dx:
      (log rho, s u_x, s u_y, log T, log10(eps s^2)),  s = dx_ref / dx.
    Reading: the criterion of Sec. 3.1.2 divided by eps depends on the
    velocity jumps between neighbours through D ~ (jump of u) / (2 dx) and on
    the temperature jumps through eps (jump of T / (2 dx))^2 / T.  With
    velocities scaled by s, neighbour differences of s u are 2 dx_ref D; with
    eps scaled by s^2, the temperature term is the same function of the
    channels at every grid spacing.  So a network trained on one grid sees
    the same inputs for the same physical state on a finer one.  At
    dx = dx_ref (the 128 x 128 grid of the unit square) the channels are
    (log rho, u_x, u_y, log T, log10 eps)."""
    s = dx_ref / dx
    rho = U[0]
    ux, uy = U[1] / rho, U[2] / rho
    T = (U[3] - 0.5 * rho * (ux * ux + uy * uy)) / rho
    return np.stack([np.log(rho), s * ux, s * uy, np.log(T), np.log10(eps * s * s)], axis=-1)


def _shift(x, dy, dx):
    """out[n, y, x] = x[n, y + dy, x + dx] with zeros outside the image."""
    N, H, W = x.shape[:3]
    out = np.zeros_like(x)
    ys, yd = slice(max(0, dy), H + min(0, dy)), slice(max(0, -dy), H + min(0, -dy))
    xs, xd = slice(max(0, dx), W + min(0, dx)), slice(max(0, -dx), W + min(0, -dx))
    out[:, yd, xd] = x[:, ys, xs]
    return out


def conv3x3(x, Wt, b):
    """'same' 3 x 3 convolution with zero padding: x (N,H,W,Ci), Wt (Co,3,3,Ci)."""
    out = np.zeros(x.shape[:3] + (Wt.shape[0],))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("nyxc,oc->nyxo", _shift(x, ky - 1, kx - 1), Wt[:, ky, kx, :])
    return out + b


def _keep(a):
    return a


def forward(theta, x, rnd=None):
    """All activations of the network for inputs x (N, H, W, 5).

    rnd: optional rounding applied to the stored activations a1, a2, for
    comparison with an implementation that stores them in a narrower type
    (bf16); None keeps float64 throughout."""
    rnd = rnd or _keep
    p = unpack(theta)
    x = np.asarray(x, np.float64)
    z1 = conv3x3(x, p["W1"], p["b1"])
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = conv3x3(a1, p["W2"], p["b2"])
    a2 = rnd(np.maximum(z2, 0.0))
    z3 = a2 @ p["w3"] + p["b3"][0]
    return dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3)


def predict(theta, x):
    """Predicted next-step kinetic flags: logit > 0."""
    return forward(theta, x)["z3"] > 0.0


def loss(theta, x, y, pos_weight):
    z = forward(theta, x)["z3"]
    y = np.asarray(y, np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    return float(np.mean(w * (np.logaddexp(0.0, z) - y * z)))


def grad(theta, x, y, pos_weight, rnd=None):
    """(loss, gradient vector) by the chain rule through the layers above.

    dL/dz3 = w (sigmoid(z3) - y) / M; the 1 x 1 head gives dL/dw3 = sum a2 dz3
    and dL/da2 = dz3 w3; relu passes the gradient where z > 0; a 'same'
    zero-padded convolution z = conv3x3(a, W) gives
      dL/dW[o, ky, kx, c] = sum_{n,y,x} dz[n,y,x,o] a[n, y+ky-1, x+kx-1, c],
      dL/da[n,y,x,c]      = sum_{ky,kx,o} dz[n, y-ky+1, x-kx+1, o] W[o,ky,kx,c],
      dL/db[o]            = sum dz[..., o].
    rnd: as in ``forward``, applied also to the stored gradients dz2, dz1."""
    rnd = rnd or _keep
    p = unpack(theta)
    f = forward(theta, x, rnd)
    y = np.asarray(y, np.float64)
    M = y.size
    w = np.where(y > 0.5, pos_weight, 1.0)
    z3 = f["z3"]
    L = float(np.mean(w * (np.logaddexp(0.0, z3) - y * z3)))
    sig = 0.5 * (1.0 + np.tanh(0.5 * z3))
    dz3 = w * (sig - y) / M
    g = {"b3": np.array([dz3.sum()]), "w3": np.einsum("nyx,nyxc->c", dz3, f["a2"])}
    da2 = dz3[..., None] * p["w3"]
    dz2 = rnd(da2 * (f["z2"] > 0))
    g["b2"] = dz2.sum(axis=(0, 1, 2))
    g["W2"] = np.zeros_like(p["W2"])
    da1 = np.zeros_like(f["a1"])
    for ky in range(3):
        for kx in range(3):
            g["W2"][:, ky, kx, :] = np.einsum("nyxo,nyxc->oc", dz2, _shift(f["a1"], ky - 1, kx - 1))
            da1 += np.einsum("nyxo,oc->nyxc", _shift(dz2, 1 - ky, 1 - kx), p["W2"][:, ky, kx, :])
    dz1 = rnd(da1 * (f["z1"] > 0))
    g["b1"] = dz1.sum(axis=(0, 1, 2))
    g["W1"] = np.zeros_like(p["W1"])
    for ky in range(3):
        for kx in range(3):
            g["W1"][:, ky, kx, :] = np.einsum("nyxo,nyxc->oc", dz1, _shift(f["x"], ky - 1, kx - 1))
    return L, pack(g)


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), step t >= 1.  Returns theta, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def learned_map(plain_flags, predicted_flags):
    """Regime map of a step under the learned switch: the criterion's map of
    Sec. 3.1.2 united with the network's prediction for the next step (the
    criterion is the fallback: its kinetic cells always stay kinetic)."""
    return np.asarray(plain_flags, bool) | np.asarray(predicted_flags, bool)
