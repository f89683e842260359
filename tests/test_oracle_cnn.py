"""Pins of the learned-switch oracle (oracle/cnn.py) against things other
than itself: torch's float64 conv2d and autograd (an independent library),
central finite differences of the loss, the closed form of the features and
the Adam update's first step."""

import numpy as np
import pytest

from oracle import cnn as C

torch = pytest.importorskip("torch")


def _case(seed=0, N=2, H=6, W=7):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(N, H, W, C.C_IN))
    y = (rng.random((N, H, W)) < 0.3).astype(np.float64)
    theta = C.init_params(seed)
    # non-zero biases so that every term of the chain rule is exercised
    p = C.unpack(theta.copy())
    p["b1"][:] = rng.normal(0, 0.1, C.C_HID)
    p["b2"][:] = rng.normal(0, 0.1, C.C_HID)
    p["b3"][:] = 0.2
    return C.pack(p), x, y


def _torch_forward(theta, x):
    p = {k: torch.tensor(v) for k, v in C.unpack(theta).items()}
    xt = torch.tensor(x).permute(0, 3, 1, 2)                        # N C H W
    w1 = p["W1"].permute(0, 3, 1, 2)                                # O I kh kw
    w2 = p["W2"].permute(0, 3, 1, 2)
    a1 = torch.relu(torch.nn.functional.conv2d(xt, w1, p["b1"], padding=1))
    a2 = torch.relu(torch.nn.functional.conv2d(a1, w2, p["b2"], padding=1))
    z3 = torch.einsum("nchw,c->nhw", a2, p["w3"]) + p["b3"][0]
    return z3


def test_forward_matches_torch_conv2d():
    theta, x, _ = _case(1)
    z_or = C.forward(theta, x)["z3"]
    z_t = _torch_forward(theta, x).numpy()
    np.testing.assert_allclose(z_or, z_t, rtol=1e-12, atol=1e-12)


def test_gradient_matches_torch_autograd():
    theta, x, y = _case(2)
    pw = 2.5
    L, g = C.grad(theta, x, y, pw)
    th = torch.tensor(theta, requires_grad=True)
    # rebuild the network from the flat vector so autograd sees the packing
    parts, o = {}, 0
    for name, shp in C.SHAPES:
        n = int(np.prod(shp))
        parts[name] = th[o:o + n].reshape(shp)
        o += n
    xt = torch.tensor(x).permute(0, 3, 1, 2)
    a1 = torch.relu(torch.nn.functional.conv2d(xt, parts["W1"].permute(0, 3, 1, 2), parts["b1"], padding=1))
    a2 = torch.relu(torch.nn.functional.conv2d(a1, parts["W2"].permute(0, 3, 1, 2), parts["b2"], padding=1))
    z = torch.einsum("nchw,c->nhw", a2, parts["w3"]) + parts["b3"][0]
    yt = torch.tensor(y)
    w = torch.where(yt > 0.5, torch.tensor(pw, dtype=torch.float64), torch.tensor(1.0, dtype=torch.float64))
    Lt = torch.mean(w * torch.nn.functional.binary_cross_entropy_with_logits(z, yt, reduction="none"))
    Lt.backward()
    assert abs(L - Lt.item()) <= 1e-12 * abs(L)
    np.testing.assert_allclose(g, th.grad.numpy(), rtol=1e-9, atol=1e-13)


def test_gradient_matches_finite_differences():
    theta, x, y = _case(3, N=1, H=5, W=5)
    pw = 3.0
    _, g = C.grad(theta, x, y, pw)
    rng = np.random.default_rng(0)
    # a sample of every parameter block
    offs, o = [], 0
    for _, shp in C.SHAPES:
        n = int(np.prod(shp))
        offs += list(o + rng.choice(n, size=min(n, 6), replace=False))
        o += n
    h = 1e-6
    for k in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (C.loss(tp, x, y, pw) - C.loss(tm, x, y, pw)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])), (k, fd, g[k])


def test_conv_of_centre_tap_is_a_matmul():
    """A kernel with only the centre tap is a per-cell linear map."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 4, 5, 3))
    Wt = np.zeros((2, 3, 3, 3))
    Wt[:, 1, 1, :] = rng.normal(size=(2, 3))
    b = rng.normal(size=2)
    np.testing.assert_allclose(C.conv3x3(x, Wt, b), x @ Wt[:, 1, 1, :].T + b, rtol=1e-14)


def test_features_closed_form():
    rho = np.array([[1.0, 0.5]])
    ux = np.array([[0.3, -0.2]])
    uy = np.array([[0.0, 0.1]])
    T = np.array([[2.0, 0.25]])
    U = np.stack([rho, rho * ux, rho * uy, 0.5 * rho * (ux ** 2 + uy ** 2) + rho * T])
    eps = np.array([[1e-2, 1e-4]])
    # on the reference grid: (log rho, u, log T, log10 eps)
    F = C.features(U, eps, 1.0 / 128)
    np.testing.assert_allclose(F[..., 0], np.log(rho))
    np.testing.assert_allclose(F[..., 1], ux, atol=1e-15)
    np.testing.assert_allclose(F[..., 2], uy, atol=1e-15)
    np.testing.assert_allclose(F[..., 3], np.log(T), atol=1e-14)
    np.testing.assert_allclose(F[..., 4], [[-2.0, -4.0]], atol=1e-14)
    # four times finer: velocities x 4, eps x 16
    F4 = C.features(U, eps, 1.0 / 512)
    np.testing.assert_allclose(F4[..., 1], 4 * ux, atol=1e-15)
    np.testing.assert_allclose(F4[..., 4], [[np.log10(0.16), np.log10(0.0016)]], atol=1e-14)


def test_features_see_the_criterion_the_same_on_every_grid():
    """The criterion of Sec. 3.1.2 on a linear velocity and temperature
    profile, sampled on two grids: the same physical state gives the same
    neighbour differences of the scaled velocity channel and the same
    eps-channel-weighted temperature term."""
    def state(n):
        x = (np.arange(n) + 0.5) / n
        X = np.tile(x, (3, 1))
        ux = 0.2 * X
        T = 1.0 + 0.5 * X
        rho = np.ones_like(X)
        U = np.stack([rho, rho * ux, 0 * ux, 0.5 * rho * ux ** 2 + rho * T])
        return C.features(U, np.full_like(X, 1e-3), 1.0 / n)
    for n in (128, 512):
        F = state(n)
        dux = (F[1, 2, 1] - F[1, 0, 1]) / 2          # per-cell difference of s u_x
        assert abs(dux - 0.2 / 128) <= 1e-12          # = dx_ref * du/dx on every grid
        s2eps = 10 ** F[1, 1, 4]                      # eps s^2
        dT = (np.exp(F[1, 2, 3]) - np.exp(F[1, 0, 3])) / 2
        # eps (dT/dx)^2 in reference units: eps s^2 (per-cell dT)^2 / dx_ref^2
        assert abs(s2eps * dT ** 2 * 128 ** 2 - 1e-3 * 0.25) <= 1e-9


def test_adam_first_step_is_signed_lr():
    """With m = v = 0, the first Adam step moves each weight by lr sign(g)
    (up to eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = C.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_learned_map_keeps_every_plain_kinetic_cell():
    rng = np.random.default_rng(5)
    plain = rng.random((8, 8)) < 0.3
    pred = rng.random((8, 8)) < 0.3
    m = C.learned_map(plain, pred)
    assert np.all(m[plain]) and np.all(m[pred]) and not np.any(m[~plain & ~pred])


# ---------------------------------------------------------------------------
# The GPU gradient bars (tests/switch_bars.py) catch plausible kernel mistakes.

GRAD_MISTAKES = [
    ('dz2 = rnd(da2 * (f["z2"] > 0))', 'dz2 = rnd(da2)', "second ReLU mask dropped"),
    ('g["b1"] = dz1.sum(axis=(0, 1, 2))', 'g["b1"] = dz1[:, 1:-1, 1:-1].sum(axis=(0, 1, 2))',
     "first bias gradient without the image edges"),
    ('g["W1"][:, ky, kx, :] = np.einsum("nyxo,nyxc->oc", dz1, _shift(f["x"], ky - 1, kx - 1))',
     'g["W1"][:, ky, kx, :] = np.einsum("nyxo,nyxc->oc", dz1, _shift(f["x"], 1 - ky, 1 - kx))',
     "first weight gradient with the taps mirrored"),
    ('"w3": np.einsum("nyx,nyxc->c", dz3, f["a2"])}', '"w3": np.einsum("nyx,nyxc->c", (sig - y) / M, f["a2"])}',
     "head gradient without the class weight"),
    ('da1 += np.einsum("nyxo,oc->nyxc", _shift(dz2, 1 - ky, 1 - kx), p["W2"][:, ky, kx, :])',
     'da1 += np.einsum("nyxo,oc->nyxc", _shift(dz2, ky - 1, kx - 1), p["W2"][:, ky, kx, :])',
     "input gradient of the second convolution with the taps mirrored"),
]


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("old,new,what", GRAD_MISTAKES, ids=[m[2] for m in GRAD_MISTAKES])
def test_gpu_gradient_bars_reject_planted_mistakes(tmp_path, old, new, what):
    """Each mistake is planted in a temporary copy of this oracle and its
    gradient computed the way the GPU stores values (bf16 a1, a2, dz2, dz1):
    the bars the GPU gradient must meet reject it on some block, while the
    unmutated bf16 emulation meets them."""
    import importlib.util
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import switch_bars
    src = open(C.__file__).read()
    assert src.count(old) == 1, old
    path = tmp_path / "cnn_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("cnn_mutant", str(path))
    mut = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mut)
    rng = np.random.default_rng(7)
    p = C.unpack(C.init_params(7))
    p["b1"][:] = rng.normal(0, 0.1, 32)
    p["b2"][:] = rng.normal(0, 0.1, 32)
    p["b3"][:] = -0.3
    p["W1"][:] = _bf16(p["W1"])
    p["W2"][:] = _bf16(p["W2"])
    theta = C.pack(p)
    x = _bf16(rng.normal(size=(2, 12, 20, 5)))
    y = (rng.random((2, 12, 20)) < 0.3).astype(np.float64)
    _, g_exact = C.grad(theta, x, y, 2.5)
    _, g_emu = C.grad(theta, x, y, 2.5, rnd=_bf16)
    assert not switch_bars.check(g_emu, g_exact, g_emu, C.unpack)
    _, g_bad = mut.grad(theta, x, y, 2.5, rnd=_bf16)
    assert switch_bars.check(g_bad, g_exact, g_emu, C.unpack), what
