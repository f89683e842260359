"""Host logic of the learned-switch training driver (no GPU): tiling of
histories into training images, the class weight, the starting parameters'
layout against the oracle network's."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    from paper_2512_03586_gb300 import build as B
    B.build()
    from paper_2512_03586_gb300 import switch_train
    return switch_train


def test_crop_tiles_cover_every_image_once(T):
    n, H, W, C, s = 2, 8, 12, 3, 4
    X = torch.arange(n * H * W * C, dtype=torch.float32).reshape(n, H, W, C)
    Y = (torch.arange(n * H * W) % 7).reshape(n, H, W).to(torch.uint8)
    Xt, Yt = T.crop(X, Y, s)
    assert Xt.shape == (n * (H // s) * (W // s), s, s, C) and Yt.shape == (n * (H // s) * (W // s), s, s)
    k = 0
    for m in range(n):                       # brute force: image-major, then tile rows, then tile columns
        for a in range(H // s):
            for b in range(W // s):
                assert torch.equal(Xt[k], X[m, a * s:(a + 1) * s, b * s:(b + 1) * s])
                assert torch.equal(Yt[k], Y[m, a * s:(a + 1) * s, b * s:(b + 1) * s])
                k += 1
    with pytest.raises(AssertionError):
        T.crop(X, Y, 5)


def test_positive_weight_is_fluid_over_kinetic(T):
    Y = torch.zeros((1, 10, 10), dtype=torch.uint8)
    Y[0, :2] = 1                             # 20 % kinetic
    assert T.positive_weight(Y) == pytest.approx(4.0)
    assert T.positive_weight(torch.ones((1, 4, 4), dtype=torch.uint8)) == 1.0
    assert T.positive_weight(torch.zeros((1, 4, 4), dtype=torch.uint8)) >= 1e5


def test_init_params_layout_matches_the_network(T):
    from oracle import cnn as C
    th = T.init_params(0)
    assert th.dtype == np.float32 and th.size == C.init_params(0).size
    p = C.unpack(th.astype(np.float64))      # the oracle's order: W1, b1, W2, b2, w3, b3
    assert p["W1"].shape == (32, 3, 3, 5) and p["W2"].shape == (32, 3, 3, 32)
    for b in ("b1", "b2", "b3"):
        assert not p[b].any()
    # He-normal scales by fan-in (45 and 288 inputs), head 1/sqrt(32)
    assert p["W1"].std() == pytest.approx(np.sqrt(2 / 45), rel=0.1)
    assert p["W2"].std() == pytest.approx(np.sqrt(2 / 288), rel=0.05)
    assert np.array_equal(T.init_params(0), th) and not np.array_equal(T.init_params(1), th)
