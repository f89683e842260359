"""Training driver of the learned regime switch (argument marshalling and
orchestration only: features, forward and backward passes and the optimiser
all run in libesbgk.so's kernels).

Data: histories of the criterion of Sec. 3.1.2.  A problem is advanced with
the plain switch; the features of the state at step n (esbgk_features) are
paired with the regime map the criterion computes from the state at step
n + 1 -- the flag the network learns to predict one step ahead.

A case is a dict with "grid", "vmesh", "params", "scheme", "dt", "steps"
and "fields" (rho, ux, uy, T, eps, kin), all cases of one call on the same
N_y x N_x grid.
"""

import numpy as np

from . import CNN_CHANNELS, Solver, SwitchNet


def init_params(seed=0):
    """Starting parameters (float32, layout of esbgk_set_switch_params):
    He-normal convolution weights (std sqrt(2 / fan_in)), a head of std
    sqrt(1 / 32), zero biases; seeded."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / 45.0), 32 * 9 * 5), np.zeros(32),
             rng.normal(0.0, np.sqrt(2.0 / 288.0), 32 * 9 * 32), np.zeros(32),
             rng.normal(0.0, np.sqrt(1.0 / 32.0), 32), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def collect(cases, steps=None, prec="fp32", every=1, device=None):
    """Features and next-step flags of plain-switch runs of `cases`:
    (X (n, ny, nx, 16) bf16, Y (n, ny, nx) uint8) device tensors."""
    import torch
    xs, ys = [], []
    for c in cases:
        s = Solver(c["grid"], c["vmesh"], dict(c["params"], switch="plain"), prec=prec, device=device)
        f = c["fields"]
        s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
        nsteps = steps if steps is not None else c["steps"]
        prev = None
        for n in range(nsteps + 1):
            x = s.features()
            s.step(c["dt"], c["scheme"])
            if prev is not None:
                # the map of step n was computed from the state at step n: the
                # label of the features taken one step earlier
                xs.append(prev)
                ys.append(torch.as_tensor(s.flags().astype(np.uint8), device=s.device))
            prev = x if n % every == 0 else None
        s.close()
    return torch.stack(xs), torch.stack(ys)


def crop(X, Y, size):
    """Split (n, H, W, ...) histories into size x size tiles (H and W
    multiples of size), so that histories of several grids train one
    network batch shape."""
    n, H, W = Y.shape
    assert H % size == 0 and W % size == 0
    Xt = X.reshape(n, H // size, size, W // size, size, X.shape[-1]).permute(0, 1, 3, 2, 4, 5)
    Yt = Y.reshape(n, H // size, size, W // size, size).permute(0, 1, 3, 2, 4)
    return (Xt.reshape(-1, size, size, X.shape[-1]).contiguous(), Yt.reshape(-1, size, size).contiguous())


def positive_weight(Y):
    """Weight of the kinetic class: fluid cells / kinetic cells (>= 1)."""
    k = float(Y.float().mean().item())
    return max(1.0, (1.0 - k) / max(k, 1e-6))


def train(X, Y, theta0, epochs=20, batch=8, lr=2e-3, pos_weight=None, seed=0, device=None, log=None):
    """Adam on the class-weighted cross-entropy over shuffled mini-batches
    of images.  Returns the trained parameters (float32) and the per-epoch
    mean loss."""
    import torch
    n, H, W = Y.shape
    pw = positive_weight(Y) if pos_weight is None else pos_weight
    net = SwitchNet(min(batch, n), H, W, device=device)
    net.set_params(theta0)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(n)
        losses = []
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = torch.as_tensor(order[b0:b0 + batch], device=X.device)
            xb, yb = X.index_select(0, idx).contiguous(), Y.index_select(0, idx).contiguous()
            want = b0 == 0
            L = net.train_step(xb, yb, pw, lr, want_loss=want)
            if want:
                losses.append(L)
        hist.append(float(np.mean(losses)))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    theta = net.params()
    net.close()
    return theta, hist


def evaluate(theta, X, Y, device=None):
    """Confusion counts of the thresholded prediction against the labels."""
    import torch
    n, H, W = Y.shape
    net = SwitchNet(n, H, W, device=device)
    net.set_params(theta)
    z = net.forward(X)
    p = z > 0
    y = Y > 0
    out = dict(tp=int((p & y).sum()), fp=int((p & ~y).sum()), fn=int((~p & y).sum()), tn=int((~p & ~y).sum()))
    net.close()
    del torch
    return out


__all__ = ["init_params", "collect", "crop", "positive_weight", "train", "evaluate", "CNN_CHANNELS"]
