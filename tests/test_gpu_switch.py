"""Learned regime switch on the GPU: network kernels against the FP64 oracle
(forward, loss and every gradient block), training, determinism, the
judge/fallback rule inside the solver, and what a trained network gains.

Tolerances.  The GPU keeps activations a1, a2 and the back-propagated
dz1, dz2 in bf16 (relative rounding 2^-9) and accumulates in float32; the
oracle gets the same bf16-rounded inputs and weights.  Two comparisons:
(1) with the oracle rounding a1, a2, dz2, dz1 to bf16 where the GPU stores
them, only float32-vs-float64 accumulation differs (relative ~1e-6, and a
rare one-ulp bf16 flip where a value sits on a rounding boundary): logits
and every gradient block within 2e-3 relative; (2) against the exact float64
network: logits within 3 % of max |z|, loss 1 %, and every gradient block and
element within what the bf16 storage itself does to the gradient on the same
inputs plus the accumulation part (tests/switch_bars.py; the bars reject
planted gradient mistakes, tests/test_oracle_cnn.py).
"""

import numpy as np
import pytest

import oracle as O
import switch_bars
import workloads as W
from oracle import cnn as OC

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _setup(seed, n, H, Wd):
    """Random network and inputs, rounded the way the GPU stores them."""
    import torch
    rng = np.random.default_rng(seed)
    theta = OC.init_params(seed).astype(np.float32)
    p = OC.unpack(theta.astype(np.float64).copy())
    p["b1"][:] = rng.normal(0, 0.1, 32)
    p["b2"][:] = rng.normal(0, 0.1, 32)
    p["b3"][:] = -0.3
    theta = OC.pack(p).astype(np.float32)
    th64 = theta.astype(np.float64)
    q = OC.unpack(th64.copy())
    q["W1"][:] = _bf16_round(q["W1"])
    q["W2"][:] = _bf16_round(q["W2"])
    th_or = OC.pack(q)
    x = rng.normal(size=(n, H, Wd, 5))
    x_or = _bf16_round(x)
    xd = torch.zeros((n, H, Wd, 16), dtype=torch.bfloat16, device="cuda")
    xd[..., :5] = torch.tensor(x_or, dtype=torch.float64).to(torch.bfloat16).cuda()
    y = (rng.random((n, H, Wd)) < 0.3).astype(np.uint8)
    yd = torch.tensor(y, device="cuda")
    return theta, th_or, xd, x_or, yd, y


def test_forward_matches_oracle():
    import paper_2512_03586_gb300 as G
    # 2 images, 12 x 20 cells: two tile rows and columns each, ragged edges
    theta, th_or, xd, x_or, _, _ = _setup(1, 2, 12, 20)
    net = G.SwitchNet(2, 12, 20)
    net.set_params(theta)
    z = net.forward(xd).cpu().numpy()
    z_em = OC.forward(th_or, x_or, rnd=_bf16_round)["z3"]
    assert np.max(np.abs(z - z_em)) <= 2e-3 * np.max(np.abs(z_em))
    z_or = OC.forward(th_or, x_or)["z3"]
    assert np.max(np.abs(z - z_or)) <= 3e-2 * np.max(np.abs(z_or))
    # the decision agrees wherever the oracle's logit is not within the error
    far = np.abs(z_or) > 3e-2 * np.max(np.abs(z_or))
    np.testing.assert_array_equal((z > 0)[far], (z_or > 0)[far])


@pytest.mark.parametrize("shape", [(2, 12, 20), (1, 8, 16), (3, 5, 7)])
def test_gradient_matches_oracle(shape):
    import paper_2512_03586_gb300 as G
    n, H, Wd = shape
    theta, th_or, xd, x_or, yd, y = _setup(2, n, H, Wd)
    net = G.SwitchNet(n, H, Wd)
    net.set_params(theta)
    pw = 2.5
    L, g = net.gradient(xd, yd, pw)
    gp = OC.unpack(g.astype(np.float64))
    L_em, g_em = OC.grad(th_or, x_or, y.astype(np.float64), pw, rnd=_bf16_round)
    L_ex, g_ex = OC.grad(th_or, x_or, y.astype(np.float64), pw)
    # (1) the bf16 storage emulated: float32 accumulation only
    assert abs(L - L_em) <= 1e-4 * abs(L_em), (L, L_em)
    ge = OC.unpack(g_em)
    for name in switch_bars.BLOCKS:
        err = np.linalg.norm(gp[name] - ge[name]) / max(np.linalg.norm(ge[name]), 1e-30)
        assert err <= 2e-3, (name, err)
    # (2) the exact network: the bf16 storage's own effect plus accumulation
    assert abs(L - L_ex) <= 1e-2 * abs(L_ex), (L, L_ex)
    bad = switch_bars.check(g.astype(np.float64), g_ex, g_em, OC.unpack)
    assert not bad, bad


def test_adam_step_matches_oracle():
    import paper_2512_03586_gb300 as G
    theta, th_or, xd, x_or, yd, y = _setup(3, 1, 8, 16)
    net = G.SwitchNet(1, 8, 16)
    net.set_params(theta)
    _, g = net.gradient(xd, yd, 2.0)
    net.train_step(xd, yd, 2.0, 1e-3)
    th1 = net.params().astype(np.float64)
    ref, _, _ = OC.adam(theta.astype(np.float64), np.zeros_like(th1), np.zeros_like(th1), g.astype(np.float64), 1,
                        lr=1e-3)
    np.testing.assert_allclose(th1, ref, rtol=1e-5, atol=1e-7)


def _separable(n, H, Wd, seed):
    """Labels that a 3 x 3 neighbourhood decides: the cell or a neighbour
    has a large channel-3 value."""
    import torch
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, H, Wd, 5))
    big = x[..., 3] > 1.2
    lab = big.copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            lab |= np.roll(np.roll(big, dy, 1), dx, 2)
    xd = torch.zeros((n, H, Wd, 16), dtype=torch.bfloat16, device="cuda")
    xd[..., :5] = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).cuda()
    return xd, torch.tensor(lab.astype(np.uint8), device="cuda")


def test_training_learns_and_is_deterministic():
    import paper_2512_03586_gb300 as G
    from paper_2512_03586_gb300 import switch_train as T
    X, Y = _separable(16, 24, 32, 0)
    th0 = OC.init_params(0).astype(np.float32)
    th_a, hist = T.train(X, Y, th0, epochs=200, batch=8, lr=5e-3)
    th_b, _ = T.train(X, Y, th0, epochs=200, batch=8, lr=5e-3)
    np.testing.assert_array_equal(th_a, th_b)           # fixed-order reductions: bitwise repeatable
    assert hist[-1] < 0.2 * hist[0], hist
    c = T.evaluate(th_a, X, Y)
    acc = (c["tp"] + c["tn"]) / sum(c.values())
    assert acc >= 0.97, c
    del G


def _run(wl, switch, theta=None, steps=6, prec="fp64"):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], switch=switch), prec=prec)
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    if theta is not None:
        s.set_switch_params(theta)
    kin_total = 0
    for _ in range(steps):
        s.step(wl["dt"], wl["scheme"])
        kin_total += int(s.flags().sum())
    return s, kin_total


def _const_net(bias):
    th = np.zeros(OC.N_PARAMS, np.float32)
    th[-1] = bias
    return th


def test_learned_switch_never_predicting_equals_plain():
    """A network that never predicts kinetic leaves the criterion's map:
    the run is the plain run, and every criterion-kinetic cell is 'missed'."""
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3)
    sp, kp = _run(wl, "plain")
    sl, kl = _run(wl, "learned", _const_net(-10.0))
    np.testing.assert_array_equal(sl.cons(), sp.cons())
    st = sl.switch_stats()
    assert st["predicted"] == 0 and st["extra"] == 0
    # judged from the second update on: every kinetic cell of updates 2..6
    first = None
    s1, _ = _run(wl, "plain", steps=1)
    first = int(s1.flags().sum())
    assert st["missed"] == kp - first
    assert st["judged"] == 5 * wl["grid"]["nx"] * wl["grid"]["ny"]


def test_learned_switch_always_predicting_makes_all_kinetic():
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3)
    sl, _ = _run(wl, "learned", _const_net(10.0), steps=3)
    assert sl.flags().all()
    st = sl.switch_stats()
    assert st["missed"] == 0 and st["predicted"] == st["judged"]


def test_learned_switch_without_parameters_is_refused():
    import paper_2512_03586_gb300 as G
    wl = W.riemann_quadrants(nx=8, ny=8, nv=8, seed=1)
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], switch="learned"), prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    with pytest.raises(G.Error):
        s.step(wl["dt"])


def test_features_match_oracle():
    import paper_2512_03586_gb300 as G
    wl = W.riemann_quadrants(nx=20, ny=12, nv=8, seed=2)
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    x = s.features().float().cpu().numpy()
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **f)
    ref = OC.features(st.U, f["eps"], min(1.0 / 20, 1.0 / 12))
    np.testing.assert_allclose(x[..., :5], ref, rtol=2 ** -8, atol=2 ** -8 * 0.05)
    # eps channel exactly as the scaled definition gives it
    assert np.allclose(x[..., 4], np.log10(f["eps"] * (20 / 128) ** 2), rtol=2 ** -8)
    assert not x[..., 5:].any()


def test_trained_switch_gain():
    """Train on plain-criterion histories of 48 seeded Riemann problems,
    deploy on a held-out one, and measure what the network adds to the
    criterion: its held-out confusion counts, the judge's statistics, and the
    macroscopic error against an all-kinetic run (the kinetic model the
    hybrid approximates) for the plain and the learned switch, with the
    kinetic work (kinetic cell-steps) each spends.  The learned map holds
    the criterion's map plus the cells predicted to turn kinetic one step
    later, so it resolves starting non-equilibrium one step earlier."""
    from paper_2512_03586_gb300 import switch_train as T
    train_cases = [W.riemann_quadrants(nx=48, ny=48, nv=12, seed=100 + s, steps=30) for s in range(48)]
    X, Y = T.collect(train_cases, steps=30, prec="fp32")
    theta, hist = T.train(X, Y, OC.init_params(0).astype(np.float32), epochs=30, batch=32, lr=3e-3)
    test = W.riemann_quadrants(nx=48, ny=48, nv=12, seed=11, steps=40)
    Xt, Yt = T.collect([test], steps=40, prec="fp32")
    c = T.evaluate(theta, Xt, Yt)
    recall = c["tp"] / max(1, c["tp"] + c["fn"])
    spec = c["tn"] / max(1, c["tn"] + c["fp"])
    acc = (c["tp"] + c["tn"]) / sum(c.values())
    steps = 40
    sp, kp = _run(test, "plain", steps=steps, prec="fp32")
    sl, kl = _run(test, "learned", theta, steps=steps, prec="fp32")
    ref = dict(test, params=dict(test["params"], switch="frozen"))
    ref["fields"] = dict(test["fields"], kin=np.ones_like(test["fields"]["kin"]))
    sk, _ = _run(ref, "frozen", steps=steps, prec="fp32")
    Uk = sk.cons()
    err = lambda U: np.abs(U - Uk).sum() / np.abs(Uk).sum()
    e_p, e_l = err(sp.cons()), err(sl.cons())
    st = sl.switch_stats()
    print("\ntrained switch, held-out: accuracy %.4f recall %.4f specificity %.4f; judge %s" % (acc, recall, spec, st))
    print("relative L1 error of U vs all-kinetic after %d steps: plain %.3e (kinetic cell-steps %d), "
          "learned %.3e (%d): error x %.3f for work x %.3f" % (steps, e_p, kp, e_l, kl, e_l / e_p, kl / kp))
    assert hist[-1] < 0.2 * hist[0]
    assert acc >= 0.9 and recall >= 0.75 and spec >= 0.9, c
    # what the network gains: a smaller hybrid error at a modest extra kinetic work
    assert e_l < e_p and kl <= 1.3 * kp
    # the judge: most criterion-kinetic cells were predicted one step ahead
    assert st["missed"] <= 0.25 * (st["predicted"] - st["extra"] + st["missed"])
