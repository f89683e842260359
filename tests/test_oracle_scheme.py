"""Pins of the oracle's time stepper and regime switch (Sec. 3.1, 3.4-3.6, 4.1.1)."""

import itertools
import json
import os

import numpy as np
import pytest

from dataclasses import replace

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(wl, **kw):
    return O.Problem(**wl["grid"], **wl["vmesh"], **dict(wl["params"], **kw))


def test_ars233_satisfies_printed_coupled_order_conditions():
    """Sec. 3.4, Eqs. cond1-cond3, mixed2, mixed3 with Abar = At, bbar = bt
    (the paper's choice): every condition up to p = 3 holds for ARS(2,3,3)."""
    T = O.ARS233
    c, ct = T.A.sum(1), T.At.sum(1)
    bs = {"b": T.b, "bt": T.bt, "bb": T.bt}
    As = {"a": T.A, "at": T.At, "ab": T.At}
    cs = {"c": c, "ct": ct, "cb": ct}
    # c_i = sum_j a_ij consistent with the printed nodes (0, alpha, 1 - alpha)
    al = (3 + np.sqrt(3)) / 6
    assert np.allclose(c, [0, al, 1 - al]) and np.allclose(ct, [0, al, 1 - al])
    for b in bs.values():
        assert np.isclose(b.sum(), 1.0)
    for b, cc in itertools.product(bs.values(), cs.values()):
        assert np.isclose(b @ cc, 0.5)
    for b, A, cc in itertools.product(bs.values(), As.values(), cs.values()):
        assert np.isclose(b @ A @ cc, 1.0 / 6.0)
    for b, c1, c2 in itertools.product(bs.values(), cs.values(), cs.values()):
        assert np.isclose(np.sum(b * c1 * c2), 1.0 / 3.0)


@pytest.mark.parametrize("name", ["ARS222", "SSP2_332"])
def test_second_order_pairs_satisfy_coupled_conditions(name):
    """The other IMEX pairs: every coupled condition up to p = 2 holds
    (b.1 = 1, b.c = 1/2 for each part and across parts), and the third-order
    condition b.c^2 = 1/3 fails for at least one part (second order only);
    explicit part strictly lower triangular, implicit part lower triangular."""
    T = getattr(O, name)
    c, ct = T.A.sum(1), T.At.sum(1)
    assert np.allclose(np.triu(T.At), 0) and np.allclose(np.triu(T.A, 1), 0)
    for b in (T.b, T.bt):
        assert np.isclose(b.sum(), 1.0)
        for cc in (c, ct):
            assert np.isclose(b @ cc, 0.5)
    assert not all(np.isclose(np.sum(b * cc * cc), 1.0 / 3.0) for b in (T.b, T.bt) for cc in (c, ct))


@pytest.mark.parametrize("name", ["ARS222", "SSP2_332"])
def test_second_order_pairs_converge_at_second_order(name):
    """The coupled hybrid (Test 1 data, random frozen map, per-stage
    coupling) with the second-order pairs: Richardson order of the finest
    pair of step sizes within 0.3 of 2."""
    T = getattr(O, name)
    wl = W.order_test(n=12, nv=12, eps=1e-2)
    P = _prob(wl)
    sols = []
    for k in (4, 8, 16, 32):
        st = O.init_state(P, **wl["fields"])
        for _ in range(k):
            st = O.step(P, st, 0.2 / k, T)
        sols.append(st.U[0].copy())
    err = [np.sqrt(np.sum((a - b) ** 2)) for a, b in zip(sols[:-1], sols[1:])]
    order = np.log2(err[-2] / err[-1])
    assert abs(order - 2.0) <= 0.3, order


def test_density_tau_equals_scaled_constant_tau_at_uniform_density():
    """Reading R23: on a spatially uniform state (periodic, rho = 2 and the
    same anisotropic non-equilibrium f in every cell, no flow) the transport
    vanishes and the density stays 2, so
    tau = tau rho must give exactly the run with constant tau doubled; and the
    criterion's lambda_A with tau = tau rho equals the constant-tau one at
    2 tau."""
    prob = O.Problem(nx=6, ny=5, nv=12, vmax=6.0, switch="frozen")
    X, Y = prob.centres()
    rho = np.full(X.shape, 2.0)
    T = np.full(X.shape, 1.2)
    kin = np.ones(X.shape, bool)
    eps = np.full(X.shape, 0.05)
    st0 = O.init_state(prob, rho, 0 * rho, 0 * rho, T, eps, kin)
    v, w = O.velocity_grid(prob.nv, prob.vmax)
    VX, VY = np.meshgrid(v, v)
    st0.f = st0.f * (1.0 + 0.1 * (VX ** 2 - VY ** 2) / (1.0 + VX ** 2 + VY ** 2))[None, None]
    st0.f *= 2.0 / (w * st0.f.sum(axis=(-2, -1)))[..., None, None]  # keep rho = 2 exactly
    st0.U = np.stack([w * np.einsum("jkab,ab->jk", st0.f, q) for q in
                      (np.ones_like(VX), VX, VY, 0.5 * (VX ** 2 + VY ** 2))])
    outs = []
    for P in (replace(prob, tau_model="density", tau=0.7), replace(prob, tau=1.4)):
        st = st0
        for _ in range(3):
            st = O.step(P, st, 1e-2, O.ARS233)
        outs.append(st)
    np.testing.assert_allclose(outs[0].f, outs[1].f, rtol=1e-12, atol=1e-15)
    # the criterion on a shear flow with a temperature gradient at rho = 2
    shear = O.init_state(prob, rho, 0.3 * np.sin(2 * np.pi * Y), 0 * rho, 1.0 + 0.2 * np.cos(2 * np.pi * X), eps,
                         np.zeros(X.shape, bool))
    lam_d, _ = O.regime_indicators(replace(prob, tau_model="density", tau=0.7), shear)
    lam_c, _ = O.regime_indicators(replace(prob, tau=1.4), shear)
    assert lam_c.max() > 1e-3
    np.testing.assert_allclose(lam_d, lam_c, rtol=1e-12)


def test_imex_euler_is_first_order_only():
    T = O.IMEX_EULER
    assert np.isclose(T.b.sum(), 1) and np.isclose(T.bt.sum(), 1)
    assert not np.isclose(T.bt @ T.At.sum(1), 0.5)


def _random_kinetic_state(prob, seed):
    rng = np.random.default_rng(seed)
    X, Y = prob.centres()
    rho = 1 + 0.3 * np.sin(2 * np.pi * X + rng.uniform()) * np.cos(2 * np.pi * Y)
    ux = 0.2 * np.cos(2 * np.pi * Y + rng.uniform())
    uy = 0.1 * np.sin(2 * np.pi * X)
    T = 1 + 0.2 * np.cos(2 * np.pi * (X + Y))
    return rho, ux, uy, T


@pytest.mark.parametrize("kin_mode", ["kinetic", "euler"])
def test_periodic_single_model_conserves(kin_mode):
    """Flux-form transport and a conservative collision: with one model on a
    periodic grid mass, momentum and energy are conserved to round-off."""
    prob = O.Problem(nx=12, ny=10, nv=12, vmax=6.0, switch="frozen")
    rho, ux, uy, T = _random_kinetic_state(prob, 0)
    kin = np.full(rho.shape, kin_mode == "kinetic")
    st = O.init_state(prob, rho, ux, uy, T, np.full_like(rho, 1e-2), kin)
    t0 = O.totals(prob, st)
    for _ in range(3):
        st = O.step(prob, st, 2e-3, O.ARS233)
    t1 = O.totals(prob, st)
    assert np.allclose(t0, t1, rtol=0, atol=1e-13 * np.abs(t0).max())


@pytest.mark.parametrize("coupling", ["stage", "step"])
def test_conservative_interface_conserves_hybrid_totals(coupling):
    """Reading R22: with the kinetic flux's moments on both sides of every
    kinetic/fluid face, a periodic hybrid (random frozen map, flowing data)
    conserves mass, momentum and energy to round-off, as the single-model runs
    do; with each model's own flux (Reading R11) the same run drifts by orders
    of magnitude more."""
    prob = O.Problem(nx=12, ny=10, nv=12, vmax=6.0, switch="frozen", coupling=coupling)
    rho, ux, uy, T = _random_kinetic_state(prob, 1)
    kin = np.random.default_rng(3).random(rho.shape) < 0.5
    drift = {}
    for iface in ("own", "conservative"):
        P = replace(prob, interface=iface)
        st = O.init_state(P, rho, ux, uy, T, np.full_like(rho, 1e-2), kin)
        t0 = O.totals(P, st)
        for _ in range(3):
            st = O.step(P, st, 2e-3, O.ARS233)
        drift[iface] = np.abs(O.totals(P, st) - t0).max() / np.abs(t0).max()
    assert drift["conservative"] <= 1e-13, drift
    assert drift["own"] >= 1e4 * max(drift["conservative"], 1e-16), drift


def test_conservative_interface_changes_nothing_without_interfaces():
    """All-kinetic and all-fluid maps have no kinetic/fluid face: the two
    interface readings give bit-identical steps."""
    prob = O.Problem(nx=8, ny=6, nv=8, vmax=6.0, switch="frozen")
    rho, ux, uy, T = _random_kinetic_state(prob, 2)
    for k in (True, False):
        kin = np.full(rho.shape, k)
        out = []
        for iface in ("own", "conservative"):
            P = replace(prob, interface=iface)
            out.append(O.step(P, O.init_state(P, rho, ux, uy, T, np.full_like(rho, 1e-2), kin), 2e-3, O.ARS233))
        assert np.array_equal(out[0].U, out[1].U) and np.array_equal(out[0].f, out[1].f)


def test_flux_moments_of_a_maxwellian_face_flux():
    """The moments of the free-streaming flux v_x M of a Maxwellian with
    u = 0 on a symmetric fine velocity grid: the mass and x-energy fluxes
    vanish, the x-momentum flux is the pressure rho T (Sec. 2, gamma = 2)."""
    from oracle.transport import flux_moments
    v, w = O.velocity_grid(64, 10.0)
    rho, T = 1.3, 0.7
    VX, VY = np.meshgrid(v, v)
    M = rho / (2 * np.pi * T) * np.exp(-(VX ** 2 + VY ** 2) / (2 * T))
    G = flux_moments((VX * M)[None], v, w)[:, 0]
    assert abs(G[0]) < 1e-12 and abs(G[2]) < 1e-12 and abs(G[3]) < 1e-12
    assert abs(G[1] - rho * T) < 1e-10


@pytest.mark.parametrize("kin_fraction", [1.0, 0.0, 0.5])
def test_uniform_maxwellian_is_steady(kin_fraction):
    """A uniform Maxwellian state is an equilibrium of the full coupled step:
    L(const) = 0, Phi(const) = 0 and Q(M) = 0 (Sec. 2, H3)."""
    wl = W.order_test(n=8, nv=12, kin_fraction=kin_fraction, seed=3)
    prob = _prob(wl)
    f = dict(wl["fields"])
    f["rho"] = np.full_like(f["rho"], 1.2)
    f["T"] = np.full_like(f["rho"], 0.7)
    f["ux"] = np.full_like(f["rho"], 0.1)
    st = O.init_state(prob, **f)
    st1 = O.step(prob, st, 0.01, O.ARS233)
    assert np.max(np.abs(st1.U - st.U)) < 1e-13
    if st.kin.any():
        assert np.max(np.abs(st1.f[st.kin] - st.f[st.kin])) < 1e-14


def test_xy_symmetry_sine_periodic():
    """Symmetric data (sin 2 pi x sin 2 pi y, u = 0) on a symmetric velocity grid
    keeps the x <-> y reflection symmetry to round-off."""
    wl = W.sine_periodic(nx=12, ny=12, nv=10, steps=2)
    prob = _prob(wl)
    st = O.init_state(prob, **wl["fields"])
    for _ in range(2):
        st = O.step(prob, st, wl["dt"], O.IMEX_EULER)
    rho, ux, uy, T = O.macro(st)
    assert np.allclose(rho, rho.T, atol=1e-14)
    assert np.allclose(ux, uy.T, atol=1e-14)
    assert np.allclose(st.f, np.transpose(st.f, (1, 0, 3, 2)), atol=1e-14)


def _state_from_prim(prob, rho, ux, uy, T, eps, kin):
    return O.init_state(prob, rho, ux, uy, T, eps, kin)


def test_criterion_shear_flow_closed_form():
    """u = (a y, 0): grad u has a single entry a, D = [[0, a], [a, 0]] with
    eigenvalues +-a, so lambda_A = eps |a| / (tau (1 - beta)) (Eq. for S_1,
    mu/(rho T) = 1/(tau (1-beta)))."""
    prob = O.Problem(nx=6, ny=8, nv=8, vmax=5.0, bc_x="periodic", bc_y="outflow",
                     beta=-0.5, tau=1.3)
    X, Y = prob.centres()
    a = 0.7
    eps = np.full_like(X, 0.05)
    st = O.init_state(prob, np.ones_like(X), a * Y, 0 * X, np.ones_like(X), eps, np.zeros_like(X, bool))
    lamA, L1 = O.regime_indicators(prob, st)
    inner = lamA[1:-1]
    assert np.allclose(inner, 0.05 * a / (1.3 * 1.5), rtol=1e-12)
    assert np.all(L1 == 0)


def test_criterion_compression_closed_form():
    """u = (a x, 0), a one-dimensional compression or expansion: grad u =
    diag(a, 0), div u = a, D = diag(2a - 2/3 a, -2/3 a) = diag(4a/3, -2a/3)
    (Reading R8: the trace part -2/3 div u I), so lambda_A =
    (4/3) eps |a| / (tau (1 - beta)) in the interior cells."""
    prob = O.Problem(nx=8, ny=5, nv=8, vmax=5.0, bc_x="outflow", bc_y="periodic", beta=-0.5, tau=1.1)
    X, Y = prob.centres()
    eps = np.full_like(X, 0.04)
    for a in (0.6, -0.9):
        st = O.init_state(prob, np.ones_like(X), a * X, 0 * X, np.ones_like(X), eps, np.zeros_like(X, bool))
        lamA, _ = O.regime_indicators(prob, st)
        assert np.allclose(lamA[:, 1:-1], (4.0 / 3.0) * 0.04 * abs(a) / (1.1 * 1.5), rtol=1e-12)


def test_criterion_temperature_gradient_closed_form():
    """T = T0 + g x, u = 0: X = 2/3 (5/2 eps/(tau sqrt T))^2 grad T grad T^T has
    the single nonzero eigenvalue 2/3 (5/2 eps/(tau sqrt T))^2 g^2
    (kappa = 5/2 rho T / tau)."""
    prob = O.Problem(nx=8, ny=5, nv=8, vmax=5.0, bc_x="outflow", bc_y="periodic", tau=0.8)
    X, Y = prob.centres()
    g = 0.9
    T = 1.0 + g * X
    eps = np.full_like(X, 0.02)
    st = O.init_state(prob, np.ones_like(X), 0 * X, 0 * X, T, eps, np.zeros_like(X, bool))
    lamA, _ = O.regime_indicators(prob, st)
    expect = (2.0 / 3.0) * (2.5 * 0.02 / (0.8 * np.sqrt(T))) ** 2 * g ** 2
    assert np.allclose(lamA[:, 1:-1], expect[:, 1:-1], rtol=1e-12)


def test_criterion_zero_knudsen_gives_all_fluid():
    """Sec. 3.6: eps = 0 gives S_1 = S_0 = I, lambda_A = 0, so no cell is ever
    kinetic whatever the data."""
    wl = W.riemann_quadrants(nx=12, ny=12, nv=8, seed=1)
    prob = _prob(wl)
    f = dict(wl["fields"], eps=np.zeros((12, 12)))
    st = O.init_state(prob, **f)
    lamA, _ = O.regime_indicators(prob, st)
    assert np.all(lamA == 0)
    assert not O.regime_update(prob, st).any()


def test_regime_update_rules():
    """crit:CompEuler and eqKintoFluid1: a kinetic cell with lambda_A <= eta
    goes back to Euler only if ||f - M||_1 <= delta as well."""
    prob = O.Problem(nx=4, ny=4, nv=12, vmax=6.0, delta=1e-3, switch="plain")
    one = np.ones((4, 4))
    kin = np.zeros((4, 4), bool)
    kin[1, 1] = kin[2, 2] = True
    st = O.init_state(prob, one, 0 * one, 0 * one, one, 1e-3 * one, kin)
    # uniform flow: lambda_A = 0 everywhere; cell (2,2) gets a non-Maxwellian f
    v, w = O.velocity_grid(prob.nv, prob.vmax)
    VX, VY = np.meshgrid(v, v)
    st.f[2, 2] *= 1.0 + 0.2 * np.tanh(VX)
    lamA, L1 = O.regime_indicators(prob, st)
    assert L1[2, 2] > prob.delta and L1[1, 1] < 1e-12
    new = O.regime_update(prob, st)
    assert new[2, 2] and not new[1, 1] and new.sum() == 1


def test_l1_deviation_closed_form():
    """Reading R9: ||f - M_hat[f]||_1 with the quadrature weight dv^2 and the
    discrete Maxwellian of f's own moments.  f = M_hat + s g with g orthogonal
    (node sums) to 1, v_x, v_y, |v|^2 has the moments of M_hat, hence the same
    M_hat, so the deviation is exactly dv^2 sum |s g|."""
    prob = O.Problem(nx=3, ny=3, nv=14, vmax=6.0, switch="plain")
    one = np.ones((3, 3))
    kin = np.zeros((3, 3), bool)
    kin[1, 1] = True
    st = O.init_state(prob, 1.3 * one, 0.2 * one, -0.1 * one, 0.9 * one, 1e-3 * one, kin)
    v, w = O.velocity_grid(prob.nv, prob.vmax)
    VX, VY = np.meshgrid(v, v)
    B = np.stack([np.ones(VX.size), VX.ravel(), VY.ravel(), (VX ** 2 + VY ** 2).ravel()], 1)
    h = np.random.default_rng(4).standard_normal(VX.size)
    g = (h - B @ np.linalg.solve(B.T @ B, B.T @ h)).reshape(VX.shape)
    assert np.abs(B.T @ g.ravel()).max() < 1e-10
    s_amp = 1e-3
    st.f[1, 1] = st.f[1, 1] + s_amp * g
    _, L1 = O.regime_indicators(prob, st)
    expect = w * np.abs(s_amp * g).sum()
    assert L1[1, 1] == pytest.approx(expect, rel=1e-9)
    assert (np.abs(v[1] - v[0]) ** 2) == pytest.approx(w)


def test_regime_conversions_keep_the_cell_state():
    """Eqs. Coupling_FluKin / Coupling_KinFlu with Reading R4: a cell turned
    kinetic gets the discrete Maxwellian whose node moments are exactly its
    (rho, rho u, E) -- on a coarse grid, where a sampled continuous Maxwellian
    would miss them by ~1e-3 -- and a cell turned fluid takes the moments of
    its f."""
    prob = O.Problem(nx=4, ny=3, nv=10, vmax=5.0, switch="plain")
    X, Y = prob.centres()
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * X)
    ux, uy = 0.4 * np.cos(2 * np.pi * Y), -0.3 + 0 * X
    T = 0.8 + 0.5 * X
    kin0 = np.zeros(X.shape, bool)
    kin0[0, :2] = True
    st = O.init_state(prob, rho, ux, uy, T, 1e-3 + 0 * X, kin0)
    v, w = O.velocity_grid(prob.nv, prob.vmax)
    VX, VY = np.meshgrid(v, v)
    st.f[0, 0] *= 1.0 + 0.1 * np.tanh(VX - VY)          # a non-equilibrium kinetic cell
    new = ~kin0                                          # every cell switches
    out = O.convert(prob, st, new)

    def node_moments(g):
        return np.stack([w * (g * q).sum(axis=(-2, -1)) for q in
                         (np.ones_like(VX), VX, VY, 0.5 * (VX ** 2 + VY ** 2))])

    up = new & ~kin0
    np.testing.assert_allclose(node_moments(out.f[up]), st.U[:, up], rtol=1e-12, atol=1e-13)
    down = kin0 & ~new
    np.testing.assert_allclose(out.U[:, down], node_moments(st.f[down]), rtol=1e-12, atol=1e-13)
    # the sampled continuous Maxwellian would not do: its moments miss U here
    G = O.gaussian(rho[up], np.stack([ux[up], uy[up]], -1), T[up][:, None, None] * np.eye(2), v)
    assert np.abs(node_moments(G) - st.U[:, up]).max() > 1e-6


def test_buffer_mask_cross_stencil():
    """Remark rem_coupling: the buffer is the fluid part of the two-cell cross
    stencil of the kinetic cells."""
    kin = np.zeros((9, 9), bool)
    kin[4, 4] = True
    P = O.Problem(nx=9, ny=9)
    buf = O.buffer_mask(P, kin)
    assert buf.sum() == 8
    assert buf[4, 2] and buf[4, 6] and buf[2, 4] and buf[6, 4] and not buf[3, 3]
    kin = np.zeros((9, 9), bool)
    kin[0, 0] = True
    assert O.buffer_mask(P, kin).sum() == 8  # periodic wrap
    Po = O.Problem(nx=9, ny=9, bc_x="outflow", bc_y="outflow")
    assert O.buffer_mask(Po, kin).sum() == 4  # outflow: ghosts are the cell itself


def test_golden_table_orders_are_log2_error_ratios():
    """The printed orders of Tables tab:order_accuracy_* are log2 of successive
    error ratios (Eq. error_temporal, Richardson), up to the rounding of the
    printed errors."""
    g = json.load(open(os.path.join(GOLDEN, "test1_orders.json")))
    for eps, t in g["tables"].items():
        for kind in ("hoc", "loc"):
            e = np.array(t[kind + "_err"])
            o = np.log2(e[:-1] / e[1:])
            assert np.allclose(o, t[kind + "_order"], atol=0.2), (eps, kind, o)


def _richardson_orders(coupling, eps, n=16, nv=12, t_end=0.2, ks=(4, 8, 16, 32)):
    wl = W.order_test(n=n, nv=nv, eps=eps, coupling=coupling)
    prob = _prob(wl)
    sols = []
    for k in ks:
        st = O.init_state(prob, **wl["fields"])
        for _ in range(k):
            st = O.step(prob, st, t_end / k, O.ARS233)
        sols.append(st.U[0].copy())
    err = [np.sqrt(prob.dx * prob.dy * np.sum((a - b) ** 2)) for a, b in zip(sols[:-1], sols[1:])]
    return np.log2(np.array(err[:-1]) / np.array(err[1:]))


@pytest.mark.parametrize("eps", ["1e-2", "1e-6"])
def test_temporal_order_hoc_vs_loc(eps):
    """Test 1 (Sec. 4.1.1) on a reduced grid: with per-stage coupling the
    hybrid keeps ARS(2,3,3)'s third order; coupling only at step end (LOC)
    drops it to first.  The finest-pair orders fall in the ranges the paper
    prints (HOC 2.72-3.43, LOC 0.49-0.98, golden file)."""
    g = json.load(open(os.path.join(GOLDEN, "test1_orders.json")))["tables"][eps]
    hoc = _richardson_orders("stage", float(eps))
    loc = _richardson_orders("step", float(eps))
    assert min(g["hoc_order"]) - 0.3 <= hoc[-1] <= max(g["hoc_order"]) + 0.3, hoc
    assert min(g["loc_order"]) - 0.3 <= loc[-1] <= max(g["loc_order"]) + 0.3, loc


def test_stiff_limit_kinetic_approaches_euler():
    """eps -> 0: the all-kinetic solution approaches the all-Euler one (the
    hydrodynamic limit of Sec. 2); their difference shrinks under refinement."""
    diffs = []
    for n in (24, 48):
        prob = O.Problem(nx=1, ny=n, nv=14, vmax=7.0, bc_x="periodic", bc_y="periodic")
        y = (np.arange(n) + 0.5) / n
        rho = (1 + 0.2 * np.sin(2 * np.pi * y))[:, None]
        T = (1 + 0.1 * np.cos(2 * np.pi * y))[:, None]
        uy = (0.1 * np.sin(2 * np.pi * y))[:, None]
        eps = np.full_like(rho, 1e-6)
        t_end = 0.05
        steps = int(np.ceil(t_end / (0.5 / n / 7.0)))
        res = []
        for kin in (np.ones_like(rho, bool), np.zeros_like(rho, bool)):
            st = O.init_state(prob, rho, 0 * rho, uy, T, eps, kin)
            for _ in range(steps):
                st = O.advance(prob, st, t_end / steps, O.ARS233)
            res.append(st.U.copy())
        diffs.append(np.mean(np.abs(res[0] - res[1])))
    assert diffs[1] < diffs[0] and diffs[1] < 1e-3, diffs


def test_one_step_domain_of_dependence_is_six_cells():
    """Each ARS(2,3,3) stage reads the two-cell cross stencil of the previous
    stage values (CWENO3 faces, Sec. 3.2), so one step of a frozen all-kinetic
    problem at a cell depends on the cells within 6 of it and on no others: the
    run on the periodic window of radius 6 around a cell reproduces the full
    run there exactly, and radius 5 does not.  (This is what lets the GPU
    tests check sampled cells of full-size problems against the oracle.)"""
    from windows import window
    wl = W.gaussian_blob(nx=40, ny=36, nv=12, u0=(0.4, -0.3))
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    full = O.advance(P, O.init_state(P, **wl["fields"]), wl["dt"], O.ARS233).U
    for (j0, i0) in [(18, 20), (5, 33), (0, 0), (35, 39)]:
        for R in (6, 5):
            w = window(wl, j0, i0, R)
            Pw = O.Problem(**w["grid"], **w["vmesh"], **w["params"])
            Uw = O.advance(Pw, O.init_state(Pw, **w["fields"]), w["dt"], O.ARS233).U[:, R, R]
            d = np.abs(Uw - full[:, j0, i0]).max()
            if R == 6:
                assert d <= 1e-15 * np.abs(full[:, j0, i0]).max(), (j0, i0, d)
            elif (j0, i0) == (18, 20):
                assert d > 1e-10, d          # the blob's flank: cells at distance 6 matter


def _explicit_rk(y0, op, dt, At, bt):
    """Textbook explicit Runge-Kutta step (Butcher tableau At, bt) of y' = -op(y)."""
    ks = []
    for i in range(len(bt)):
        y = y0.copy()
        for j in range(i):
            y -= dt * At[i, j] * ks[j]
        ks.append(op(y))
    out = y0.copy()
    for i in range(len(bt)):
        out -= dt * bt[i] * ks[i]
    return out


@pytest.mark.parametrize("tab_name", ["ARS222", "IMEX_EULER", "ARS233"])
def test_collisionless_and_fluid_steps_are_the_explicit_rk(tab_name):
    """Sec. 3.4: the explicit part of the IMEX pair is (At, bt).  With the
    collisions switched off (eps -> infinity, nu ~ 1e-30) an all-kinetic step
    is the explicit RK step of the transport, and an all-fluid step is the
    explicit RK step of the Euler divergence -- in particular the final
    combination weights the fluxes by bt, not b (ARS(2,2,2) and IMEX-Euler
    have bt != b)."""
    tab = getattr(O, tab_name)
    wl = W.gaussian_blob(nx=10, ny=8, nv=10, vmax=6.0, u0=(0.4, -0.2))
    g = wl["grid"]
    dt = 0.02
    # all kinetic, no collisions
    P = O.Problem(**g, **wl["vmesh"], **dict(wl["params"], switch="frozen"))
    f = dict(wl["fields"], eps=np.full((8, 10), 1e30))
    st = O.init_state(P, **f)
    v, _ = O.velocity_grid(P.nv, P.vmax)
    args = (P.dx, P.dy, P.bc_x, P.bc_y, P.cweno_eps)
    ref = _explicit_rk(st.f, lambda y: O.kinetic_transport(y, v, *args), dt, tab.At, tab.bt)
    out = O.advance(P, st, dt, tab)
    assert np.abs(out.f - ref).max() <= 1e-13 * np.abs(ref).max()
    # all fluid
    f = dict(wl["fields"], kin=np.zeros((8, 10), bool))
    st = O.init_state(P, **f)
    ref = _explicit_rk(st.U, lambda y: O.euler_phi(y, *args), dt, tab.At, tab.bt)
    out = O.advance(P, st, dt, tab)
    assert np.abs(out.U - ref).max() <= 1e-13 * np.abs(ref).max()

