"""Pins of the oracle's spatial operators (Sec. 3.2): CWENO3, the kinetic
transport L(f) and the Euler divergence Phi(U)."""

import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

import oracle as O
from riemann_exact import exact_riemann_density


def test_cweno_linear_and_constant_data_exact():
    """Every sub-polynomial reproduces a line, so any weights give the exact
    face values of linear data; constants are kept."""
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(2, 50))
    for eps_w in (1e-6, 1.0, 1e-30):
        L, R = O.cweno3_faces(a - b, a, a + b, eps_w)
        assert np.allclose(L, a - 0.5 * b, atol=1e-14)
        assert np.allclose(R, a + 0.5 * b, atol=1e-14)


def test_cweno_linear_weights_give_optimal_parabola():
    """With eps_w -> infinity the weights are the linear ones and the
    reconstruction is P_opt, exact at the faces for cell averages of any
    quadratic (this fixes P_opt and the definition of P_0)."""
    rng = np.random.default_rng(1)
    c = rng.normal(size=(3, 20))
    p = [Poly(c[:, k]) for k in range(20)]

    def avg(P, lo, hi):
        I = P.integ()
        return (I(hi) - I(lo)) / (hi - lo)

    qm = np.array([avg(P, -1.5, -0.5) for P in p])
    q0 = np.array([avg(P, -0.5, 0.5) for P in p])
    qp = np.array([avg(P, 0.5, 1.5) for P in p])
    L, R = O.cweno3_faces(qm, q0, qp, 1e40)
    assert np.allclose(L, [P(-0.5) for P in p], atol=1e-12)
    assert np.allclose(R, [P(0.5) for P in p], atol=1e-12)


def test_cweno_indicators_are_jiang_shu_integrals():
    """IS_k = sum_l int_{-1/2}^{1/2} (d^l P_k/ds^l)^2 ds for P_L, P_R and
    P_0 = (P_opt - P_L/4 - P_R/4)/(1/2), evaluated by polynomial calculus."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        qm, q0, qp = rng.normal(size=3)
        PL = Poly([q0, q0 - qm])
        PR = Poly([q0, qp - q0])
        D = qp - 2 * q0 + qm
        Popt = Poly([q0 - D / 24, (qp - qm) / 2, D / 2])
        P0 = (Popt - 0.25 * PL - 0.25 * PR) / 0.5

        def js(P):
            tot = 0.0
            for l in (1, 2):
                d = P.deriv(l) if P.degree() >= l else Poly([0.0])
                I = (d * d).integ()
                tot += I(0.5) - I(-0.5)
            return tot

        IS0, ISL, ISR = O.cweno3_indicators(qm, q0, qp)
        assert np.isclose(IS0, js(P0), rtol=1e-12, atol=1e-14)
        assert np.isclose(ISL, js(PL), rtol=1e-12, atol=1e-14)
        assert np.isclose(ISR, js(PR), rtol=1e-12, atol=1e-14)


def test_cweno_picks_smooth_substencil():
    """With eps_w ~ 0 a constant left (right) sub-stencil takes all the weight:
    IS_L = (q0 - qm)^2 (IS_R = (qp - q0)^2) is what vanishes."""
    L, R = O.cweno3_faces(np.array(1.0), np.array(1.0), np.array(5.0), 1e-100)
    assert np.isclose(L, 1.0) and np.isclose(R, 1.0)
    L, R = O.cweno3_faces(np.array(5.0), np.array(1.0), np.array(1.0), 1e-100)
    assert np.isclose(L, 1.0) and np.isclose(R, 1.0)


def _cell_avg_sin(xc, h, k=1):
    # average of sin(2 pi k x) over [xc - h/2, xc + h/2]
    return np.sin(2 * np.pi * k * xc) * np.sin(np.pi * k * h) / (np.pi * k * h)


def test_cweno_third_order_on_smooth_data():
    """Face values of smooth data converge at (about) third order in L1."""
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        q = 1.5 + _cell_avg_sin(xc, h)
        qe = O.pad_cells(q, 0, "periodic")
        L, R = O.cweno3_faces(qe[1:n + 1], qe[2:n + 2], qe[3:n + 3], 1e-6)
        exact_R = 1.5 + np.sin(2 * np.pi * (xc + h / 2))
        errs.append(np.mean(np.abs(R - exact_R)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 2.5, (errs, orders)


def test_kinetic_transport_consistency_and_order():
    """L(f) approximates v . grad f in both directions and for both signs of v:
    for cell averages of a smooth periodic profile the error of L against the
    exact face-difference quotient falls at second order in L1 (third-order
    face values; CWENO3 with a fixed eps_w loses one order at smooth extrema,
    which shows in the max norm)."""
    nv, vmax = 4, 1.0
    v, w = O.velocity_grid(nv, vmax)
    errs = []
    for n in (32, 64):
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        ax = _cell_avg_sin(xc, h)
        ay = _cell_avg_sin(xc, h, 2)
        f = np.broadcast_to((2.0 + ax[None, :] * ay[:, None])[:, :, None, None], (n, n, nv, nv)).copy()
        L = O.kinetic_transport(f, v, h, h, "periodic", "periodic", 1e-6)
        # exact: v_x d/dx + v_y d/dy of the cell average
        dfx = (np.sin(2 * np.pi * (xc + h / 2)) - np.sin(2 * np.pi * (xc - h / 2))) / h
        gx = dfx[None, :] * ay[:, None]
        gy = ax[None, :] * (np.sin(4 * np.pi * (xc + h / 2)) - np.sin(4 * np.pi * (xc - h / 2)))[:, None] / h
        exact = v[None, None, None, :] * gx[:, :, None, None] + v[None, None, :, None] * gy[:, :, None, None]
        errs.append(np.mean(np.abs(L - exact)))
    assert np.log2(errs[0] / errs[1]) > 1.8, errs


def test_free_transport_matches_exact_shift():
    """nu -> 0 (eps huge): the kinetic step is pure free transport; after time t
    the cell averages equal those of f0(x - v t), with an L1 error falling at
    (at least) second order -- this fixes the upwind direction of the flux."""
    nv, vmax = 4, 1.0
    v, w = O.velocity_grid(nv, vmax)
    errs = []
    t_end = 0.25
    for n in (16, 32):
        prob = O.Problem(nx=n, ny=n, nv=nv, vmax=vmax, switch="frozen")
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h

        def prof(sx, sy):
            return 2.0 + _cell_avg_sin(xc - sx, h)[None, :] * _cell_avg_sin(xc - sy, h)[:, None]

        f0 = np.empty((n, n, nv, nv))
        for a in range(nv):
            for b in range(nv):
                f0[:, :, a, b] = prof(0, 0) * (1.0 + 0.1 * a + 0.05 * b)
        U = np.moveaxis(O.cons_from_moments(O.moments(f0, v, w)), -1, 0)
        st = O.State(f=f0, U=U.copy(), kin=np.ones((n, n), bool), eps=np.full((n, n), 1e14))
        steps = 4 * n // 8
        dt = t_end / steps
        for _ in range(steps):
            st = O.advance(prob, st, dt, O.ARS233)
        err = 0.0
        for a in range(nv):
            for b in range(nv):
                ex = prof(v[b] * t_end, v[a] * t_end) * (1.0 + 0.1 * a + 0.05 * b)
                err += np.mean(np.abs(st.f[:, :, a, b] - ex)) / nv ** 2
        errs.append(err)
    assert errs[1] < 0.02
    assert np.log2(errs[0] / errs[1]) > 1.6, errs


def test_euler_constant_state_is_steady():
    U = np.empty((4, 6, 7))
    U[0], U[1], U[2], U[3] = 1.3, 0.4, -0.2, 2.0
    for bc in ("periodic", "outflow"):
        P = O.euler_phi(U, 0.1, 0.2, bc, bc, 1e-6)
        assert np.max(np.abs(P)) < 1e-13


def test_euler_sod_converges_to_exact_riemann_solution():
    """Test 2 setting (Sec. 4.1.2) on the Euler part alone: Sod data along y,
    (rho, u, p) = (1, 0, 1) | (1/8, 0, 1/32), gamma = 2 (d_v = 2), compared
    with the exact Riemann solution at t = 0.15; the L1 error decreases under
    refinement."""
    errs = []
    for n in (100, 200):
        prob = O.Problem(nx=1, ny=n, x0=0, x1=0.1, y0=0, y1=1, bc_x="periodic", bc_y="outflow",
                         nv=4, vmax=8.0, switch="frozen")
        y = (np.arange(n) + 0.5) / n
        rho = np.where(y <= 0.5, 1.0, 0.125)[:, None]
        p = np.where(y <= 0.5, 1.0, 1.0 / 32)[:, None]
        st = O.init_state(prob, rho, 0 * rho, 0 * rho, p / rho, np.full_like(rho, 1e-6),
                          kin=np.zeros_like(rho, bool))
        t_end = 0.15
        steps = int(np.ceil(t_end / (0.4 / n / 2.0)))
        for _ in range(steps):
            st = O.advance(prob, st, t_end / steps, O.ARS233)
        r = O.macro(st)[0][:, 0]
        ex = exact_riemann_density(1.0, 0.0, 1.0, 0.125, 0.0, 1.0 / 32, 2.0, (y - 0.5) / t_end)
        errs.append(np.mean(np.abs(r - ex)))
    assert errs[1] < errs[0] and errs[1] < 0.01, errs


def test_exact_riemann_helper_reproduces_the_published_sod_star_state():
    """The exact Riemann solution used as the Sod reference is pinned to the
    published exact values of the classic Sod problem at gamma = 1.4 (Toro,
    Riemann Solvers and Numerical Methods for Fluid Dynamics, Ch. 4, Test 1:
    rho*_L = 0.42632, rho*_R = 0.26557), the rarefaction fan's closed form,
    and the undisturbed states."""
    g = 1.4
    xi = np.array([-2.0, -0.5, 0.5, 1.2, 2.0])
    rho = exact_riemann_density(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, xi)
    cL, gm = np.sqrt(g), (g - 1) / (g + 1)
    fan = (2 / (g + 1) + gm / cL * 0.5) ** (2 / (g - 1))     # s = -0.5 inside the fan
    np.testing.assert_allclose(rho, [1.0, fan, 0.42632, 0.26557, 0.125], rtol=2e-5)



# ---------------------------------------------------------------------------
# The Euler flux's dissipation speed, pinned by the linearisation about a
# uniform state (von Neumann analysis of the semi-discrete scheme).

GAMMA_TEST = 2.0  # gamma = (d_v + 2)/d_v with d_v = 2


def _textbook_flux(U, d):
    """Physical flux of the 2-D Euler equations (textbook form)."""
    rho, mx, my, E = U
    P = (GAMMA_TEST - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
    mn = mx if d == 0 else my
    return np.array([mn, mx * mn / rho + (P if d == 0 else 0.0), my * mn / rho + (P if d == 1 else 0.0),
                     (E + P) * mn / rho])


def _linear_symbol(U0, d, theta, h):
    """M(theta) with Phi(U0 + delta r e^{i theta j}) = delta M r e^{i theta j} + O(delta^2):
    on small perturbations the CWENO3 weights take their linear values, so the
    face states are the optimal parabola's, q^- = (-q_{j-1} + 5 q_j + 2 q_{j+1})/6
    and q^+ = (2 q_j + 5 q_{j+1} - q_{j+2})/6 at face j+1/2; the local
    Lax-Friedrichs flux 1/2 A (q^- + q^+) - 1/2 a (q^+ - q^-) then has the flux
    Jacobian A of U0 and the speed a = |u_d| + sqrt(gamma P/rho) of U0 (its
    perturbation multiplies q^+ - q^-, a second-order term)."""
    e = np.exp(1j * theta)
    qm = (-1.0 / e + 5.0 + 2.0 * e) / 6.0
    qp = (2.0 + 5.0 * e - e * e) / 6.0
    A = np.empty((4, 4))
    for k in range(4):  # complex-step derivative: exact to rounding
        dU = np.zeros(4, complex)
        dU[k] = 1e-30j
        A[:, k] = _textbook_flux(U0.astype(complex) + dU, d).imag / 1e-30
    rho, mx, my, E = U0
    un = (mx if d == 0 else my) / rho
    P = (GAMMA_TEST - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
    a = abs(un) + np.sqrt(GAMMA_TEST * P / rho)
    return (1.0 - 1.0 / e) / h * (0.5 * (qm + qp) * A - 0.5 * (qp - qm) * a * np.eye(4)), a


@pytest.mark.parametrize("d", [0, 1])
@pytest.mark.parametrize("mode", [1, 3])
def test_euler_flux_dissipation_matches_linearisation(d, mode):
    """Phi of a small sine perturbation of a uniform moving state equals the
    closed-form linear symbol of CWENO3 + local Lax-Friedrichs with
    a = |u_n| + sqrt(gamma P/rho): a wrong dissipation speed (half of it, or
    the speed without |u_n|) changes the damping part of the symbol by far
    more than the tolerance."""
    n, h = 12, 0.1
    rho0, ux0, uy0, p0 = 1.3, 0.4, -0.25, 0.9
    U0 = np.array([rho0, rho0 * ux0, rho0 * uy0, p0 / (GAMMA_TEST - 1.0) + 0.5 * rho0 * (ux0 ** 2 + uy0 ** 2)])
    r = np.array([1.0, -0.7, 0.45, 1.9])  # a generic direction: every characteristic field is excited
    delta = 1e-7
    theta = 2.0 * np.pi * mode / n
    jj = np.arange(n)
    shape = (1, n) if d == 0 else (n, 1)
    pert = np.cos(theta * jj + 0.3).reshape(shape)
    U = U0[:, None, None] + delta * r[:, None, None] * pert[None]
    U = np.broadcast_to(U, (4, 3, n) if d == 0 else (4, n, 3)).copy()
    phi = O.euler_phi(U, h, h, "periodic", "periodic", 1e-6)
    phi = phi[:, 1, :] if d == 0 else phi[:, :, 1]
    M, a = _linear_symbol(U0, d, theta, h)
    want = delta * np.real((M @ r)[:, None] * np.exp(1j * (theta * jj + 0.3))[None])
    scale = np.abs(want).max()
    assert np.abs(phi - want).max() <= 1e-5 * scale
    # the damping part is resolved: the same symbol with half the speed is far off
    M_half = M + (1.0 - 1.0 / np.exp(1j * theta)) / h * 0.25 * a * \
        ((2.0 + 5.0 * np.exp(1j * theta) - np.exp(2j * theta)) / 6.0
         - (-np.exp(-1j * theta) + 5.0 + 2.0 * np.exp(1j * theta)) / 6.0) * np.eye(4)
    other = delta * np.real((M_half @ r)[:, None] * np.exp(1j * (theta * jj + 0.3))[None])
    assert np.abs(other - want).max() > 1e-3 * scale


def test_euler_wave_speed_of_a_face_state_without_pressure():
    """Reading R25: a reconstructed face state whose pressure is not positive
    (component-wise reconstruction of the conserved variables can give one
    next to a strong expansion) has no sound speed, so its local
    Lax-Friedrichs speed is |u_n|; a positive pressure gives
    |u_n| + sqrt(gamma P/rho).  The flux itself is the physical flux."""
    from oracle import transport as T
    rho, ux, uy = 0.8, -1.5, 0.6
    for P, want in ((-0.05, None), (0.0, None), (0.3, np.sqrt(GAMMA_TEST * 0.3 / rho))):
        E = P / (GAMMA_TEST - 1.0) + 0.5 * rho * (ux * ux + uy * uy)
        U = np.array([rho, rho * ux, rho * uy, E])
        for d, un in ((0, ux), (1, uy)):
            F, a = T.euler_flux(U, d)
            assert np.isfinite(a) and a == pytest.approx(abs(un) + (want or 0.0), rel=1e-14)
            assert np.allclose(F, _textbook_flux(U, d), rtol=1e-12, atol=1e-14)
