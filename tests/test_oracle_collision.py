"""Pins of the oracle's collision part against what the paper and mathematics fix.

Hypotheses H1-H3 and the ES Gaussian of Sec. 2; the implicit IMEX stage of
Eq. RKEI1.  None of these tests re-runs the oracle's own formula: each checks a
closed form, an invariant, a limit or a brute-force property.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W


def textbook_maxwellian(rho, ux, uy, T, VX, VY):
    return rho / (2 * np.pi * T) * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2) / (2 * T))


def test_moments_of_fine_maxwellian():
    """H3: the moments of a Maxwellian are its (rho, u, T); on a fine grid the
    rectangle rule is spectrally accurate."""
    v, w = O.velocity_grid(220, 16.0)
    VX, VY = np.meshgrid(v, v)
    for rho, ux, uy, T in [(1.3, 0.3, -0.2, 0.8), (0.2, -1.0, 0.5, 2.5), (2.0, 0.0, 0.0, 0.3)]:
        M = textbook_maxwellian(rho, ux, uy, T, VX, VY)
        r, u, TT, Th = O.macro_from_moments(O.moments(M, v, w))
        assert abs(r - rho) < 1e-12 * rho
        assert np.allclose(u, [ux, uy], atol=1e-12)
        assert abs(TT - T) < 1e-12 * T
        assert np.allclose(Th, T * np.eye(2), atol=1e-12)
        U = O.cons_from_moments(O.moments(M, v, w))
        assert np.allclose(U, [rho, rho * ux, rho * uy, 0.5 * rho * (ux ** 2 + uy ** 2) + rho * T], rtol=1e-12)


def test_gaussian_moments_fine_grid():
    """Sec. 2: G[rho, u, Tt] has density rho, velocity u and temperature tensor
    Tt (this fixes the normalisation det(2 pi Tt), the inverse and the 1/2)."""
    rng = np.random.default_rng(1)
    v, w = O.velocity_grid(200, 14.0)
    for _ in range(4):
        rho = rng.uniform(0.2, 2.0)
        u = rng.uniform(-0.8, 0.8, size=2)
        B = rng.normal(size=(2, 2))
        Tt = 0.5 * np.eye(2) + 0.3 * B @ B.T
        G = O.gaussian(np.array(rho), u, Tt, v)
        r, uu, T, Th = O.macro_from_moments(O.moments(G, v, w))
        assert abs(r - rho) < 1e-11 * rho
        assert np.allclose(uu, u, atol=1e-11)
        assert np.allclose(Th, Tt, atol=1e-11)


@pytest.mark.parametrize("nv,vmax", [(16, 6.0), (32, 8.0), (12, 5.0)])
def test_projected_gaussian_exact_on_grid(nv, vmax):
    """Reading R4: G_hat reproduces (rho, rho u, rho (Tt + u u)) to round-off on
    the coarse grid, and is a small correction of G there."""
    rng = np.random.default_rng(2)
    v, w = O.velocity_grid(nv, vmax)
    rho = rng.uniform(0.3, 1.5, size=5)
    u = rng.uniform(-0.6, 0.6, size=(5, 2))
    Tt = np.empty((5, 2, 2))
    for c in range(5):
        T = rng.uniform(0.5, 1.5)
        th = rng.uniform(-0.3, 0.3)
        Tt[c] = T * np.array([[1 + th, 0.2 * th], [0.2 * th, 1 - th]])
    Gh = O.projected_gaussian(rho, u, Tt, v, w)
    m = O.moments(Gh, v, w)
    assert np.allclose(m[:, 0], rho, rtol=1e-13, atol=0)
    assert np.allclose(m[:, 1:3], rho[:, None] * u, rtol=0, atol=1e-13)
    S = np.stack([m[:, 3], m[:, 4], m[:, 5]], -1)
    S_ref = rho[:, None] * np.stack([Tt[:, 0, 0] + u[:, 0] ** 2, Tt[:, 0, 1] + u[:, 0] * u[:, 1],
                                     Tt[:, 1, 1] + u[:, 1] ** 2], -1)
    assert np.allclose(S, S_ref, rtol=1e-13, atol=1e-13)
    G = O.gaussian(rho, u, Tt, v)
    assert np.max(np.abs(Gh - G)) < 1e-3 * np.max(G)


def test_quadratic_projection_needs_three_nodes_per_direction():
    """Reading R4 corrects the Gaussian within span(1, v_x, v_y, v_x^2, v_x v_y,
    v_y^2).  Brute force on the grid: the six functions are independent on the
    N_v x N_v nodes only for N_v >= 3 (on two points v^2 is constant), the
    bound the library enforces; on the smallest such grid the projected
    Gaussian still reproduces its moments to round-off."""
    for nv in (2, 3, 4, 5):
        v, _ = O.velocity_grid(nv, 3.0)
        VX, VY = np.meshgrid(v, v)
        B = np.stack([np.ones_like(VX), VX, VY, VX * VX, VX * VY, VY * VY]).reshape(6, -1)
        assert np.linalg.matrix_rank(B) == (4 if nv == 2 else 6)
    v, w = O.velocity_grid(3, 3.0)
    rho, u = np.array([1.1]), np.array([[0.2, -0.1]])
    Tt = np.array([[[1.2, 0.1], [0.1, 0.9]]])
    m = O.moments(O.projected_gaussian(rho, u, Tt, v, w), v, w)
    S_ref = rho * np.array([Tt[0, 0, 0] + u[0, 0] ** 2, Tt[0, 0, 1] + u[0, 0] * u[0, 1], Tt[0, 1, 1] + u[0, 1] ** 2])
    assert np.allclose(m[0, :3], [rho[0], rho[0] * u[0, 0], rho[0] * u[0, 1]], rtol=1e-13, atol=1e-14)
    assert np.allclose(m[0, 3:6], S_ref, rtol=1e-13, atol=1e-14)


def test_collision_conserves_h1():
    """H1: the relaxation step conserves mass, momentum and energy exactly:
    w sum (1, v, |v|^2/2) (G_hat - f) = 0 for random positive f."""
    nv, vmax = 16, 6.0
    v, w = O.velocity_grid(nv, vmax)
    VX, VY = np.meshgrid(v, v)
    fs = W.random_cells(8, nv, vmax, seed=3)
    h = np.array([1e-3, 0.1, 1.0, 10.0, 1e4, 0.5, 2.0, 1e6])
    f, Gh = O.relax(fs, h, -0.5, v, w)
    for g in (f, Gh):
        for phi in (np.ones_like(VX), VX, VY, 0.5 * (VX ** 2 + VY ** 2)):
            a = w * np.sum(g * phi, axis=(-2, -1))
            b = w * np.sum(fs * phi, axis=(-2, -1))
            assert np.allclose(a, b, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("beta", [-0.5, 0.0, 0.4])
def test_implicit_stage_residual(beta):
    """Eq. RKEI1, implicit part: the returned f solves f = f* + h (G_hat[f] - f)
    with G_hat[f] recomputed from f's own moments (so the closed-form update of
    Theta is the exact solution of the discrete implicit equation)."""
    nv, vmax = 16, 6.0
    v, w = O.velocity_grid(nv, vmax)
    fs = W.random_cells(6, nv, vmax, seed=4)
    h = np.array([1e-2, 0.3, 1.0, 7.0, 1e3, 1e6])
    f, _ = O.relax(fs, h, beta, v, w)
    Gf = O.es_gaussian_of(f, v, w, beta)
    res = f - fs - h[:, None, None] * (Gf - f)
    scale = (1 + h)[:, None, None] * np.max(fs)
    assert np.max(np.abs(res / scale)) < 1e-13


def test_bgk_limit_pr_one():
    """Pr = 1/(1-beta) = 1 (beta = 0): the ES Gaussian is the Maxwellian and the
    homogeneous relaxation contracts f - M_hat by exactly 1/(1+h) (Sec. 2)."""
    nv, vmax = 16, 6.0
    v, w = O.velocity_grid(nv, vmax)
    fs = W.random_cells(4, nv, vmax, seed=5)
    rho, u, T, _ = O.macro_from_moments(O.moments(fs, v, w))
    M = O.maxwellian_hat(rho, u, T, v, w)
    G = O.es_gaussian_of(fs, v, w, 0.0)
    assert np.max(np.abs(G - M)) < 1e-14 * np.max(M) * 10
    h = 0.7
    f, _ = O.relax(fs, h, 0.0, v, w)
    assert np.allclose(f - M, (fs - M) / (1 + h), atol=1e-14)


def test_equilibrium_is_fixed_point():
    """H3: Q(M) = 0 -- the ES Gaussian of a Maxwellian is that Maxwellian."""
    nv, vmax = 16, 6.0
    v, w = O.velocity_grid(nv, vmax)
    rho = np.array([0.7, 1.4])
    u = np.array([[0.2, -0.1], [0.0, 0.4]])
    T = np.array([0.9, 1.6])
    M = O.maxwellian_hat(rho, u, T, v, w)
    for beta in (-0.5, 0.3):
        G = O.es_gaussian_of(M, v, w, beta)
        assert np.max(np.abs(G - M)) < 1e-13 * np.max(M)


def stability_function(A, b, z):
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


@pytest.mark.parametrize("tab_name", ["ARS233", "IMEX_EULER"])
@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-5])
def test_homogeneous_relaxation_stability_function(tab_name, eps):
    """Space-homogeneous problem: the stress deviation y = Theta - T I obeys
    y' = -(1-beta) nu y, so one IMEX step multiplies it by the implicit
    tableau's stability function R(z) = 1 + z b^T (I - z A)^{-1} 1 with
    z = -(1-beta) nu dt; rho, u, T stay fixed."""
    tab = getattr(O, tab_name)
    prob = O.Problem(nx=1, ny=1, nv=16, vmax=6.0, beta=-0.5, tau=1.0, switch="frozen")
    v, w = O.velocity_grid(prob.nv, prob.vmax)
    f0 = W.random_cells(1, prob.nv, prob.vmax, seed=6, anisotropy=0.6)
    mom = O.moments(f0, v, w)
    U = O.cons_from_moments(mom)
    st = O.State(f=f0[None].copy(), U=np.moveaxis(U, -1, 0)[:, None].reshape(4, 1, 1).copy(),
                 kin=np.ones((1, 1), bool), eps=np.full((1, 1), eps))
    dt = 0.01
    z = -(1.0 - prob.beta) * (prob.tau / eps) * dt
    R = stability_function(tab.A, tab.b, z)
    rho0, u0, T0, Th0 = O.macro_from_moments(mom[0])
    y = Th0 - T0 * np.eye(2)
    for _ in range(3):
        st = O.advance(prob, st, dt, tab)
        y = R * y
        rho, u, T, Th = O.macro_from_moments(O.moments(st.f[0, 0], v, w))
        tol = 1e-14 * (1 + abs(z))
        assert abs(rho - rho0) < tol * rho0 and np.allclose(u, u0, atol=tol) and abs(T - T0) < tol * T0
        # round-off of the stiff solve grows like |z| eps_machine
        assert np.allclose(Th - T * np.eye(2), y, atol=1e-15 * (1 + abs(z)), rtol=0)
