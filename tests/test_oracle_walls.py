"""Pins of the oracle's specular walls (Sec. 4.2.3-4.2.4; reading R24).

A wall on a symmetry line: a periodic problem whose data is mirror-symmetric
about two faces evolves symmetrically, so its half between the faces must be
reproduced exactly by the same half enclosed by solid cells, whose stencil
values are the mirror images the wall rule forms.  This fixes the mirror
positions, the reflection of f (v_n -> -v_n) and of the Euler state
(m_n -> -m_n), the criterion's gradients at a wall and the buffer cells that
a wall's mirror images need, in the transport, the Euler flux and the switch
alike.  Around an interior obstacle mass and energy are conserved exactly.
"""

import numpy as np
import pytest

import oracle as O


def _symmetric_pair(axis, N=10, Ws=5, nt=6, nv=12, seed=3):
    """Reference: 2N periodic cells along `axis`, data mirror-symmetric about
    the face between cells N-1 and N and (periodically) the face between 2N-1
    and 0; nt periodic cells across.  Walled: N fluid cells then a band of Ws
    solid cells (periodic, so the fluid strip has a wall on each side)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(N) + 0.5) / N
    # a smooth part and a jump, on the half line; mirrored for the other half
    rho_h = 1.0 + 0.3 * np.sin(2.7 * x) + 0.4 * (x > 0.55)
    T_h = 1.0 + 0.2 * np.cos(1.9 * x) - 0.3 * (x > 0.55)
    un_h = 0.4 * np.sin(np.pi * x) + 0.2 * x
    ut_h = 0.3 * np.cos(2.0 * x)
    trans = 1.0 + 0.05 * rng.random(nt)

    def line(h, sign=1.0):
        return np.concatenate([h, sign * h[::-1]])

    fields_ref = {}
    for name, h, sgn in (("rho", rho_h, 1.0), ("T", T_h, 1.0), ("un", un_h, -1.0), ("ut", ut_h, 1.0)):
        fields_ref[name] = np.outer(trans, line(h, sgn))  # (nt, 2N): across, along
    nw = N + Ws
    fields_w = {}
    for name in fields_ref:
        a = np.empty((nt, nw))
        a[:, :N] = fields_ref[name][:, :N]
        a[:, N:] = fields_ref[name][:, :1]  # solid cells: any valid state
        fields_w[name] = a
    solid = np.zeros((nt, nw), bool)
    solid[:, N:] = True

    def orient(a):
        return a if axis == 0 else a.T.copy()

    def make(fl, n_along, solid_mask):
        un, ut = orient(fl["un"]), orient(fl["ut"])
        ux, uy = (un, ut) if axis == 0 else (ut, un)
        rho, T = orient(fl["rho"]), orient(fl["T"])
        eps = np.full(rho.shape, 3e-3)
        ny, nx = rho.shape
        P = O.Problem(nx=nx, ny=ny, x0=0.0, x1=nx / 40.0, y0=0.0, y1=ny / 40.0, nv=nv, vmax=6.0,
                      switch="plain", eta_factor=6.0, delta=1e-3,
                      solid=None if solid_mask is None else orient(solid_mask))
        kin = np.zeros(rho.shape, bool)
        return P, O.init_state(P, rho, ux, uy, T, eps, kin)

    Pr, sr = make(fields_ref, 2 * N, None)
    Pw, sw = make(fields_w, nw, solid)
    return Pr, sr, Pw, sw, N


@pytest.mark.parametrize("axis", [0, 1])
def test_wall_on_a_symmetry_line_reproduces_the_mirrored_periodic_problem(axis):
    Pr, sr, Pw, sw, N = _symmetric_pair(axis)
    dt = 0.5 * min(Pr.dx, Pr.dy) / Pr.vmax
    sel = (slice(None), slice(0, N)) if axis == 0 else (slice(0, N), slice(None))
    saw_kinetic_at_wall = saw_fluid_at_wall = False
    for _ in range(4):
        sr = O.step(Pr, sr, dt, O.ARS233)
        sw = O.step(Pw, sw, dt, O.ARS233)
        np.testing.assert_array_equal(sw.kin[sel], sr.kin[sel])
        kin = sr.kin[sel]
        # the cells touching the two walls of the strip
        edges = np.concatenate([kin[:, 0], kin[:, -1]]) if axis == 0 else np.concatenate([kin[0], kin[-1]])
        saw_kinetic_at_wall |= edges.any()
        saw_fluid_at_wall |= (~edges).any()
        scale = np.abs(sr.U[(slice(None),) + sel]).max()
        assert np.abs(sw.U[(slice(None),) + sel] - sr.U[(slice(None),) + sel]).max() <= 1e-13 * scale
        fk = sr.kin
        if fk.any():
            assert np.abs(sw.f[sel][kin] - sr.f[sel][kin]).max() <= 1e-13 * np.abs(sr.f).max()
    # both models meet a wall somewhere in the run
    assert saw_kinetic_at_wall and saw_fluid_at_wall


def test_mass_and_energy_conserved_around_an_obstacle():
    """Periodic box, a 4 x 5 obstacle, a flow hitting it: all-kinetic and
    all-fluid runs conserve mass and energy to rounding (the wall fluxes of
    both models vanish); the momentum changes (the wall pushes)."""
    n, nv = 16, 12
    X, Y = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n)
    solid = (np.abs(X - 0.5) < 0.13) & (np.abs(Y - 0.5) < 0.16)
    assert 12 <= solid.sum() <= 30
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * Y)
    ux = np.full_like(rho, 0.8)
    uy = 0.1 * np.cos(2 * np.pi * X)
    T = np.ones_like(rho)
    eps = np.full_like(rho, 1e-3)
    for kin in (np.ones((n, n), bool), np.zeros((n, n), bool)):
        P = O.Problem(nx=n, ny=n, nv=nv, vmax=6.0, solid=solid)
        st = O.init_state(P, rho, ux, uy, T, eps, kin)
        t0 = O.totals(P, st)
        dt = 0.5 * P.dx / P.vmax
        for _ in range(5):
            st = O.advance(P, st, dt, O.ARS233)
        t1 = O.totals(P, st)
        assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
        assert abs(t1[3] - t0[3]) <= 1e-13 * t0[3]
        assert abs(t1[1] - t0[1]) > 1e-6 * t0[0]


def test_obstacles_stay_away_from_outflow_edges():
    solid = np.zeros((10, 10), bool)
    solid[1, 5] = True
    with pytest.raises(ValueError):
        O.Problem(nx=10, ny=10, bc_y="outflow", solid=solid).walls
    O.Problem(nx=10, ny=10, bc_y="periodic", solid=solid).walls
