"""CWENO3 reconstruction, kinetic transport L(f) and Euler divergence Phi(U).

Test infrastructure only (see the package docstring).

Sec. 3.2 names third-order CWENO reconstruction with a Lax-Friedrichs
numerical flux for both the kinetic advection and the Euler flux, and prints
no formula for either.
Reading R5: the third-order CWENO reconstruction of Levy, Puppo and Russo
(1999), applied dimension by dimension on cell averages, evaluated at the two
faces of each cell; the Lax-Friedrichs (Rusanov) numerical flux with the local
wave speed (|v_k| for the kinetic transport, max |u_n| + sqrt(gamma P/rho) of
the two face states for Euler).  Reading R6: two ghost cells per side,
periodic or outflow (copy of the nearest interior cell).
"""

import numpy as np

GAMMA = 2.0  # gamma = (d_v + 2)/d_v with d_v = 2 (Sec. 2)


def pad_cells(a, axis, bc, n=2):
    """Add n ghost cells on both sides of `axis` ('periodic' or 'outflow')."""
    m = a.shape[axis]
    idx = np.arange(-n, m + n)
    idx = idx % m if bc == "periodic" else np.clip(idx, 0, m - 1)
    return np.take(a, idx, axis=axis)


def cweno3_faces(qm, q0, qp, eps_w):
    """CWENO3 values at the left and right face of the middle cell.

    With s = (x - x_j)/dx on the cell [-1/2, 1/2] and cell averages
    qm, q0, qp of cells j-1, j, j+1:
      P_L(s) = q0 + (q0 - qm) s,   P_R(s) = q0 + (qp - q0) s,
      P_opt(s) = a0 + a1 s + a2 s^2, the parabola whose averages over the three
        cells are qm, q0, qp (the average of s^2 over [c-1/2, c+1/2] is
        c^2 + 1/12), so a2 = (qp - 2 q0 + qm)/2, a1 = (qp - qm)/2,
        a0 = q0 - a2/12,
      P_0 = (P_opt - d_L P_L - d_R P_R)/d_0 with linear weights
        d_0 = 1/2, d_L = d_R = 1/4,
      smoothness indicators (Jiang-Shu, of P_L, P_R and P_0):
        IS_L = (q0 - qm)^2, IS_R = (qp - q0)^2,
        IS_0 = 13/3 (qp - 2 q0 + qm)^2 + 1/4 (qp - qm)^2,
      nonlinear weights alpha_k = d_k/(eps_w + IS_k)^2, omega_k = alpha_k/sum,
      R(s) = omega_0 P_0(s) + omega_L P_L(s) + omega_R P_R(s).
    Returns (R(-1/2), R(+1/2)).
    """
    a2 = 0.5 * (qp - 2.0 * q0 + qm)
    a1 = 0.5 * (qp - qm)
    a0 = q0 - a2 / 12.0
    d0, dL, dR = 0.5, 0.25, 0.25

    def P_L(s):
        return q0 + (q0 - qm) * s

    def P_R(s):
        return q0 + (qp - q0) * s

    def P_opt(s):
        return a0 + a1 * s + a2 * s * s

    def P_0(s):
        return (P_opt(s) - dL * P_L(s) - dR * P_R(s)) / d0

    IS_0, IS_L, IS_R = cweno3_indicators(qm, q0, qp)
    al0 = d0 / (eps_w + IS_0) ** 2
    alL = dL / (eps_w + IS_L) ** 2
    alR = dR / (eps_w + IS_R) ** 2
    tot = al0 + alL + alR

    def R(s):
        return (al0 * P_0(s) + alL * P_L(s) + alR * P_R(s)) / tot

    return R(-0.5), R(0.5)


def cweno3_indicators(qm, q0, qp):
    """Jiang-Shu smoothness indicators IS = sum_l dx^(2l-1) int_cell (d^l P/dx^l)^2
    of P_0, P_L and P_R in closed form (Levy-Puppo-Russo CWENO3):
    IS_0 = 13/3 (qp - 2 q0 + qm)^2 + 1/4 (qp - qm)^2,
    IS_L = (q0 - qm)^2, IS_R = (qp - q0)^2."""
    IS_0 = 13.0 / 3.0 * (qp - 2.0 * q0 + qm) ** 2 + 0.25 * (qp - qm) ** 2
    return IS_0, (q0 - qm) ** 2, (qp - q0) ** 2


def _face_states(q, axis, bc, eps_w):
    """States left (q^-) and right (q^+) of the faces i-1/2, i = 0..n along
    `axis` (n+1 faces)."""
    n = q.shape[axis]
    qp = pad_cells(q, axis, bc)

    def sl(a, b):
        return np.take(qp, np.arange(a, b), axis=axis)

    left, right = cweno3_faces(sl(0, n + 2), sl(1, n + 3), sl(2, n + 4), eps_w)
    # reconstructed cells are -1..n; face i-1/2 sits between cells i-1 and i
    qminus = np.take(right, np.arange(0, n + 1), axis=axis)
    qplus = np.take(left, np.arange(1, n + 2), axis=axis)
    return qminus, qplus


def _divergence(F, axis, h):
    n = F.shape[axis] - 1
    return (np.take(F, np.arange(1, n + 1), axis=axis)
            - np.take(F, np.arange(0, n), axis=axis)) / h


def _recon(eps_w):
    def r(qm, q0, qp):
        return cweno3_faces(qm, q0, qp, eps_w)
    return r


def kinetic_face_fluxes(f, v, bc_x, bc_y, eps_w, walls=None):
    """The numerical fluxes of the kinetic transport at every face: Fx at the
    faces i-1/2 (i = 0..nx) along x, Fy at j-1/2 along y, per velocity node
    (the F of kinetic_transport, whose divergence is L(f)).  walls: None, or
    (solid mask, stencil maps) of oracle.walls (specular walls, reading R24)."""
    from . import walls as Wl
    vx = v[None, None, None, :]
    vy = v[None, None, :, None]
    if walls is None:
        qm, qp = _face_states(f, 1, bc_x, eps_w)
    else:
        qm, qp = Wl.face_states(f, walls[0], walls[1], 0, bc_x, eps_w, Wl.reflect_f, _recon(eps_w))
    Fx = 0.5 * vx * (qm + qp) - 0.5 * np.abs(vx) * (qp - qm)
    if walls is None:
        qm, qp = _face_states(f, 0, bc_y, eps_w)
    else:
        qm, qp = Wl.face_states(f, walls[0], walls[1], 1, bc_y, eps_w, Wl.reflect_f, _recon(eps_w))
    Fy = 0.5 * vy * (qm + qp) - 0.5 * np.abs(vy) * (qp - qm)
    return Fx, Fy


def kinetic_transport(f, v, dx, dy, bc_x, bc_y, eps_w, walls=None):
    """L(f), the discretisation of v . grad_x f (Eq. semidiscrete ES-BGK).

    f: (ny, nx, nv, nv) indexed [j, i, vy, vx].  Per velocity node and axis the
    Lax-Friedrichs flux with the exact local speed,
    F = 1/2 v (q^- + q^+) - 1/2 |v| (q^+ - q^-), then L = dF/dx + dG/dy.
    """
    Fx, Fy = kinetic_face_fluxes(f, v, bc_x, bc_y, eps_w, walls)
    return _divergence(Fx, 1, dx) + _divergence(Fy, 0, dy)


def flux_moments(F, v, w):
    """Moments w sum F (1, v_x, v_y, |v|^2/2) of a face flux per velocity node
    (F: (..., nv, nv) indexed [vy, vx]); the conserved-variable flux it
    carries."""
    VX, VY = np.meshgrid(v, v)
    psi = np.stack([np.ones_like(VX), VX, VY, 0.5 * (VX * VX + VY * VY)])
    return w * np.einsum("...ab,qab->q...", F, psi)


def euler_flux(U, d):
    """Physical Euler flux F_x (d=0) or F_y (d=1) of Eq. Euler_Compact, with
    P = (gamma - 1)(E - 1/2 rho |u|^2), and the local wave speed
    |u_n| + sqrt(gamma P / rho).  U: (4, ...).  Reading R25: a reconstructed
    face state whose pressure is not positive has no sound speed; its wave
    speed is |u_n| (the sound speed with P clipped at 0)."""
    rho, mx, my, E = U
    ux, uy = mx / rho, my / rho
    P = (GAMMA - 1.0) * (E - 0.5 * rho * (ux * ux + uy * uy))
    un = ux if d == 0 else uy
    return np.stack([rho * un,
                     mx * un + (P if d == 0 else 0.0),
                     my * un + (P if d == 1 else 0.0),
                     un * (E + P)]), np.abs(un) + np.sqrt(GAMMA * np.maximum(P, 0.0) / rho)


def euler_phi(U, dx, dy, bc_x, bc_y, eps_w, override=None, walls=None):
    """Phi(U), the discretisation of div_x F(U) (Eq. semidiscrete Euler).

    U: (4, ny, nx).  Component-wise CWENO3 face states and the local
    Lax-Friedrichs flux  F = 1/2 (F(U^-) + F(U^+)) - 1/2 a (U^+ - U^-),
    a = max over the two states of |u_n| + sqrt(gamma P / rho).
    override: None, or ((Gx, mask_x), (Gy, mask_y)) -- face fluxes (4, ny,
    nx+1) / (4, ny+1, nx) that replace the Euler flux where the boolean face
    mask is set.  walls: None, or (solid mask, stencil maps) of oracle.walls
    (the mirror state across a wall, reading R24).
    """
    from . import walls as Wl
    out = np.zeros_like(U)
    for k, (d, axis, h, bc) in enumerate(((0, 2, dx, bc_x), (1, 1, dy, bc_y))):
        if walls is None:
            Um, Up = _face_states(U, axis, bc, eps_w)
        else:
            Uc = np.moveaxis(U, 0, -1)
            Um, Up = Wl.face_states(Uc, walls[0], walls[1], d, bc, eps_w, Wl.reflect_U, _recon(eps_w))
            Um, Up = np.moveaxis(Um, -1, 0), np.moveaxis(Up, -1, 0)
        Fm, am = euler_flux(Um, d)
        Fp, ap = euler_flux(Up, d)
        a = np.maximum(am, ap)
        F = 0.5 * (Fm + Fp) - 0.5 * a[None] * (Up - Um)
        if override is not None:
            G, mask = override[k]
            F = np.where(mask[None], G, F)
        out += _divergence(F, axis, h)
    return out
