"""Velocity grid, moments, ES Gaussian and implicit relaxation (oracle, FP64).

Test infrastructure only (see the package docstring).

Array convention: a distribution of one cell is ``g[vy, vx]``; leading axes are
cells.  Macroscopic conserved variables are ``U = (rho, rho u_x, rho u_y, E)``
along the LAST axis in this module.
"""

import numpy as np

DV = 2  # velocity dimension of every simulation in the paper (Sec. 4 opening)


def velocity_grid(nv, vmax):
    """Nodes and quadrature weight of the discrete velocity grid (Sec. 3.2).

    The paper truncates velocity space to [-v_max, v_max]^2 with N_v points and
    step dv per direction.  Reading R1: midpoint nodes
    v_k = -v_max + (k + 1/2) dv, dv = 2 v_max / N_v, and the rectangle rule,
    i.e. every node carries weight w = dv^2.
    """
    dv = 2.0 * vmax / nv
    v = -vmax + (np.arange(nv) + 0.5) * dv
    return v, dv * dv


def moments(g, v, w):
    """The six discrete velocity moments of g (hypothesis H3 and the stress
    tensor of Sec. 2): rho = w sum g, m = w sum v g, S = w sum v (x) v g.

    Returns an array (..., 6) = (rho, m_x, m_y, S_xx, S_xy, S_yy).
    """
    vx = v[None, :]
    vy = v[:, None]
    ax = (-2, -1)
    return np.stack([
        w * np.sum(g, axis=ax),
        w * np.sum(g * vx, axis=ax),
        w * np.sum(g * vy, axis=ax),
        w * np.sum(g * vx * vx, axis=ax),
        w * np.sum(g * vx * vy, axis=ax),
        w * np.sum(g * vy * vy, axis=ax),
    ], axis=-1)


def macro_from_moments(mom):
    """rho, u, T and the tensor Theta from the moments (H3 and Sec. 2).

    u = m / rho;  Theta = (1/rho) int (v-u)(x)(v-u) f dv = S/rho - u (x) u;
    T = (1/(d_v rho)) int |v-u|^2 f dv = tr(Theta) / d_v with d_v = 2.
    Theta is returned as (..., 2, 2).
    """
    rho = mom[..., 0]
    u = np.stack([mom[..., 1] / rho, mom[..., 2] / rho], axis=-1)
    S = np.empty(mom.shape[:-1] + (2, 2))
    S[..., 0, 0] = mom[..., 3]
    S[..., 0, 1] = S[..., 1, 0] = mom[..., 4]
    S[..., 1, 1] = mom[..., 5]
    Theta = S / rho[..., None, None] - u[..., :, None] * u[..., None, :]
    T = np.trace(Theta, axis1=-2, axis2=-1) / DV
    return rho, u, T, Theta


def cons_from_moments(mom):
    """U = (rho, rho u_x, rho u_y, E) from moments; E = tr(S)/2 is
    (1/2) rho |u|^2 + (d_v/2) rho T (Sec. 2, energy of the Euler system)."""
    return np.stack([mom[..., 0], mom[..., 1], mom[..., 2],
                     0.5 * (mom[..., 3] + mom[..., 5])], axis=-1)


def cons_from_prim(rho, ux, uy, T):
    """U from (rho, u, T): E = 1/2 rho |u|^2 + (d_v/2) rho T, d_v = 2 (Sec. 2)."""
    E = 0.5 * rho * (ux * ux + uy * uy) + 0.5 * DV * rho * T
    return np.stack([rho, rho * ux, rho * uy, E], axis=-1)


def prim_from_cons(U):
    """(rho, u_x, u_y, T) from U, inverting cons_from_prim."""
    rho = U[..., 0]
    ux = U[..., 1] / rho
    uy = U[..., 2] / rho
    T = (U[..., 3] - 0.5 * rho * (ux * ux + uy * uy)) / (0.5 * DV * rho)
    return rho, ux, uy, T


def gaussian(rho, u, Tt, v):
    """Anisotropic Gaussian of the ES-BGK operator at the velocity nodes (Sec. 2):

        G = rho / sqrt(det(2 pi Tt)) * exp(-(v-u)^T Tt^{-1} (v-u) / 2).

    rho: (...), u: (..., 2), Tt: (..., 2, 2).  Returns (..., nv, nv) [vy, vx].
    """
    det = np.linalg.det(2.0 * np.pi * Tt)
    inv = np.linalg.inv(Tt)
    cx = v[None, :] - u[..., 0, None, None]
    cy = v[:, None] - u[..., 1, None, None]
    quad = (inv[..., 0, 0, None, None] * cx * cx
            + (inv[..., 0, 1, None, None] + inv[..., 1, 0, None, None]) * cx * cy
            + inv[..., 1, 1, None, None] * cy * cy)
    return (rho / np.sqrt(det))[..., None, None] * np.exp(-0.5 * quad)


def _basis(u, T, v):
    """psi = (1, xi_x, xi_y, xi_x^2, xi_x xi_y, xi_y^2), xi = (v-u)/sqrt(T).
    Returns (..., 6, nv, nv)."""
    s = np.sqrt(T)[..., None, None]
    xx = (v[None, :] - u[..., 0, None, None]) / s
    xy = (v[:, None] - u[..., 1, None, None]) / s
    xx, xy = np.broadcast_arrays(xx, xy)
    one = np.ones_like(xx)
    return np.stack([one, xx, xy, xx * xx, xx * xy, xy * xy], axis=-3)


def projected_gaussian(rho, u, Tt, v, w):
    """Discrete ES Gaussian G_hat reproducing its moments exactly on the grid.

    Reading R4 (the paper is silent on discrete conservation; this is the
    project's choice so that hypothesis H1 holds to round-off on the grid):
    G_hat = G (1 + a . psi) with psi the quadratic basis of ``_basis`` and a the
    solution of the 6x6 system  H a = t - r,  H_mn = w sum G psi_m psi_n,
    r_m = w sum G psi_m, t = (rho, 0, 0, rho Tt_xx/T, rho Tt_xy/T, rho Tt_yy/T),
    T = tr(Tt)/2.  Then w sum psi G_hat = t: G_hat has density rho, mean
    velocity u and temperature tensor Tt exactly.
    """
    G = gaussian(rho, u, Tt, v)
    T = np.trace(Tt, axis1=-2, axis2=-1) / DV
    psi = _basis(u, T, v)
    H = w * np.einsum("...mab,...nab,...ab->...mn", psi, psi, G)
    r = w * np.einsum("...mab,...ab->...m", psi, G)
    z = np.zeros_like(rho)
    t = np.stack([rho, z, z, rho * Tt[..., 0, 0] / T, rho * Tt[..., 0, 1] / T,
                  rho * Tt[..., 1, 1] / T], axis=-1)
    a = np.linalg.solve(H, (t - r)[..., None])[..., 0]
    return G * (1.0 + np.einsum("...m,...mab->...ab", a, psi))


def maxwellian_hat(rho, u, T, v, w):
    """Discrete Maxwellian with moments (rho, u, T): the projected Gaussian with
    Tt = T I (hypothesis H3; the ES Gaussian with beta = 0 and Theta = T I)."""
    Tt = T[..., None, None] * np.eye(2)
    return projected_gaussian(rho, u, Tt, v, w)


def temperature_tensor(T, Theta, beta):
    """Tt = (1 - beta) T I + beta Theta (Sec. 2)."""
    return (1.0 - beta) * T[..., None, None] * np.eye(2) + beta * Theta


def es_gaussian_of(g, v, w, beta):
    """G_hat[g]: the discrete ES Gaussian built from g's own moments (Sec. 2)."""
    rho, u, T, Theta = macro_from_moments(moments(g, v, w))
    return projected_gaussian(rho, u, temperature_tensor(T, Theta, beta), v, w)


def relax(fstar, h, beta, v, w):
    """Solve the implicit relaxation  f = f* + h (G_hat[f] - f)  for f.

    This is the implicit part of one IMEX stage (Eq. RKEI1) with
    h = dt a_ii tau/eps, solved through the conserved moments as in the
    first-order IMEX scheme of Filbet and Jin that the paper extends (Sec. 3.4,
    Sec. 4 opening).  Derivation (the paper cites it without writing it out):
    G_hat[f] has the density, velocity and temperature of f, which the
    relaxation does not change, so rho, u, T are those of f*.  Taking the
    stress moment of  (1+h) f = f* + h G_hat  gives
    (1+h) Theta = Theta* + h Tt  with  Tt = (1-beta) T I + beta Theta, i.e.
        Theta = (Theta* + h (1-beta) T I) / (1 + h (1-beta)).
    Then f = (f* + h G_hat[rho, u, Tt]) / (1 + h).

    fstar: (N, nv, nv); h: scalar or (N,).  Returns (f, G_hat).
    """
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), fstar.shape[:-2])
    rho, u, T, Theta_s = macro_from_moments(moments(fstar, v, w))
    k = h * (1.0 - beta)
    Theta = (Theta_s + (k * T)[..., None, None] * np.eye(2)) / (1.0 + k)[..., None, None]
    Tt = temperature_tensor(T, Theta, beta)
    Gh = projected_gaussian(rho, u, Tt, v, w)
    f = (fstar + h[..., None, None] * Gh) / (1.0 + h)[..., None, None]
    return f, Gh
