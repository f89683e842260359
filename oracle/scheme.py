"""Regime switch and coupled IMEX time step (Algorithm 1), oracle, FP64.

Test infrastructure only (see the package docstring).

State arrays: f (ny, nx, nv, nv) indexed [j, i, vy, vx]; U (4, ny, nx) with
U = (rho, rho u_x, rho u_y, E); kin (ny, nx) bool (True = kinetic cell);
eps (ny, nx) the Knudsen number field.  f is only meaningful in kinetic cells.
"""

from dataclasses import dataclass, replace
from functools import lru_cache

import numpy as np

from .kinetic import (velocity_grid, moments, cons_from_moments, cons_from_prim,
                      prim_from_cons, maxwellian_hat, es_gaussian_of, relax)
from .transport import pad_cells, kinetic_transport, kinetic_face_fluxes, flux_moments, euler_phi
from . import walls as Wl


@lru_cache(maxsize=16)
def _wall_maps(solid_bytes, ny, nx, bc_x, bc_y):
    solid = Wl.check_solid(np.frombuffer(solid_bytes, bool).reshape(ny, nx), bc_x, bc_y)
    return solid, Wl.stencil_maps(solid, bc_x, bc_y)


@dataclass(frozen=True)
class Problem:
    """Grid (Sec. 3.2), velocity mesh and model/switch parameters.

    beta: ES-BGK parameter, Pr = 1/(1-beta) (Sec. 2.1); the paper uses -0.5.
    tau: Reading R2 -- the collision rate is nu = tau/eps(x), tau constant.
    eta_factor: eta = eta_factor * eps(x) (Reading R9; the tests use
        eta = eps, 4 eps, eps/2, 10 eps).
    delta: threshold of the L1 deviation test (Eq. eqKintoFluid1).
    switch: 'frozen' keeps the regime map fixed (Test 1), 'plain' applies the
        criteria of Sec. 3.1.2 before every step (Algorithm 1).
    coupling: 'stage' couples at every stage (Algorithm 1), 'step' only at the
        end of the step (the LOC-hybrid of Sec. 3.5).
    solid: None, or a bool mask (ny, nx) of solid obstacle cells (Sec. 4.2.3-
        4.2.4): no integrator runs in them and their walls reflect
        specularly (Reading R24, oracle.walls).
    tau_model: 'constant' -- tau fixed (Reading R2); 'density' -- tau = tau *
        rho (Sec. 2 lets tau depend on the macroscopic moments; Reading
        R23): the collision rate of a kinetic cell is nu = tau rho / eps with
        the density of its f* at each stage (which the relaxation conserves),
        and the criterion's mu and kappa use tau rho.
    interface: 'own' -- every cell uses its own model's flux (Reading R11);
        'conservative' -- at a face between a kinetic and a fluid cell the
        fluid cell's Euler update takes the moments (1, v, |v|^2/2) of the
        kinetic cell's numerical flux through that face, so that what leaves
        one side enters the other and the totals are conserved (Sec. 3.6
        states conservation without giving an interface flux; Reading R22).
    """
    nx: int
    ny: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    bc_x: str = "periodic"
    bc_y: str = "periodic"
    nv: int = 16
    vmax: float = 6.0
    beta: float = -0.5
    tau: float = 1.0
    eta_factor: float = 1.0
    delta: float = 1e-3
    cweno_eps: float = 1e-6
    switch: str = "frozen"
    coupling: str = "stage"
    interface: str = "own"
    tau_model: str = "constant"
    solid: object = None

    @property
    def walls(self):
        """(solid mask, stencil maps) of the obstacles (reading R24), or None."""
        if self.solid is None:
            return None
        return _wall_maps(np.asarray(self.solid, bool).tobytes(), self.ny, self.nx, self.bc_x, self.bc_y)

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny

    def centres(self):
        x = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        y = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
        return np.meshgrid(x, y)  # X[j, i], Y[j, i]


@dataclass
class State:
    f: np.ndarray
    U: np.ndarray
    kin: np.ndarray
    eps: np.ndarray


@dataclass(frozen=True)
class Tableau:
    """Butcher tableaux of an IMEX-RK scheme (Sec. 3.4, Eqs. RKEI1-RKEI2):
    explicit (At, bt) for transport and Euler (Abar = At, bbar = bt), implicit
    (A, b) for the relaxation."""
    At: np.ndarray
    bt: np.ndarray
    A: np.ndarray
    b: np.ndarray

    @property
    def s(self):
        return len(self.b)


_al = (3.0 + np.sqrt(3.0)) / 6.0
#: ARS(2,3,3), the paper's third-order IMEX DIRK scheme (Sec. 3.4).
ARS233 = Tableau(
    At=np.array([[0.0, 0.0, 0.0], [_al, 0.0, 0.0], [_al - 1.0, 2.0 - 2.0 * _al, 0.0]]),
    bt=np.array([0.0, 0.5, 0.5]),
    A=np.array([[0.0, 0.0, 0.0], [0.0, _al, 0.0], [0.0, 1.0 - 2.0 * _al, _al]]),
    b=np.array([0.0, 0.5, 0.5]))
#: Reading R12: the lowest-order scheme is the first-order IMEX scheme of
#: Filbet and Jin (Sec. 4 opening) written as ARS(1,1,1):
#: f^{n+1} = relax(f^n - dt L(f^n)).
IMEX_EULER = Tableau(At=np.array([[0.0, 0.0], [1.0, 0.0]]), bt=np.array([1.0, 0.0]),
                     A=np.array([[0.0, 0.0], [0.0, 1.0]]), b=np.array([0.0, 1.0]))
#: Other second-order IMEX tableaux (Sec. 3.4 admits any IMEX-RK pair):
#: ARS(2,2,2) of Ascher, Ruuth and Spiteri (1997), gamma = 1 - 1/sqrt(2),
#: delta = 1 - 1/(2 gamma), first stage explicit, L-stable implicit part.
_g = 1.0 - 1.0 / np.sqrt(2.0)
_d = 1.0 - 1.0 / (2.0 * _g)
ARS222 = Tableau(At=np.array([[0.0, 0.0, 0.0], [_g, 0.0, 0.0], [_d, 1.0 - _d, 0.0]]),
                 bt=np.array([_d, 1.0 - _d, 0.0]),
                 A=np.array([[0.0, 0.0, 0.0], [0.0, _g, 0.0], [0.0, 1.0 - _g, _g]]),
                 b=np.array([0.0, 1.0 - _g, _g]))
#: IMEX-SSP2(3,3,2) of Pareschi and Russo (2005): SSP explicit part, implicit
#: first stage (a_11 = 1/4), stiffly accurate implicit part.
SSP2_332 = Tableau(At=np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5, 0.5, 0.0]]),
                   bt=np.array([1.0, 1.0, 1.0]) / 3.0,
                   A=np.array([[0.25, 0.0, 0.0], [0.0, 0.25, 0.0], [1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0]]),
                   b=np.array([1.0, 1.0, 1.0]) / 3.0)


def _vgrid(prob):
    return velocity_grid(prob.nv, prob.vmax)


def _mhat_of_U(prob, U):
    """f := M_hat[U] for U of shape (4, N) (Eq. Coupling_FluKin)."""
    v, w = _vgrid(prob)
    rho, ux, uy, T = prim_from_cons(U.T)
    return maxwellian_hat(rho, np.stack([ux, uy], -1), T, v, w)


def _U_of_f(prob, g):
    """U := moments of g for g of shape (N, nv, nv) (Eq. Coupling_KinFlu)."""
    v, w = _vgrid(prob)
    return cons_from_moments(moments(g, v, w)).T


def init_state(prob, rho, ux, uy, T, eps, kin=None):
    """Initial state: U from (rho, u, T); f = M_hat[U] in kinetic cells
    (every test of Sec. 4 starts from a Maxwellian)."""
    U = np.moveaxis(cons_from_prim(rho, ux, uy, T), -1, 0).copy()
    kin = np.ones((prob.ny, prob.nx), bool) if kin is None else np.asarray(kin, bool).copy()
    if prob.solid is not None:
        kin &= ~np.asarray(prob.solid, bool)  # no integrator runs in a solid cell
    f = np.zeros((prob.ny, prob.nx, prob.nv, prob.nv))
    if kin.any():
        f[kin] = _mhat_of_U(prob, U[:, kin])
    return State(f=f, U=U, kin=kin, eps=np.asarray(eps, np.float64).copy())


def macro(st):
    """(rho, u_x, u_y, T) of every cell."""
    return prim_from_cons(np.moveaxis(st.U, 0, -1))


def totals(prob, st):
    """Global mass, momentum and energy: sum over cells of U dx dy (solid
    cells hold no state and are left out)."""
    if prob.solid is not None:
        return st.U[:, ~np.asarray(prob.solid, bool)].sum(axis=1) * prob.dx * prob.dy
    return st.U.reshape(4, -1).sum(axis=1) * prob.dx * prob.dy


def buffer_mask(prob, kin):
    """Fluid cells inside the transport stencil (two cells along x or y, ghost
    cells mapped through the boundary condition) of some kinetic cell: the
    buffer region of Remark rem_coupling where f must be reconstructed."""
    ny, nx = kin.shape
    hit = np.zeros_like(kin)
    if prob.walls is not None:
        # the cells the kinetic stencils read, mirror images included
        solid, maps = prob.walls
        flat = hit.reshape(-1)
        for src, _ in maps:
            for k in (0, 1, 3, 4):
                flat[src[k][kin]] = True
        return hit & ~kin & ~solid
    J, I = np.nonzero(kin)
    for d in (-2, -1, 1, 2):
        ii = I + d
        ii = ii % nx if prob.bc_x == "periodic" else np.clip(ii, 0, nx - 1)
        hit[J, ii] = True
        jj = J + d
        jj = jj % ny if prob.bc_y == "periodic" else np.clip(jj, 0, ny - 1)
        hit[jj, I] = True
    return hit & ~kin


def regime_indicators(prob, st):
    """lambda_A = max |lambda - 1| over Sp(S_1), and the L1 deviation of f from
    its Maxwellian in kinetic cells (Sec. 3.1.1-3.1.2).

    S_1 = I - eps D(u) mu/(rho T) - 2/3 (eps kappa/(rho T^{3/2}))^2 grad T grad T^T
    (Eq. for S_1, Sec. 3.1.1) with mu = rho T/(tau (1-beta)) and
    kappa = 5/2 rho T/tau (Sec. 2.1), so with X = I - S_1:
        X = eps/(tau (1-beta)) D + 2/3 (5/2 eps/(tau sqrt T))^2 grad T grad T^T,
    and lambda_A = max |eig X|.  Reading R8: D(u) = grad u + grad u^T
    - 2/3 div u I, the printed d_v = 3 constants.  Reading R7: grad u and
    grad T are second-order central differences of cell-centre values, ghost
    cells per boundary condition.  Reading R9: the L1 norm uses the quadrature
    weights and the discrete Maxwellian built from f's own moments.
    Returns (lamA, L1) with L1 = 0 in fluid cells.
    """
    rho, ux, uy, T = macro(st)
    dx, dy = prob.dx, prob.dy

    def ddx(a):
        ap = pad_cells(a, 1, prob.bc_x, 1)
        return (ap[:, 2:] - ap[:, :-2]) / (2.0 * dx)

    def ddy(a):
        ap = pad_cells(a, 0, prob.bc_y, 1)
        return (ap[2:, :] - ap[:-2, :]) / (2.0 * dy)

    gu = np.empty(rho.shape + (2, 2))  # gu[..., a, b] = d u_a / d x_b
    if prob.walls is None:
        gu[..., 0, 0], gu[..., 0, 1] = ddx(ux), ddy(ux)
        gu[..., 1, 0], gu[..., 1, 1] = ddx(uy), ddy(uy)
        gT = np.stack([ddx(T), ddy(T)], axis=-1)
    else:
        # neighbour states across a wall are mirror states (reading R24)
        solid, maps = prob.walls
        Uc = np.moveaxis(st.U, 0, -1)
        gT = np.empty(rho.shape + (2,))
        for b, h in ((0, dx), (1, dy)):
            lo, hi = Wl.neighbour_values(Uc, maps, b, Wl.reflect_U)
            _, uxl, uyl, Tl = prim_from_cons(lo)
            _, uxh, uyh, Th = prim_from_cons(hi)
            gu[..., 0, b] = (uxh - uxl) / (2.0 * h)
            gu[..., 1, b] = (uyh - uyl) / (2.0 * h)
            gT[..., b] = (Th - Tl) / (2.0 * h)
    div = gu[..., 0, 0] + gu[..., 1, 1]
    D = gu + np.swapaxes(gu, -1, -2) - (2.0 / 3.0) * div[..., None, None] * np.eye(2)
    eps = st.eps
    tau = prob.tau * rho if prob.tau_model == "density" else prob.tau
    c1 = eps / (tau * (1.0 - prob.beta))
    c2 = (2.0 / 3.0) * (2.5 * eps / (tau * np.sqrt(T))) ** 2
    X = c1[..., None, None] * D + c2[..., None, None] * gT[..., :, None] * gT[..., None, :]
    lamA = np.max(np.abs(np.linalg.eigvalsh(X)), axis=-1)
    L1 = np.zeros_like(rho)
    if st.kin.any():
        v, w = _vgrid(prob)
        g = st.f[st.kin]
        Ug = _U_of_f(prob, g)
        L1[st.kin] = w * np.sum(np.abs(g - _mhat_of_U(prob, Ug)), axis=(-2, -1))
    return lamA, L1


def regime_update(prob, st):
    """New regime map (Algorithm 1, regime update; criteria crit:CompEuler and
    eqKintoFluid1): a cell is kinetic after the update iff lambda_A > eta, or
    it was kinetic and ||f - M||_{L1_v} > delta (both conditions must hold to
    go back to Euler)."""
    lamA, L1 = regime_indicators(prob, st)
    eta = prob.eta_factor * st.eps
    new = (lamA > eta) | (st.kin & (L1 > prob.delta))
    if prob.solid is not None:
        new &= ~np.asarray(prob.solid, bool)  # no integrator runs in a solid cell
    return new


def convert(prob, st, new_kin):
    """Apply a regime change (Sec. 3.3): fluid->kinetic cells get
    f := M_hat[U] (Eq. Coupling_FluKin); kinetic->fluid cells keep
    U = moments(f) (Eq. Coupling_KinFlu), which the coupling already holds."""
    new_kin = np.asarray(new_kin, bool)
    f = st.f.copy()
    U = st.U.copy()
    down = st.kin & ~new_kin
    if down.any():
        U[:, down] = _U_of_f(prob, st.f[down])
    up = new_kin & ~st.kin
    if up.any():
        f[up] = _mhat_of_U(prob, U[:, up])
    return State(f=f, U=U, kin=new_kin.copy(), eps=st.eps)


def _interface_fluxes(prob, f, kin, v, w):
    """Face-flux overrides of the conservative interface (Reading R22): the
    moments of the kinetic numerical flux at every face with a kinetic cell on
    one side and a fluid cell on the other (the faces i-1/2 of the ghost-padded
    map, as in the transport).  f must hold f in the kinetic and buffer cells,
    which cover the stencils of those faces."""
    Fx, Fy = kinetic_face_fluxes(f, v, prob.bc_x, prob.bc_y, prob.cweno_eps, prob.walls)
    out = []
    for F, axis, bc in ((Fx, 1, prob.bc_x), (Fy, 0, prob.bc_y)):
        k = pad_cells(kin, axis, bc, n=1)
        n = kin.shape[axis]
        left = np.take(k, np.arange(0, n + 1), axis=axis)
        right = np.take(k, np.arange(1, n + 2), axis=axis)
        out.append((flux_moments(F, v, w), left != right))
    return tuple(out)


def advance(prob, st, dt, tab):
    """One step of Algorithm 1 with the regime map held fixed.

    Stage i (Eqs. RKEuler, RKEI1, with Abar = At, bbar = bt, Sec. 3.4):
      fluid cells:   U^(i) = U^n - dt sum_{j<i} at_ij Phi(U^(j))
      kinetic cells: f^(i) = f^n - dt sum_{j<i} at_ij L(f^(j))
                              + dt sum_{j<=i} a_ij nu (G_hat[f^(j)] - f^(j)),
                     the j = i term solved by ``relax``;
      coupling: U^(i) := moments(f^(i)) in kinetic cells, f^(i) := M_hat[U^(i)]
      in the buffer cells (Remark rem_coupling).  With coupling='step' the
      buffer keeps f^n's reconstruction and kinetic cells keep U^n during the
      stages (LOC-hybrid).
    Final (Eqs. RKEI2, RKEuler_2): f^{n+1} = f^n - dt sum bt_i L_i
    + dt sum b_i Q_i, U^{n+1} = U^n - dt sum bt_i Phi_i, then coupling.
    Reading R11: each cell uses its own model's flux.
    """
    v, w = _vgrid(prob)
    kin = st.kin
    buf = buffer_mask(prob, kin)
    nu = prob.tau / st.eps
    s = tab.s
    args = (prob.dx, prob.dy, prob.bc_x, prob.bc_y, prob.cweno_eps)
    walls = prob.walls
    fluid_only = 1.0 if walls is None else (~walls[0]).astype(np.float64)  # solid cells keep U

    U_n = st.U.copy()
    f_n = np.zeros_like(st.f)
    f_n[kin] = st.f[kin]
    if kin.any():
        U_n[:, kin] = _U_of_f(prob, f_n[kin])
    if buf.any():
        f_n[buf] = _mhat_of_U(prob, U_n[:, buf])

    Ls, Qs, Phis = [], [], []
    for i in range(s):
        U_i = U_n.copy()
        for j in range(i):
            U_i -= dt * tab.At[i, j] * Phis[j]
        f_i = np.zeros_like(f_n)
        Q_i = np.zeros_like(f_n)
        if kin.any():
            fstar = f_n[kin].copy()
            for j in range(i):
                fstar -= dt * tab.At[i, j] * Ls[j][kin]
                fstar += dt * tab.A[i, j] * Qs[j][kin]
            # collision rate of the stage (Reading R23: with tau = tau rho, the
            # density of f*, equal to that of f^(i))
            nu_i = nu[kin] * (_U_of_f(prob, fstar)[0] if prob.tau_model == "density" else 1.0)
            if tab.A[i, i] != 0.0:
                f_i[kin], _ = relax(fstar, dt * tab.A[i, i] * nu_i, prob.beta, v, w)
            else:
                f_i[kin] = fstar
            needQ = tab.b[i] != 0.0 or np.any(tab.A[i + 1:, i] != 0.0)
            if needQ:
                g = f_i[kin]
                Q_i[kin] = nu_i[:, None, None] * (es_gaussian_of(g, v, w, prob.beta) - g)
        if prob.coupling == "stage":
            if kin.any():
                U_i[:, kin] = _U_of_f(prob, f_i[kin])
            if buf.any():
                f_i[buf] = _mhat_of_U(prob, U_i[:, buf])
        else:
            U_i[:, kin] = U_n[:, kin]
            f_i[buf] = f_n[buf]
        Ls.append(kinetic_transport(f_i, v, *args, walls=walls))
        if prob.interface == "conservative" and kin.any() and not kin.all():
            Phis.append(fluid_only * euler_phi(U_i, *args, override=_interface_fluxes(prob, f_i, kin, v, w),
                                               walls=walls))
        else:
            Phis.append(fluid_only * euler_phi(U_i, *args, walls=walls))
        Qs.append(Q_i)

    f_new = st.f.copy()
    U_new = U_n.copy()
    for i in range(s):
        U_new -= dt * tab.bt[i] * Phis[i]
    if kin.any():
        g = f_n[kin].copy()
        for i in range(s):
            g -= dt * tab.bt[i] * Ls[i][kin]
            g += dt * tab.b[i] * Qs[i][kin]
        f_new[kin] = g
        U_new[:, kin] = _U_of_f(prob, g)
    return State(f=f_new, U=U_new, kin=kin.copy(), eps=st.eps)


def step(prob, st, dt, tab):
    """Algorithm 1, one time step: regime update (plain switch), conversion,
    then the coupled stages."""
    if prob.switch == "plain":
        st = convert(prob, st, regime_update(prob, st))
    return advance(prob, st, dt, tab)


def with_switch(prob, switch):
    return replace(prob, switch=switch)
