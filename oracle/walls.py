"""Solid obstacles with specular reflection (Sec. 4.2.3-4.2.4, Tests 5 and 6).

Test infrastructure only (see the package docstring).

The paper places a solid cylinder (Test 5) or rectangle (Test 6) inside the
domain: no integrator runs in it, and its surface reflects specularly
(Cercignani).  It gives no discretisation of the wall.  Reading R24: cells
whose centre lies in the obstacle are solid; they hold no state.  Every
stencil value a fluid cell needs from beyond a wall is the mirror image,
across that wall face, of a fluid cell on its own side, with the velocity
reflected in the wall's normal:
  f(v_n, v_t) -> f(-v_n, v_t)           (specular reflection of the kinetic
                                          distribution; on the midpoint grid
                                          v_n -> -v_n reverses the node index)
  (rho, m_n, m_t, E) -> (rho, -m_n, m_t, E)   (mirror state of the Euler ghost)
Along an axis, for a cell c and the stencil position p = c + d (d = +-1, +-2):
if a solid cell lies between c and p (inclusive of p), let w be the first one
and a = w - sign(d) the last fluid cell before it; p is replaced by its mirror
p' = 2a + sign(d) - p across the face between a and w, reflected; if p' is
itself solid (a fluid gap narrower than the stencil), a is used.  A solid
cell's reconstructed value at a face it shares with a fluid cell is the
reflection of the fluid cell's value at that face.  So the numerical flux
through a wall face is computed from a state and its mirror: the kinetic
mass and energy fluxes through it vanish exactly (the velocity grid is
symmetric), and so do the Euler ones.  Obstacles stay at least three cells
away from an outflow edge of the domain (the boundary condition applies
before the wall rule and never meets it); a periodic axis wraps.
"""

import numpy as np

OFFSETS = (-2, -1, 0, 1, 2)


def check_solid(solid, bc_x="periodic", bc_y="periodic"):
    """Validate a solid mask (ny, nx): no solid cell within 3 cells of an
    outflow edge (a periodic axis wraps, so walls may cross it)."""
    solid = np.asarray(solid, bool)
    if solid.any():
        J, I = np.nonzero(solid)
        ny, nx = solid.shape
        if bc_x != "periodic" and (I.min() < 3 or I.max() > nx - 4):
            raise ValueError("obstacles must stay three cells away from an outflow edge")
        if bc_y != "periodic" and (J.min() < 3 or J.max() > ny - 4):
            raise ValueError("obstacles must stay three cells away from an outflow edge")
    return solid


def _bc(i, n, bc):
    if bc == "periodic":
        return i % n
    return min(max(i, 0), n - 1)


def stencil_maps(solid, bc_x, bc_y):
    """Per axis (0: x, 1: y) the stencil of every cell: src[5, ny, nx] flat
    cell indices of the values at offsets -2..2 and refl[5, ny, nx] whether the
    value is reflected (a mirror image across a wall).  Solid centres map to
    themselves (unused)."""
    solid = np.asarray(solid, bool)
    ny, nx = solid.shape
    out = []
    for axis in (0, 1):
        n, bc = (nx, bc_x) if axis == 0 else (ny, bc_y)
        src = np.zeros((5, ny, nx), np.int64)
        refl = np.zeros((5, ny, nx), bool)
        for j in range(ny):
            for i in range(nx):
                c = i if axis == 0 else j

                def cell(pos):
                    q = _bc(pos, n, bc)
                    return (j, q) if axis == 0 else (q, i)

                def is_solid(pos):
                    return solid[cell(pos)]

                for k, d in enumerate(OFFSETS):
                    p = c + d
                    if d == 0 or solid[j, i]:
                        jj, ii = cell(p) if d else (j, i)
                        src[k, j, i] = jj * nx + ii
                        continue
                    sg = 1 if d > 0 else -1
                    w = None
                    for s in range(c + sg, p + sg, sg):
                        if is_solid(s):
                            w = s
                            break
                    if w is None:
                        jj, ii = cell(p)
                        src[k, j, i] = jj * nx + ii
                        continue
                    a = w - sg
                    pm = 2 * a + sg - p
                    if is_solid(pm):
                        pm = a
                    jj, ii = cell(pm)
                    src[k, j, i] = jj * nx + ii
                    refl[k, j, i] = True
        out.append((src, refl))
    return out


def reflect_f(g, axis):
    """Specular reflection of distributions g (..., nv_y, nv_x) in the wall
    normal to `axis` (0: v_x -> -v_x, 1: v_y -> -v_y)."""
    return g[..., ::-1] if axis == 0 else g[..., ::-1, :]


def reflect_U(U, axis):
    """Mirror state of conserved variables U (..., 4): the normal momentum
    changes sign."""
    out = U.copy()
    out[..., 1 + axis] *= -1.0
    return out


def line_values(q, maps, axis, reflect):
    """The stencil values of every cell along `axis`: list over offsets
    -2..2 of arrays shaped like q (cells first: (ny, nx, ...))."""
    src, refl = maps[axis]
    ny, nx = q.shape[:2]
    flat = q.reshape((ny * nx,) + q.shape[2:])
    vals = []
    for k in range(5):
        g = flat[src[k]]
        if refl[k].any():
            g[refl[k]] = reflect(g[refl[k]], axis)
        vals.append(g)
    return vals


def face_states(q, solid, maps, axis, bc, eps_w, reflect, recon):
    """States left (q^-) and right (q^+) of the faces i-1/2 (i = 0..n) along
    `axis` with the wall rule; q is cells first (ny, nx, ...), the result has
    n+1 faces along `axis`.  recon(qm, q0, qp) -> (left face, right face)."""
    solid = np.asarray(solid, bool)
    vals = line_values(q, maps, axis, reflect)
    Lf, Rf = recon(vals[1], vals[2], vals[3])
    Lf, Rf = Lf.copy(), Rf.copy()
    ny, nx = solid.shape
    n = nx if axis == 0 else ny
    # a solid cell's value at a face it shares with a fluid cell: the reflection
    for j, i in zip(*np.nonzero(solid)):
        c = i if axis == 0 else j
        cl, ch = _bc(c - 1, n, bc), _bc(c + 1, n, bc)
        lo = (j, cl) if axis == 0 else (cl, i)
        hi = (j, ch) if axis == 0 else (ch, i)
        if not solid[lo]:
            Lf[j, i] = reflect(Rf[lo][None], axis)[0]
        if not solid[hi]:
            Rf[j, i] = reflect(Lf[hi][None], axis)[0]
    ax = 1 if axis == 0 else 0
    take = lambda a, idx: np.take(a, idx, axis=ax)
    if bc == "periodic":
        left_ghost_R, right_ghost_L = take(Rf, [n - 1]), take(Lf, [0])
    else:
        left_ghost_R, right_ghost_L = take(q, [0]), take(q, [n - 1])
    qminus = np.concatenate([left_ghost_R, take(Rf, np.arange(n))], axis=ax)
    qplus = np.concatenate([take(Lf, np.arange(n)), right_ghost_L], axis=ax)
    return qminus, qplus


def neighbour_values(q, maps, axis, reflect):
    """Values of the neighbours at offsets -1 and +1 along `axis` with the wall
    rule (for the criterion's central differences)."""
    vals = line_values(q, maps, axis, reflect)
    return vals[1], vals[3]
