"""Seeded synthetic inputs shaped like the paper's 2-D tests.

This module only draws input fields and names problem parameters.  It holds
none of the method's arithmetic (no moments, no Maxwellians, no fluxes), so it
can feed both the CUDA library and the CPU oracle without coupling them.

Every generator returns a plain dict:
  grid   -- nx, ny, x0, x1, y0, y1, bc_x, bc_y ('periodic' | 'outflow')
  vmesh  -- nv, vmax
  params -- beta, tau, eta_factor, delta, cweno_eps, switch, coupling
  scheme -- 'ars233' | 'imex_euler'
  dt, steps
  fields -- rho, ux, uy, T, eps (float64 [ny, nx]) and kin (bool [ny, nx])

The paper's workloads are analytic initial conditions (Test 1-6, Sec. 4), not
datasets; these stand in for them at the sizes of the benchmark configurations.
"""

import numpy as np

PARAMS = dict(beta=-0.5, tau=1.0, eta_factor=1.0, delta=1e-3, cweno_eps=1e-6,
              switch="frozen", coupling="stage")


def _centres(nx, ny, x0, x1, y0, y1):
    x = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    y = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    return np.meshgrid(x, y)


def _dt(cfl, nx, ny, x0, x1, y0, y1, vmax):
    """dt = CFL min(dx, dy) / v_max, the time-step rule of Tests 2-6."""
    return cfl * min((x1 - x0) / nx, (y1 - y0) / ny) / vmax


def sine_periodic(nx=32, ny=32, nv=16, vmax=6.0, eps=1e-2, steps=10, cfl=0.5,
                  scheme="imex_euler"):
    """Plain ES-BGK, all kinetic, periodic [0,1]^2:
    rho = 1 + 0.2 sin(2 pi x) sin(2 pi y), u = 0, T = 1, uniform eps."""
    X, Y = _centres(nx, ny, 0, 1, 0, 1)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    z = np.zeros_like(rho)
    return dict(
        grid=dict(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="periodic", bc_y="periodic"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS), scheme=scheme,
        dt=_dt(cfl, nx, ny, 0, 1, 0, 1, vmax), steps=steps,
        fields=dict(rho=rho, ux=z.copy(), uy=z.copy(), T=np.ones_like(rho),
                    eps=np.full_like(rho, eps), kin=np.ones(rho.shape, bool)))


def sod_tube(nx=21, ny=150, nv=32, vmax=8.0, eps=1e-6, initial="fluid", switch="plain", t_end=0.15):
    """Test 2 (Sec. 4.1.2): Sod data along y on [0, 0.1] x [0, 1], uniform
    along x (periodic in x, outflow in y): (rho, u, p) = (1, 0, 1) for
    y <= 0.5, (1/8, 0, 1/32) above; T = p / rho.  eps = 1e-6, plain switch
    with eta = eps, delta = 1e-3, all cells macroscopic at t = 0 (initial =
    'fluid'; 'kinetic' for the full kinetic run).  dt = t_end / steps with
    steps = ceil(t_end / (0.8 min(dx, dy) / vmax)): at most the rule's value."""
    X, Y = _centres(nx, ny, 0, 0.1, 0, 1)
    left = Y <= 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 1.0 / 32.0)
    z = np.zeros_like(rho)
    dx, dy = 0.1 / nx, 1.0 / ny
    steps = int(np.ceil(t_end / (0.8 * min(dx, dy) / vmax)))
    kin = np.zeros(rho.shape, bool) if initial == "fluid" else np.ones(rho.shape, bool)
    return dict(
        grid=dict(nx=nx, ny=ny, x0=0.0, x1=0.1, y0=0.0, y1=1.0, bc_x="periodic", bc_y="outflow"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS, switch=switch), scheme="ars233",
        dt=t_end / steps, steps=steps,
        fields=dict(rho=rho, ux=z, uy=z.copy(), T=p / rho, eps=np.full_like(rho, eps), kin=kin))


def riemann_quadrants(nx=128, ny=128, nv=32, vmax=8.0, seed=0, steps=200, cfl=0.5,
                      t_range=(0.25, 3.0), scheme="ars233", initial="fluid"):
    """Coupled ES-BGK/Euler four-quadrant 2-D Riemann data on [0,1]^2, outflow.

    Per quadrant rho, p ~ U[0.1, 1.5] and |u| ~ U[0, 0.7] at a uniform angle,
    redrawn until T = p/rho lies in t_range so that the velocity grid resolves
    the Maxwellians.  log10 eps = -2.5 + 1.5 sin(2 pi x) sin(2 pi y), a smooth
    field between 1e-4 and 1e-1.  Plain switch with eta = eps, delta = 1e-3.
    initial='fluid' starts all cells macroscopic, as the Sod test of Sec. 4.
    """
    rng = np.random.default_rng(seed)
    X, Y = _centres(nx, ny, 0, 1, 0, 1)
    rho = np.empty_like(X)
    ux = np.empty_like(X)
    uy = np.empty_like(X)
    T = np.empty_like(X)
    for qx in (0, 1):
        for qy in (0, 1):
            while True:
                r, p = rng.uniform(0.1, 1.5, size=2)
                if t_range[0] <= p / r <= t_range[1]:
                    break
            mag = rng.uniform(0.0, 0.7)
            ang = rng.uniform(0.0, 2 * np.pi)
            m = ((X >= 0.5) == bool(qx)) & ((Y >= 0.5) == bool(qy))
            rho[m], T[m] = r, p / r
            ux[m], uy[m] = mag * np.cos(ang), mag * np.sin(ang)
    eps = 10.0 ** (-2.5 + 1.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y))
    kin = np.zeros(X.shape, bool) if initial == "fluid" else np.ones(X.shape, bool)
    params = dict(PARAMS, switch="plain")
    return dict(
        grid=dict(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="outflow", bc_y="outflow"),
        vmesh=dict(nv=nv, vmax=vmax), params=params, scheme=scheme,
        dt=_dt(cfl, nx, ny, 0, 1, 0, 1, vmax), steps=steps,
        fields=dict(rho=rho, ux=ux, uy=uy, T=T, eps=eps, kin=kin))


def gaussian_blob(nx=256, ny=256, nv=48, vmax=8.0, eps=1e-3, steps=100, cfl=0.5,
                  amp=0.5, width=0.1, u0=(0.3, 0.0), T0=1.0, scheme="ars233"):
    """Precision form: periodic [0,1]^2, all kinetic,
    rho = 1 + amp exp(-|x - (1/2,1/2)|^2 / width^2), u = u0, T = T0."""
    X, Y = _centres(nx, ny, 0, 1, 0, 1)
    rho = 1.0 + amp * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / width ** 2)
    return dict(
        grid=dict(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="periodic", bc_y="periodic"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS), scheme=scheme,
        dt=_dt(cfl, nx, ny, 0, 1, 0, 1, vmax), steps=steps,
        fields=dict(rho=rho, ux=np.full_like(rho, u0[0]), uy=np.full_like(rho, u0[1]),
                    T=np.full_like(rho, T0), eps=np.full_like(rho, eps),
                    kin=np.ones(rho.shape, bool)))


def learned_switch_case(nx=512, ny=512, nv=32, vmax=8.0, seed=0, steps=200, cfl=0.5, blob_amp=0.5,
                        blob_width=0.1, blob_centre=(0.3, 0.7), scheme="ars233"):
    """Learned-switch deployment: the four-quadrant Riemann data of
    riemann_quadrants (same eps field, outflow, starting all fluid) with a
    Gaussian density blob of amplitude blob_amp and width blob_width added at
    blob_centre; 'learned' switch, ARS(2,3,3)."""
    wl = riemann_quadrants(nx=nx, ny=ny, nv=nv, vmax=vmax, seed=seed, steps=steps, cfl=cfl, scheme=scheme)
    X, Y = _centres(nx, ny, 0, 1, 0, 1)
    bump = blob_amp * np.exp(-((X - blob_centre[0]) ** 2 + (Y - blob_centre[1]) ** 2) / blob_width ** 2)
    wl["fields"]["rho"] = wl["fields"]["rho"] * (1.0 + bump)
    wl["params"] = dict(wl["params"], switch="learned")
    return wl


def order_test(n=90, nv=32, vmax=5.0, L=6.0, eps=1e-2, seed=0, kin_fraction=0.5,
               coupling="stage"):
    """Test 1 (Sec. 4.1.1): [0,6]^2 periodic, rho = 1 + 0.1 exp(-3 d^2),
    T = 0.3 (1 + 0.1 exp(-3 d^2)), u = 0, d the distance to the centre, and a
    random regime map frozen for the whole run."""
    rng = np.random.default_rng(seed)
    X, Y = _centres(n, n, 0, L, 0, L)
    d2 = (X - L / 2) ** 2 + (Y - L / 2) ** 2
    bump = 0.1 * np.exp(-3.0 * d2)
    rho = 1.0 + bump
    T = 0.3 * (1.0 + bump)
    z = np.zeros_like(rho)
    kin = rng.uniform(size=rho.shape) < kin_fraction
    return dict(
        grid=dict(nx=n, ny=n, x0=0.0, x1=L, y0=0.0, y1=L, bc_x="periodic", bc_y="periodic"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS, coupling=coupling),
        scheme="ars233", dt=None, steps=None,
        fields=dict(rho=rho, ux=z.copy(), uy=z.copy(), T=T, eps=np.full_like(rho, eps), kin=kin))


def random_cells(n, nv, vmax, seed=0, anisotropy=0.3):
    """Random positive per-cell distributions (n, nv, nv): a Gaussian-like
    bump with random centre, widths and tilt times a random positive factor.
    Used for per-cell kernel checks (collision, moments)."""
    rng = np.random.default_rng(seed)
    dv = 2.0 * vmax / nv
    v = -vmax + (np.arange(nv) + 0.5) * dv
    VX, VY = np.meshgrid(v, v)
    out = np.empty((n, nv, nv))
    for c in range(n):
        cx, cy = rng.uniform(-0.5, 0.5, size=2)
        sx, sy = rng.uniform(0.7, 1.4, size=2)
        tilt = rng.uniform(-anisotropy, anisotropy)
        q = ((VX - cx) / sx) ** 2 + ((VY - cy) / sy) ** 2 + 2 * tilt * (VX - cx) * (VY - cy) / (sx * sy)
        out[c] = rng.uniform(0.5, 1.5) * np.exp(-0.5 * q) * (1 + 0.2 * rng.uniform(size=(nv, nv)))
    return out


def batched_cases(n_cases=64, seed0=0, sizes=None, nvs=None, steps=100):
    """Batched form: independent periodic cases of uneven sizes.

    Case c (seed = seed0 + c): N_x = N_y from {64, 80, ..., 256}, N_v from
    {16, 18, ..., 40}, v_max = 8, eps log-uniform in [1e-4, 1e-1], rho and T
    random smooth fields (4 Fourier modes, wavenumber <= 3) mapped affinely
    into [0.5, 1.5] and [0.5, 2], u = 0, plain switch, ARS(2,3,3).
    """
    sizes = list(range(64, 257, 16)) if sizes is None else list(sizes)
    nvs = list(range(16, 41, 2)) if nvs is None else list(nvs)
    cases = []
    for c in range(n_cases):
        rng = np.random.default_rng(seed0 + c)
        n = int(rng.choice(sizes))
        nv = int(rng.choice(nvs))
        X, Y = _centres(n, n, 0, 1, 0, 1)

        def smooth():
            acc = np.zeros_like(X)
            for _ in range(4):
                kx, ky = rng.integers(0, 4, size=2)
                ph = rng.uniform(0, 2 * np.pi)
                acc += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
            lo, hi = acc.min(), acc.max()
            return (acc - lo) / (hi - lo) if hi > lo else np.zeros_like(acc)

        rho = 0.5 + smooth()
        T = 0.5 + 1.5 * smooth()
        eps = 10.0 ** rng.uniform(-4, -1)
        z = np.zeros_like(rho)
        cases.append(dict(
            grid=dict(nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="periodic", bc_y="periodic"),
            vmesh=dict(nv=nv, vmax=8.0), params=dict(PARAMS, switch="plain"), scheme="ars233",
            dt=_dt(0.5, n, n, 0, 1, 0, 1, 8.0), steps=steps,
            fields=dict(rho=rho, ux=z.copy(), uy=z.copy(), T=T, eps=np.full_like(rho, eps),
                        kin=np.ones(rho.shape, bool))))
    return cases


def obstacle_flow(kind="cylinder", n=78, nv=32, vmax=8.0, eps=1e-6, eta_factor=10.0, t_end=0.15, cfl=0.5,
                  initial="fluid", switch="plain"):
    """Tests 5 and 6 (Sec. 4.2.3-4.2.4): flow u = (2, 0), rho = 1, p = 1 on
    [0,1]^2 (n x n cells, outflow edges) toward a solid cylinder of radius 1/12
    (kind='cylinder') or a rectangle of 10 x 4 cells (kind='rectangle')
    centred at (2/5, 1/2); eps = 1e-6, eta = 10 eps, delta = 1e-3, 32^2
    velocities on [-8, 8]^2, dt = 0.5 min(dx, dy)/8 to t_end = 0.15.
    'solid' in the result is the obstacle mask (cell centres inside it)."""
    X, Y = _centres(n, n, 0, 1, 0, 1)
    xc, yc = 0.4, 0.5
    if kind == "cylinder":
        solid = (X - xc) ** 2 + (Y - yc) ** 2 < (1.0 / 12.0) ** 2
    else:
        solid = (np.abs(X - xc) < 5.0 / n) & (np.abs(Y - yc) < 2.0 / n)
    rho = np.ones_like(X)
    dt0 = _dt(cfl, n, n, 0, 1, 0, 1, vmax)
    steps = int(np.ceil(t_end / dt0))
    kin = np.zeros(X.shape, bool) if initial == "fluid" else np.ones(X.shape, bool)
    return dict(
        grid=dict(nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="outflow", bc_y="outflow"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS, switch=switch, eta_factor=eta_factor), scheme="ars233",
        dt=t_end / steps, steps=steps,
        fields=dict(rho=rho, ux=np.full_like(rho, 2.0), uy=np.zeros_like(rho), T=np.ones_like(rho),
                    eps=np.full_like(rho, eps), kin=kin),
        solid=solid)


def kelvin_helmholtz(nx=150, ny=75, nv=32, vmax=8.0, eps=1e-6, t_end=1.7, cfl=0.5, steps=None,
                     initial="kinetic", switch="plain"):
    """Test 3 (Sec. 4.2.1): shear layer on [0, 1] x [0, 0.5] (periodic in x,
    outflow in y), (rho, u_x, p) = (2, -0.5, 1) for y <= 1/4 and (1, 0.5, 1)
    above, u_y = 0.01 sin(4 pi x), T = p / rho; eps = 1e-6, plain switch with
    eta = 4 eps, delta = 1e-3; every cell starts kinetic with f the Maxwellian
    of its state ('fluid': all macroscopic).  dt = 0.5 min(dx, dy) / 8 to
    t_end = 1.7 (steps: fewer, for a shortened run)."""
    X, Y = _centres(nx, ny, 0, 1, 0, 0.5)
    low = Y <= 0.25
    rho = np.where(low, 2.0, 1.0)
    ux = np.where(low, -0.5, 0.5)
    uy = 0.01 * np.sin(4 * np.pi * X)
    dt = _dt(cfl, nx, ny, 0, 1, 0, 0.5, vmax)
    n = int(np.ceil(t_end / dt - 1e-9)) if steps is None else steps
    kin = np.full(X.shape, initial == "kinetic")
    return dict(
        grid=dict(nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=0.5, bc_x="periodic", bc_y="outflow"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS, switch=switch, eta_factor=4.0), scheme="ars233",
        dt=dt, steps=n,
        fields=dict(rho=rho, ux=ux, uy=uy, T=1.0 / rho, eps=np.full_like(rho, eps), kin=kin))


def shock_bubble(nx=150, ny=50, nv=32, vmax=8.0, eps=1e-6, t_end=1.5, cfl=0.5, steps=None,
                 initial="kinetic", switch="plain"):
    """Test 4 (Sec. 4.2.2): on [-2, 3] x [-0.5, 0.5] (outflow edges) a shock
    state (rho, u_x, p) = (16/7, sqrt(5/3) 7/16, 4.75) for x <= -1 runs into
    (1 + 1.5 exp(-16 d^2), 0, 1), d the distance to (0.5, 0); u_y = 0,
    T = p / rho; eps = 1e-6, plain switch with eta = eps/2, delta = 1e-3;
    every cell starts kinetic with f the Maxwellian of its state.
    dt = 0.5 min(dx, dy) / 8 to t_end = 1.5."""
    X, Y = _centres(nx, ny, -2, 3, -0.5, 0.5)
    left = X <= -1.0
    d2 = (X - 0.5) ** 2 + Y ** 2
    rho = np.where(left, 16.0 / 7.0, 1.0 + 1.5 * np.exp(-16.0 * d2))
    ux = np.where(left, np.sqrt(5.0 / 3.0) * 7.0 / 16.0, 0.0)
    p = np.where(left, 4.75, 1.0)
    dt = _dt(cfl, nx, ny, -2, 3, -0.5, 0.5, vmax)
    n = int(np.ceil(t_end / dt - 1e-9)) if steps is None else steps
    kin = np.full(X.shape, initial == "kinetic")
    return dict(
        grid=dict(nx=nx, ny=ny, x0=-2.0, x1=3.0, y0=-0.5, y1=0.5, bc_x="outflow", bc_y="outflow"),
        vmesh=dict(nv=nv, vmax=vmax), params=dict(PARAMS, switch=switch, eta_factor=0.5), scheme="ars233",
        dt=dt, steps=n,
        fields=dict(rho=rho, ux=ux, uy=np.zeros_like(rho), T=p / rho, eps=np.full_like(rho, eps), kin=kin))
