"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 storage -- relative L1 <= 1e-10 on the macroscopic fields
(rho, E; momentum relative to rho) and on f; FP32 storage -- <= 1e-5.  Flags
must be identical except in cells within 1e-6 (FP64) or 1e-3 (FP32 storage)
relative of a threshold (lambda_A vs eta, or the L1 deviation vs delta),
where the oracle's flag is imposed on the library so that the fields stay
comparable.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def gpu_solver(wl, prec="fp64", **over):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], **over), prec=prec)
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    return s


# parameters of the library's arithmetic that the FP64 oracle has no use for
LIBRARY_ONLY = ("moment_sums",)


def oracle_pair(wl, **over):
    params = {k: v for k, v in dict(wl["params"], **over).items() if k not in LIBRARY_ONLY}
    P = O.Problem(**wl["grid"], **wl["vmesh"], **params)
    return P, O.init_state(P, **wl["fields"])


def field_errors(U_gpu, U_ref):
    """Relative L1 errors of (rho, m_x, m_y, E); momentum is measured against
    the L1 norm of rho (a velocity scale of one)."""
    r = np.abs(U_ref[0]).sum()
    return (np.abs(U_gpu[0] - U_ref[0]).sum() / r,
            np.abs(U_gpu[1] - U_ref[1]).sum() / r,
            np.abs(U_gpu[2] - U_ref[2]).sum() / r,
            np.abs(U_gpu[3] - U_ref[3]).sum() / np.abs(U_ref[3]).sum())


def f_error(f_gpu, f_ref, kin):
    if not kin.any():
        return 0.0
    a, b = f_gpu[kin], f_ref[kin]
    return np.abs(a - b).sum() / np.abs(b).sum()


def tableau_of(name):
    return {"ars233": O.ARS233, "imex_euler": O.IMEX_EULER, "ars222": O.ARS222, "ssp2_332": O.SSP2_332}[name]


def run_parity(wl, steps, prec="fp64", check_f=True, **over):
    """Advance library and oracle side by side; return the worst errors."""
    g = gpu_solver(wl, prec, **over)
    P, st = oracle_pair(wl, **over)
    tab = tableau_of(wl["scheme"])
    worst = np.zeros(5)
    exempt_total = 0
    for n in range(steps):
        if P.switch == "plain":
            g.regime_update()
            lam_o, l1_o = O.regime_indicators(P, st)
            new_o = (lam_o > P.eta_factor * st.eps) | (st.kin & (l1_o > P.delta))
            flags_g = g.flags()
            lam_g, l1_g = g.indicators()
            # indicators agree to round-off on the scale of the threshold they
            # are compared with (values far below eta or delta only need to stay below)
            # FP32 storage: the L1 sum of |f - M| carries ~1e-7 absolute rounding
            tol_ind = 1e-9 if prec == "fp64" else 1e-3
            eta = P.eta_factor * st.eps
            assert np.all(np.abs(lam_g - lam_o) <= tol_ind * np.maximum(np.abs(lam_o), eta)), "lambda_A"
            dl1 = np.abs(l1_g - l1_o)[st.kin]
            # FP64: f itself agrees to 1e-10 relative L1 (the field bar), so
            # the L1 norm of f - M may move by 1e-10 of the cell's density
            slack = 1e-10 * np.abs(st.U[0][st.kin]) if prec == "fp64" else 0.0
            assert np.all(dl1 <= tol_ind * np.maximum(l1_o[st.kin], P.delta) + slack), "L1"
            bad = flags_g != new_o
            near = (np.abs(lam_o - eta) <= 1e-6 * np.maximum(eta, 1e-300)) | \
                   (st.kin & (np.abs(l1_o - P.delta) <= 1e-6 * P.delta))
            if prec != "fp64":
                near |= (np.abs(lam_o - eta) <= 1e-3 * eta) | (st.kin & (np.abs(l1_o - P.delta) <= 1e-3 * P.delta))
            assert not (bad & ~near).any(), "flag mismatch away from thresholds at %s" % np.argwhere(bad & ~near)[:5]
            if bad.any():
                exempt_total += int(bad.sum())
                g.set_flags(new_o)
            st = O.convert(P, st, new_o)
        g.advance(wl["dt"], wl["scheme"])
        st = O.advance(P, st, wl["dt"], tab)
        e = field_errors(g.cons(), st.U)
        worst[:4] = np.maximum(worst[:4], e)
        if check_f:
            worst[4] = max(worst[4], f_error(g.f(), st.f, st.kin))
    return worst, g, P, st, exempt_total


# ---------------------------------------------------------------------------
# per-cell collision kernel

@pytest.mark.parametrize("nv,vmax", [(16, 6.0), (32, 8.0), (15, 6.0), (48, 8.0), (64, 8.0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_relax_cells_matches_oracle(nv, vmax, prec):
    import torch
    import paper_2512_03586_gb300 as G
    n = 37
    fs = W.random_cells(n, nv, vmax, seed=nv)
    h = np.geomspace(1e-3, 1e6, n)
    v, w = O.velocity_grid(nv, vmax)
    f_ref, g_ref = O.relax(fs, h, -0.5, v, w)
    dt = torch.float64 if prec == "fp64" else torch.float32
    f, g = G.relax_cells(torch.tensor(fs, dtype=dt, device="cuda"), torch.tensor(h, device="cuda"), vmax,
                         beta=-0.5, prec=prec)
    torch.cuda.synchronize()
    f, g = f.double().cpu().numpy(), g.double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    scale = np.abs(f_ref).max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(f - f_ref) / scale) < tol
    assert np.max(np.abs(g - g_ref) / scale) < tol
    if prec == "fp64":
        # exact conservation on the grid (H1)
        m_ref = O.moments(fs, v, w)
        m = O.moments(f, v, w)
        assert np.allclose(m[:, :3], m_ref[:, :3], rtol=1e-13, atol=1e-14)
        assert np.allclose(m[:, 3] + m[:, 5], m_ref[:, 3] + m_ref[:, 5], rtol=1e-13)


# ---------------------------------------------------------------------------
# whole steps

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sine_periodic_imex_euler_full_config(prec):
    """Plain ES-BGK, 32^2 periodic, 16^2 velocities on [-6,6]^2, eps = 1e-2,
    Pr = 2/3, IMEX-Euler, CFL 0.5, 10 steps -- at its full size."""
    wl = W.sine_periodic()
    worst, g, P, st, _ = run_parity(wl, wl["steps"], prec)
    assert worst.max() <= TOL[prec], worst
    tot = g.totals()
    tot0 = O.totals(P, oracle_pair(wl)[1])
    assert abs(tot[0] - tot0[0]) <= (1e-13 if prec == "fp64" else 1e-6) * tot0[0]
    assert abs(tot[3] - tot0[3]) <= (1e-13 if prec == "fp64" else 1e-6) * tot0[3]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ars233_all_kinetic_blob(prec):
    wl = W.gaussian_blob(nx=16, ny=12, nv=16, steps=3)
    worst, *_ = run_parity(wl, 3, prec)
    assert worst.max() <= TOL[prec], worst


@pytest.mark.parametrize("coupling", ["stage", "step"])
def test_hybrid_frozen_random_map(coupling):
    """Test 1 setting (random frozen regime map) with per-stage and end-of-step
    coupling: kinetic, buffer and fluid cells all active, ragged lists."""
    wl = W.order_test(n=17, nv=12, eps=1e-2, coupling=coupling, seed=2)
    wl["dt"] = 0.2 / 8
    worst, *_ = run_parity(wl, 3, "fp64")
    assert worst.max() <= TOL["fp64"], worst


def test_riemann_plain_switch_small():
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3)
    worst, g, P, st, ex = run_parity(wl, 6, "fp64")
    assert worst.max() <= TOL["fp64"], worst
    assert 0 < st.kin.sum() < st.kin.size


def test_riemann_plain_switch_fp32():
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=4)
    worst, *_ = run_parity(wl, 4, "fp32")
    assert worst.max() <= TOL["fp32"], worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_criterion_in_nearly_uniform_flow(prec):
    """Sec. 3.1.2's lambda_A where the flow is uniform up to rounding: with
    eps = 1e-12 and density ripples of 1e-14, (X_xx - X_yy)^2/4 + X_xy^2 is
    ~1e-49, below float's range; the criterion must stay finite and equal the
    oracle's, and no cell turns kinetic."""
    wl = W.obstacle_flow("cylinder", n=30, nv=16)
    rng = np.random.default_rng(7)
    f = wl["fields"]
    f["rho"] = f["rho"] * (1.0 + 1e-14 * rng.standard_normal(f["rho"].shape))
    f["eps"] = np.full_like(f["eps"], 1e-12)
    g = gpu_solver(wl, prec)
    P, st = oracle_pair(wl)
    g.regime_update()
    lam_g, _ = g.indicators()
    lam_o, _ = O.regime_indicators(P, st)
    eta = P.eta_factor * st.eps
    assert np.isfinite(lam_g).all()
    assert lam_o.max() < 1e-20
    assert np.all(np.abs(lam_g - lam_o) <= 1e-9 * np.maximum(lam_o, eta))
    assert not g.flags().any()


def test_riemann_full_size_first_steps():
    """Coupled configuration at its full size (128^2 cells, 32^2 velocities on
    [-8,8]^2, dynamic switch, ARS(2,3,3)) in FP64: two steps against the
    oracle, every cell compared."""
    wl = W.riemann_quadrants(seed=0)
    worst, g, P, st, _ = run_parity(wl, 2, "fp64", check_f=False)
    assert worst.max() <= TOL["fp64"], worst
    assert st.kin.sum() > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blob_full_size_sampled_cells(prec):
    """Precision-form configuration at its full size (256^2 periodic cells,
    48^2 velocities on [-8,8]^2, all kinetic, ARS(2,3,3)) in the per-cell form
    the bench times: one step on the GPU, and at sampled cells (centre, flank,
    far field, cells whose stencils wrap) the oracle's step on the periodic
    window of radius 7 around the cell -- one step depends on the cells within
    6 (pinned in the oracle tests)."""
    from windows import window
    wl = W.gaussian_blob()
    g = gpu_solver(wl, prec)
    g.advance(wl["dt"], wl["scheme"])
    U = g.cons()
    tab = tableau_of(wl["scheme"])
    R = 7
    for (j0, i0) in [(128, 128), (128, 155), (100, 140), (0, 0), (255, 3), (40, 220)]:
        w = window(wl, j0, i0, R)
        P, st = oracle_pair(w)
        Uo = O.advance(P, st, wl["dt"], tab).U[:, R, R]
        Ug = U[:, j0, i0]
        rel = max(abs(Ug[0] - Uo[0]) / Uo[0], abs(Ug[1] - Uo[1]) / Uo[0], abs(Ug[2] - Uo[2]) / Uo[0],
                  abs(Ug[3] - Uo[3]) / Uo[3])
        assert rel <= TOL[prec], (j0, i0, rel)


# (precision, N_v, expected form: nodes per group, cells per warp)
STRADDLE = [("fp64", 10, (2, 2)), ("fp64", 26, (2, 1)), ("fp32", 12, (4, 2)), ("fp32", 20, (4, 2)),
            ("fp32", 28, (4, 1)), ("fp32", 18, (2, 2)), ("fp32", 26, (2, 1)), ("fp32", 11, (1, 1))]


@pytest.mark.parametrize("prec,nv,form", STRADDLE)
def test_vector_groups_straddling_zero_velocity(prec, nv, form):
    """Velocity grids whose node groups straddle v_x = 0 (N_v/2 not a
    multiple of the group width): the group holding v_x = 0 takes the upwind
    stencil node by node.  Covers groups of 4 and 2 nodes, one and two cells
    per warp, and the scalar form (odd N_v)."""
    wl = W.gaussian_blob(nx=12, ny=10, nv=nv, vmax=6.0, u0=(0.4, -0.2), steps=3)
    worst, g, *_ = run_parity(wl, 3, prec)
    assert g.kinetic_form() == form
    assert worst.max() <= TOL[prec], worst


@pytest.mark.parametrize("nv,form", [(18, (2, 2)), (30, (2, 1)), (20, (4, 2))])
def test_bf16_narrow_and_straddling_groups(nv, form):
    """BF16 storage in the 2-node and straddling 4-node forms: macroscopic
    fields within the BF16 storage bound (2e-3 relative L1) of the FP64
    oracle after 3 steps."""
    wl = W.gaussian_blob(nx=12, ny=10, nv=nv, vmax=6.0, u0=(0.4, -0.2), steps=3)
    g = gpu_solver(wl, "bf16")
    assert g.kinetic_form() == form
    P, st = oracle_pair(wl)
    tab = tableau_of(wl["scheme"])
    for _ in range(3):
        g.step(wl["dt"], wl["scheme"])
        st = O.step(P, st, wl["dt"], tab)
    U = g.cons()
    r = np.abs(st.U[0]).sum()
    for q in range(4):
        scale = np.abs(st.U[3]).sum() if q == 3 else r
        assert np.abs(U[q] - st.U[q]).sum() / scale <= 2e-3, q


# ---------------------------------------------------------------------------
# edge cases

def test_all_fluid_is_euler_only():
    wl = W.riemann_quadrants(nx=16, ny=16, nv=8, seed=5)
    wl["params"] = dict(wl["params"], switch="frozen")
    worst, g, *_ = run_parity(wl, 3, "fp64")
    assert worst.max() <= TOL["fp64"], worst
    assert g.counters()["kinetic_cell_updates"] == 0


def test_one_dimensional_and_odd_velocity_grid():
    wl = W.sine_periodic(nx=1, ny=24, nv=11, steps=3, scheme="ars233")
    worst, *_ = run_parity(wl, 3, "fp64")
    assert worst.max() <= TOL["fp64"], worst


@pytest.mark.parametrize("nv", [48, 64])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_largest_velocity_grids_tiny_space(nv, prec):
    """N_v = 64 is the largest velocity grid the library accepts: 4096 nodes,
    32 KB of f* per warp in FP64."""
    wl = W.gaussian_blob(nx=5, ny=3, nv=nv, steps=2)
    worst, *_ = run_parity(wl, 2, prec)
    assert worst.max() <= TOL[prec], worst


@pytest.mark.parametrize("nx,ny,bc", [(1, 1, "periodic"), (1, 1, "outflow"), (2, 1, "outflow"), (1, 3, "periodic")])
@pytest.mark.parametrize("switch", ["frozen", "plain"])
def test_grids_of_one_to_three_cells(nx, ny, bc, switch):
    """Degenerate grids: every stencil read wraps (periodic) or copies (outflow)
    onto the few cells there are; one cell is a space-homogeneous problem."""
    wl = W.riemann_quadrants(nx=nx, ny=ny, nv=8, seed=2)
    wl["grid"] = dict(wl["grid"], bc_x=bc, bc_y=bc)
    if switch == "frozen":
        wl["fields"]["kin"] = np.ones((ny, nx), bool)
    wl["params"] = dict(wl["params"], switch=switch)
    worst, *_ = run_parity(wl, 3, "fp64")
    assert worst.max() <= TOL["fp64"], worst


def test_single_kinetic_cell_outflow_corner():
    wl = W.riemann_quadrants(nx=9, ny=7, nv=12, seed=6)
    kin = np.zeros((7, 9), bool)
    kin[0, 0] = True
    wl["fields"]["kin"] = kin
    wl["params"] = dict(wl["params"], switch="frozen")
    worst, *_ = run_parity(wl, 2, "fp64")
    assert worst.max() <= TOL["fp64"], worst


def test_work_counter_counts_transport_evaluations():
    wl = W.gaussian_blob(nx=8, ny=8, nv=8, steps=2)
    g = gpu_solver(wl)
    for _ in range(2):
        g.step(wl["dt"], "ars233")
    c = g.counters()
    assert c["kinetic_cell_updates"] == 2 * 3 * 64 and c["steps"] == 2 and c["kinetic_cells"] == 64


# ---------------------------------------------------------------------------
# errors, determinism, checkpoint/resume

def test_bad_inputs_are_rejected():
    import paper_2512_03586_gb300 as G
    wl = W.sine_periodic(nx=4, ny=4, nv=8)
    wl["fields"]["rho"][1, 1] = -1.0
    with pytest.raises(G.Error) as e:
        gpu_solver(wl)
    assert e.value.code == -1
    g = gpu_solver(W.sine_periodic(nx=4, ny=4, nv=8))
    with pytest.raises(G.Error):
        g.step(-1.0)
    with pytest.raises(G.Error):
        g.step(1e-3, dict(At=[[0.0, 1.0], [0.0, 0.0]], bt=[1, 0], A=[[0, 0], [0, 1]], b=[0, 1]))


def test_nonrealizable_state_reports_cell():
    import paper_2512_03586_gb300 as G
    wl = W.sine_periodic(nx=4, ny=4, nv=8)
    g = gpu_solver(wl)
    f = g.f()
    f[2, 3] = -f[2, 3]  # negative density in cell c = 2*4 + 3
    g.set_f(f)
    g.step(wl["dt"], "imex_euler")
    with pytest.raises(G.Error) as e:
        g.sync()
    assert e.value.code == -4 and e.value.bad_cell == 11
    # set_state clears the sticky error
    fl = wl["fields"]
    g.set_state(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["eps"], fl["kin"])
    g.step(wl["dt"], "imex_euler")
    g.sync()


def test_bitwise_deterministic():
    wl = W.riemann_quadrants(nx=20, ny=20, nv=12, seed=7)
    outs = []
    for _ in range(2):
        g = gpu_solver(wl, "fp32")
        for _ in range(3):
            g.step(wl["dt"], "ars233")
        outs.append((g.cons(), g.flags(), g.f()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    kin = outs[0][1]
    assert np.array_equal(outs[0][2][kin], outs[1][2][kin])


def test_checkpoint_resume():
    wl = W.gaussian_blob(nx=12, ny=12, nv=12, steps=4)
    a = gpu_solver(wl)
    for _ in range(2):
        a.step(wl["dt"], "ars233")
    f_mid = a.f()
    for _ in range(2):
        a.step(wl["dt"], "ars233")
    b = gpu_solver(wl)
    b.set_f(f_mid)
    for _ in range(2):
        b.step(wl["dt"], "ars233")
    assert np.allclose(a.cons(), b.cons(), rtol=1e-14, atol=1e-15)
    assert np.allclose(a.f(), b.f(), rtol=1e-14, atol=1e-16)
