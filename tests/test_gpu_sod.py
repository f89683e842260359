"""Test 2 (Sec. 4.1.2, Sod shock tube) at the paper's size on the GPU.

21 x 150 cells on [0, 0.1] x [0, 1] (Sod data along y), 32 x 32 velocities on
[-8, 8]^2, eps = 1e-6, ARS(2,3,3), dt = 0.8 min(dx, dy) / 8 to t_end = 0.15,
FP64 storage.  Three runs, as in the paper's comparison: the hybrid (plain
switch, all cells macroscopic at t = 0), the full Euler solver (every cell
fluid, regime frozen) and the full kinetic ES-BGK solver (every cell kinetic,
frozen).  All three approach the exact solution of the Euler Riemann problem
(gamma = 2), the hybrid follows the Euler run, and the kinetic regime is
engaged only near the waves.  The hybrid's interfaces use each model's own
flux, so mass is conserved only up to the interface mismatch; the drift is
printed and bounded loosely.
"""

import numpy as np
import pytest

import workloads as W
from riemann_exact import exact_riemann_density

pytestmark = pytest.mark.gpu


def _run(wl, switch, kin):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], switch=switch), prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], kin)
    m0 = s.totals()[0]
    kin_max = 0
    for _ in range(wl["steps"]):
        s.step(wl["dt"], "ars233")
        if switch == "plain":
            kin_max = max(kin_max, int(s.flags().sum()))
    rho = s.cons()[0].reshape(wl["grid"]["ny"], wl["grid"]["nx"])
    drift = abs(s.totals()[0] - m0) / m0
    s.close()
    return rho, drift, kin_max


def test_sod_hybrid_euler_kinetic_against_exact_solution():
    wl = W.sod_tube()
    ny, nx = wl["grid"]["ny"], wl["grid"]["nx"]
    none, every = np.zeros((ny, nx), bool), np.ones((ny, nx), bool)
    r_hyb, d_hyb, kmax = _run(wl, "plain", none)
    r_eul, d_eul, _ = _run(wl, "frozen", none)
    r_kin, d_kin, _ = _run(wl, "frozen", every)
    y = (np.arange(ny) + 0.5) / ny
    ex = exact_riemann_density(1.0, 0.0, 1.0, 0.125, 0.0, 1.0 / 32, 2.0, (y - 0.5) / 0.15)
    # the data are uniform along x and stay so
    for r in (r_hyb, r_eul, r_kin):
        assert np.max(np.abs(r - r[:, :1])) <= 1e-12
    e_hyb, e_eul, e_kin = (np.mean(np.abs(r[:, 0] - ex)) for r in (r_hyb, r_eul, r_kin))
    gap = np.mean(np.abs(r_hyb[:, 0] - r_eul[:, 0]))
    print("\nSod, t = 0.15: mean |rho - exact| hybrid %.3e, Euler %.3e, kinetic %.3e; hybrid vs Euler %.3e; "
          "most kinetic cells %d of %d; mass drift hybrid %.2e, Euler %.2e, kinetic %.2e"
          % (e_hyb, e_eul, e_kin, gap, kmax, ny * nx, d_hyb, d_eul, d_kin))
    # 150 cells across a shock, a contact and a rarefaction: first-order-in-space
    # error near the discontinuities dominates
    assert max(e_hyb, e_eul, e_kin) < 0.02
    # at eps = 1e-6 the kinetic model is the Euler limit: all three runs agree
    assert gap < 5e-3 and np.mean(np.abs(r_kin[:, 0] - r_eul[:, 0])) < 5e-3
    # the criterion engages kinetic cells near the waves only
    assert 0 < kmax < 0.3 * ny * nx
    # waves stay inside the tube: the single-model runs conserve mass
    assert d_eul < 1e-12 and d_kin < 1e-12 and d_hyb < 1e-3
