"""Conservative kinetic/fluid interface (Reading R22) on the GPU.

A buffer cell's Euler update takes, at each face shared with a kinetic cell,
the moments (1, v, |v|^2/2) of the kinetic numerical flux there, the same
face values the kinetic cell's transport uses.  Checked: parity with the FP64
oracle run with the same reading (per-stage and end-of-step coupling), exact
conservation of the totals on a periodic hybrid in FP64 (each model's own
flux drifts), and the Sod tube of Test 2 with the conservative interface.
"""

import numpy as np
import pytest

import workloads as W
from test_gpu_parity import TOL, run_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("coupling", ["stage", "step"])
def test_conservative_interface_matches_oracle(coupling):
    wl = W.order_test(n=17, nv=12, eps=1e-2, coupling=coupling, seed=2)
    wl["params"] = dict(wl["params"], interface="conservative")
    wl["dt"] = 0.2 / 8
    worst, *_ = run_parity(wl, 3, "fp64")
    assert worst.max() <= TOL["fp64"], worst


def _drift(wl, iface, steps, prec):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], interface=iface), prec=prec)
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    t0 = s.totals()
    for _ in range(steps):
        s.step(wl["dt"], "ars233")
    d = np.abs(s.totals() - t0) / np.abs(t0).max()
    s.close()
    return d


def test_conservative_interface_conserves_hybrid_totals():
    """Periodic 48^2 hybrid, random frozen map (half the cells kinetic),
    flowing data, 20 ARS(2,3,3) steps in FP64: mass, momentum and energy to
    rounding with the conservative interface, a drift many orders larger
    with each model's own flux."""
    wl = W.order_test(n=48, nv=16, eps=1e-2, seed=4)
    X, Y = np.meshgrid((np.arange(48) + 0.5) / 8, (np.arange(48) + 0.5) / 8)
    wl["fields"]["ux"] = 0.3 * np.sin(2 * np.pi * Y / 6)
    wl["fields"]["uy"] = 0.2 * np.cos(2 * np.pi * X / 6)
    wl["dt"] = 0.5 * (6.0 / 48) / 5.0
    own = _drift(wl, "own", 20, "fp64")
    cons = _drift(wl, "conservative", 20, "fp64")
    print("\nhybrid totals drift (rho, m_x, m_y, E): own %s, conservative %s" % (own, cons))
    assert cons.max() <= 1e-13, cons
    assert own.max() >= 1e4 * max(cons.max(), 1e-16), (own, cons)


def test_sod_with_conservative_interface():
    """Test 2 with the conservative interface: the hybrid conserves mass to
    rounding and stays as close to the exact solution as with each model's
    own flux."""
    import paper_2512_03586_gb300 as G
    from riemann_exact import exact_riemann_density
    wl = W.sod_tube()
    ny, nx = wl["grid"]["ny"], wl["grid"]["nx"]
    out = {}
    for iface in ("own", "conservative"):
        s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], interface=iface), prec="fp64")
        f = wl["fields"]
        s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
        m0 = s.totals()[0]
        for _ in range(wl["steps"]):
            s.step(wl["dt"], "ars233")
        rho = s.cons()[0].reshape(ny, nx)[:, 0]
        out[iface] = (rho, abs(s.totals()[0] - m0) / m0)
        s.close()
    y = (np.arange(ny) + 0.5) / ny
    ex = exact_riemann_density(1.0, 0.0, 1.0, 0.125, 0.0, 1.0 / 32, 2.0, (y - 0.5) / 0.15)
    e = {k: np.mean(np.abs(v[0] - ex)) for k, v in out.items()}
    print("\nSod: mean |rho - exact| own %.3e conservative %.3e; mass drift own %.2e conservative %.2e"
          % (e["own"], e["conservative"], out["own"][1], out["conservative"][1]))
    assert out["conservative"][1] <= 1e-13
    assert e["conservative"] <= 1.2 * e["own"] + 1e-4
