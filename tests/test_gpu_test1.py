"""Test 1 (Sec. 4.1.1, order of accuracy) at the paper's size on the GPU.

90 x 90 periodic cells on [0,6]^2, 32 x 32 velocities on [-5,5]^2, a random
regime map frozen for the run, ARS(2,3,3) to t_end = 0.86, FP64 storage.  The
temporal error of Eq. error_temporal is the discrete L2 norm of the density
difference between the runs with dt and dt/2, for dt = 0.86/64 ... 0.86/512
(the paper's 0.0135 ... 0.0017).  With per-stage coupling (HOC) the hybrid
keeps the scheme's third order, with end-of-step coupling (LOC) it drops to
first; Tables tab:order_accuracy_2/4/6 (golden file test1_orders.json) print
both.  The regime map is random, as in the paper, so the HOC errors match the
printed ones in magnitude, not digit for digit.  The LOC errors depend on
what the buffer cells hold during the stages, which the paper leaves open:
here they keep their start-of-step values (M_hat[U^n]) and the kinetic cells
show U^n to the fluid side, which gives a larger first-order constant than
the printed one; only the order and the gap to HOC are asserted for LOC.

One step of the full-size hybrid is also compared with the FP64 oracle.
"""

import json
import os
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
T_END = 0.86
KS = (64, 128, 256, 512, 1024)  # steps to t_end: dt = 0.0134 ... 0.00084


def _run(wl, k):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    for _ in range(k):
        s.step(T_END / k, "ars233")
    rho = s.cons()[0]
    upd = s.counters()["kinetic_cell_updates"]
    s.close()
    return rho, upd


def _study(eps, coupling):
    wl = W.order_test(eps=eps, coupling=coupling)
    dx = (wl["grid"]["x1"] - wl["grid"]["x0"]) / wl["grid"]["nx"]
    t0 = time.perf_counter()
    runs = [_run(wl, k) for k in KS]
    wall = time.perf_counter() - t0
    sols = [r[0] for r in runs]
    err = np.array([np.sqrt(dx * dx * np.sum((a - b) ** 2)) for a, b in zip(sols[:-1], sols[1:])])
    updates = sum(r[1] for r in runs) * wl["vmesh"]["nv"] ** 2
    return err, np.log2(err[:-1] / err[1:]), wall, updates


@pytest.mark.parametrize("eps", ["1e-2", "1e-4", "1e-6"])
def test_test1_orders_full_size(eps):
    g = json.load(open(os.path.join(GOLDEN, "test1_orders.json")))["tables"][eps]
    he, ho, hw, hu = _study(float(eps), "stage")
    le, lo, lw, lu = _study(float(eps), "step")
    print("\nTest 1, eps %s: HOC err %s orders %s; LOC err %s orders %s; %.1f s, %.3e kinetic updates/s" % (
        eps, ["%.3e" % e for e in he], ["%.2f" % o for o in ho], ["%.3e" % e for e in le],
        ["%.2f" % o for o in lo], hw + lw, (hu + lu) / (hw + lw)))
    # orders of the two finest pairs within the printed range (+- 0.35)
    for o in ho[-2:]:
        assert min(g["hoc_order"]) - 0.35 <= o <= max(g["hoc_order"]) + 0.35, ho
    for o in lo[-2:]:
        assert min(g["loc_order"]) - 0.35 <= o <= max(g["loc_order"]) + 0.35, lo
    # HOC errors at the paper's four dt within a factor 4 of the printed ones
    r = he / np.array(g["hoc_err"])
    assert np.all((r > 0.25) & (r < 4.0)), r
    print("HOC / printed %s; LOC / printed %s" % (["%.2f" % x for x in r],
                                                  ["%.0f" % x for x in le / np.array(g["loc_err"])]))
    # end-of-step coupling is far less accurate at every dt
    assert np.all(le > 100 * he), le / he


def test_test1_full_size_step_matches_oracle():
    """One ARS(2,3,3) step of the full-size hybrid (dt = 0.86/64), every cell
    compared with the FP64 oracle at 1e-10."""
    import paper_2512_03586_gb300 as G
    wl = W.order_test(eps=1e-2, coupling="stage")
    dt = T_END / KS[0]
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    s.step(dt, "ars233")
    U = s.cons()
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.step(P, O.init_state(P, **f), dt, O.ARS233)
    r = np.abs(st.U[0]).sum()
    for q in range(4):
        scale = np.abs(st.U[3]).sum() if q == 3 else r
        assert np.abs(U[q] - st.U[q]).sum() / scale <= 1e-10, q
