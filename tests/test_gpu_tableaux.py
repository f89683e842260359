"""Other IMEX pairs on the GPU (Sec. 3.4 admits any IMEX-RK pair): ARS(2,2,2)
(first stage explicit) and IMEX-SSP2(3,3,2) (implicit first stage).  Their
launches do not match the compiled ARS(2,3,3) / IMEX-Euler stage shapes, so
they run the generic stage kernel, which reads every tableau flag at run
time.  Checked: parity with the FP64 oracle (FP64 1e-10, FP32 1e-5) on a
hybrid with a frozen random map and on the coupled Riemann data with the
plain switch, and second-order convergence on the GPU.
"""

import numpy as np
import pytest

import workloads as W
from test_gpu_parity import TOL, run_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", ["ars222", "ssp2_332"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pair_matches_oracle_hybrid(scheme, prec):
    wl = W.order_test(n=17, nv=12, eps=1e-2, seed=2)
    wl["scheme"] = scheme
    wl["dt"] = 0.2 / 8
    worst, *_ = run_parity(wl, 3, prec)
    assert worst.max() <= TOL[prec], worst


@pytest.mark.parametrize("scheme", ["ars222", "ssp2_332"])
def test_pair_matches_oracle_plain_switch(scheme):
    wl = W.riemann_quadrants(nx=20, ny=16, nv=16, seed=3)
    wl["scheme"] = scheme
    worst, *_ = run_parity(wl, 4, "fp64")
    assert worst.max() <= TOL["fp64"], worst


@pytest.mark.parametrize("scheme", ["ars222", "ssp2_332"])
def test_pair_is_second_order_on_gpu(scheme):
    import paper_2512_03586_gb300 as G
    wl = W.order_test(n=48, nv=16, eps=1e-2)
    f = wl["fields"]
    sols = []
    for k in (8, 16, 32, 64):
        s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec="fp64")
        s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
        for _ in range(k):
            s.step(0.4 / k, scheme)
        sols.append(s.cons()[0].copy())
        s.close()
    err = [np.sqrt(np.sum((a - b) ** 2)) for a, b in zip(sols[:-1], sols[1:])]
    orders = np.log2(np.array(err[:-1]) / np.array(err[1:]))
    print("\n%s orders %s" % (scheme, orders))
    assert abs(orders[-1] - 2.0) <= 0.3, orders


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_first_relaxed_stage_without_transport_coefficient(prec):
    """ARS(2,3,3) with the explicit coefficient of its second stage set to
    zero (At[1][0] = 0): f* of the first relaxed stage is f^n itself, so the
    specialised first-stage kernel (which rebuilds its partial accumulators
    from f* - f^n and the ratio of the coefficients) cannot serve it and the
    generic stage kernel takes the stage.  The result matches the FP64 oracle
    with the same tableau."""
    import oracle as O
    from test_gpu_parity import field_errors, gpu_solver, oracle_pair
    At = O.ARS233.At.copy()
    At[1, 0] = 0.0
    tab_o = O.Tableau(At=At, bt=O.ARS233.bt, A=O.ARS233.A, b=O.ARS233.b)
    tab_g = {"At": At, "bt": O.ARS233.bt, "A": O.ARS233.A, "b": O.ARS233.b}
    wl = W.order_test(n=17, nv=12, eps=1e-2, seed=2)
    wl["dt"] = 0.2 / 8
    g = gpu_solver(wl, prec)
    P, st = oracle_pair(wl)
    worst = np.zeros(4)
    for _ in range(3):
        g.advance(wl["dt"], tab_g)
        st = O.advance(P, st, wl["dt"], tab_o)
        worst = np.maximum(worst, field_errors(g.cons(), st.U))
    assert np.all(np.isfinite(g.cons())), "non-finite state"
    assert worst.max() <= TOL[prec], worst
