"""Failure detection on the GPU without a fault: a bounded device wait that
runs out is reported as a status, and the context stays usable.

esbgk_wait_probe runs the library's bounded barrier wait in one CTA; with the
arrival withheld (a barrier nothing completes) the wait gives up after its
poll limit, the kernel records the timeout in a device error word and exits,
and the call returns ESBGK_E_TIMEOUT.  A solver step and a completed probe
afterwards show the context is intact.
"""

import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

E_TIMEOUT = -5


def test_bounded_wait_times_out_and_context_survives():
    import paper_2512_03586_gb300 as G
    assert G.wait_probe(True) == 0
    t0 = time.perf_counter()
    assert G.wait_probe(False) == E_TIMEOUT
    dt = time.perf_counter() - t0
    print("\nbounded wait of 4096 polls ran out in %.3f s" % dt)
    assert dt < 5.0
    # the context still works: a step of a small problem, then a completed probe
    wl = W.sine_periodic(nx=8, ny=8, nv=8, steps=1)
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec="fp64")
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    m0 = s.totals()[0]
    s.step(wl["dt"], wl["scheme"])
    assert np.isfinite(s.cons()).all() and abs(s.totals()[0] - m0) <= 1e-12 * m0
    s.close()
    assert G.wait_probe(True) == 0


def test_wait_probe_rejects_bad_limits():
    import paper_2512_03586_gb300 as G
    assert G.wait_probe(True, polls=0) == -1
    assert G.wait_probe(True, polls=(1 << 20) + 1) == -1
