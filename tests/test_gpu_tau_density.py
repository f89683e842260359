"""Relaxation time proportional to the density (Reading R23,
tau_model = 'density'): nu = tau rho / eps with the density of the cell's f*
at each stage, and the criterion's viscosity and conductivity with tau rho.
Parity with the FP64 oracle run with the same reading: a frozen hybrid map
and the coupled Riemann data with the plain switch (flags and indicators
compared by the harness), FP64 1e-10 and FP32 1e-5.
"""

import pytest

import workloads as W
from test_gpu_parity import TOL, run_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_density_tau_hybrid_matches_oracle(prec):
    wl = W.order_test(n=17, nv=12, eps=1e-2, seed=2)
    wl["params"] = dict(wl["params"], tau_model="density", tau=0.8)
    wl["dt"] = 0.2 / 8
    worst, *_ = run_parity(wl, 3, prec)
    assert worst.max() <= TOL[prec], worst


def test_density_tau_plain_switch_matches_oracle():
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3)
    wl["params"] = dict(wl["params"], tau_model="density")
    worst, g, P, st, ex = run_parity(wl, 5, "fp64")
    assert worst.max() <= TOL["fp64"], worst
    assert 0 < st.kin.sum() < st.kin.size
