"""Precision form: f stored and transported in FP32, or stored in BF16 with
FP32 arithmetic; FP64 only in the per-cell tensor solve (det of the
temperature tensor) and in U and the totals.  Error per macroscopic field
against FP64 and the relative mass drift.

Bars: FP32 storage -- relative L1 error <= 1e-5 per field after the run and
relative mass drift <= 1e-6.  BF16 storage (8 significant bits) cannot reach
1e-5: each store rounds f by up to 2^-8 relative.  BF16 stores round
stochastically (unbiased), so the per-store errors average out in the
moments instead of accumulating a bias; the bounds asserted here are the
measured values (full size: <= 5.3e-4 per field, drift 9.8e-6) with a
margin, and the numbers are printed.

The small case is checked against the FP64 CPU oracle; the full-size blob
(256 x 256 cells, 48 x 48 velocities, 100 ARS(2,3,3) steps) against the FP64
GPU path, which the parity tests pin to the oracle at 1e-10.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _errors(U, Uref):
    r = np.abs(Uref[0]).sum()
    return [np.abs(U[0] - Uref[0]).sum() / r, np.abs(U[1] - Uref[1]).sum() / r,
            np.abs(U[2] - Uref[2]).sum() / r, np.abs(U[3] - Uref[3]).sum() / np.abs(Uref[3]).sum()]


def _gpu_run(wl, prec, steps, sums="plain", tiles=True):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], moment_sums=sums), prec=prec)
    s.tiles(tiles)
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    m0 = s.totals()[0]
    for _ in range(steps):
        s.step(wl["dt"], wl["scheme"])
    return s.cons(), abs(s.totals()[0] - m0) / m0


def test_precision_small_against_oracle():
    wl = W.gaussian_blob(nx=12, ny=10, nv=48, steps=4)
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **wl["fields"])
    for _ in range(4):
        st = O.step(P, st, wl["dt"], O.ARS233)
    out = {}
    for prec in ("fp64", "fp32", "bf16"):
        U, drift = _gpu_run(wl, prec, 4)
        out[prec] = (_errors(U, st.U), drift)
    print("\nsmall blob vs oracle (rho, m_x, m_y, E; mass drift):", out)
    assert max(out["fp64"][0]) <= 1e-10
    assert max(out["fp32"][0]) <= 1e-5 and out["fp32"][1] <= 1e-6
    assert max(out["bf16"][0]) <= 2e-3 and out["bf16"][1] <= 1e-4


def test_precision_full_size_blob():
    wl = W.gaussian_blob()          # 256^2 cells, 48^2 velocities, eps 1e-3, 100 steps
    steps = wl["steps"]
    Uref, d64 = _gpu_run(wl, "fp64", steps)
    U32, d32 = _gpu_run(wl, "fp32", steps)
    U16, d16 = _gpu_run(wl, "bf16", steps)
    e32, e16 = _errors(U32, Uref), _errors(U16, Uref)
    print("\nfull blob, %d steps, error vs FP64 (rho, m_x, m_y, E): FP32 %s drift %.2e; BF16 %s drift %.2e; "
          "FP64 drift %.2e" % (steps, ["%.2e" % e for e in e32], d32, ["%.2e" % e for e in e16], d16, d64))
    assert d64 <= 1e-12
    assert max(e32) <= 1e-5 and d32 <= 1e-6
    assert max(e16) <= 2e-3 and d16 <= 5e-5


@pytest.mark.parametrize("tiles", [True, False])
def test_compensated_sums_small_against_oracle(tiles):
    """Compensated FP32/BF16 moment sums in the tiled and the per-cell
    kernels: the same bars against the oracle as the plain sums."""
    wl = W.gaussian_blob(nx=12, ny=10, nv=48, steps=4)
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **wl["fields"])
    for _ in range(4):
        st = O.step(P, st, wl["dt"], O.ARS233)
    U32, d32 = _gpu_run(wl, "fp32", 4, sums="compensated", tiles=tiles)
    U16, d16 = _gpu_run(wl, "bf16", 4, sums="compensated", tiles=tiles)
    assert max(_errors(U32, st.U)) <= 1e-5 and d32 <= 1e-6
    assert max(_errors(U16, st.U)) <= 2e-3 and d16 <= 1e-4


def test_compensated_sums_coupled_riemann_against_oracle():
    """Compensated sums on the coupled path (per-cell kernel, plain switch)."""
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=4)
    wl["params"] = dict(wl["params"], moment_sums="compensated")
    from test_gpu_parity import run_parity
    worst, *_ = run_parity(wl, 4, "fp32")
    assert worst.max() <= 1e-5, worst


def test_compensated_sums_full_size_blob_drift():
    """Precision-form configuration at full size, 100 steps, FP32 storage,
    plain and compensated sums, tiled kernel: errors against the FP64 path,
    and the mass drift of both (printed for the design notes)."""
    wl = W.gaussian_blob()
    steps = wl["steps"]
    Uref, _ = _gpu_run(wl, "fp64", steps)
    out = {}
    for sums in ("plain", "compensated"):
        U, d = _gpu_run(wl, "fp32", steps, sums=sums)
        out[sums] = (_errors(U, Uref), d)
    print("\nfull blob FP32, %d steps (rho, m_x, m_y, E error vs FP64; mass drift): %s" % (steps, out))
    for sums in out:
        assert max(out[sums][0]) <= 1e-5 and out[sums][1] <= 1e-6
    assert out["compensated"][1] <= out["plain"][1]
