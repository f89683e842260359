"""The seeded input generators produce the recipes they state: ranges,
structure, time steps, determinism per seed.  No method arithmetic is
involved (the generators hold none)."""

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("seed", range(6))
def test_riemann_quadrants_recipe(seed):
    wl = W.riemann_quadrants(nx=64, ny=48, seed=seed)
    f = wl["fields"]
    rho, T, u = f["rho"], f["T"], np.hypot(f["ux"], f["uy"])
    assert rho.min() >= 0.1 and rho.max() <= 1.5
    p = rho * T
    assert p.min() >= 0.1 - 1e-12 and p.max() <= 1.5 + 1e-12
    assert T.min() >= 0.25 and T.max() <= 3.0 and u.max() <= 0.7
    # four constant quadrants split at x = 1/2, y = 1/2
    for q in (rho, T, f["ux"], f["uy"]):
        for blk in (q[:24, :32], q[:24, 32:], q[24:, :32], q[24:, 32:]):
            assert np.ptp(blk) == 0
    assert len({rho[0, 0], rho[0, -1], rho[-1, 0], rho[-1, -1]}) > 1
    # eps smooth between 1e-4 and 1e-1: log10 eps = -2.5 + 1.5 sin sin
    le = np.log10(f["eps"])
    assert le.min() >= -4 - 1e-12 and le.max() <= -1 + 1e-12 and le.max() - le.min() > 2.8
    assert not f["kin"].any() and wl["params"]["switch"] == "plain"
    assert wl["dt"] == pytest.approx(0.5 * min(1 / 64, 1 / 48) / 8.0)
    assert wl["grid"]["bc_x"] == wl["grid"]["bc_y"] == "outflow"


def test_generators_are_deterministic_per_seed():
    a, b, c = (W.riemann_quadrants(nx=16, ny=16, seed=s) for s in (3, 3, 4))
    for k in ("rho", "ux", "uy", "T", "eps"):
        assert np.array_equal(a["fields"][k], b["fields"][k])
    assert not np.array_equal(a["fields"]["rho"], c["fields"]["rho"])
    x, y = W.batched_cases(n_cases=3, seed0=7), W.batched_cases(n_cases=3, seed0=7)
    for p, q in zip(x, y):
        assert np.array_equal(p["fields"]["rho"], q["fields"]["rho"]) and p["vmesh"] == q["vmesh"]


def test_batched_recipe_sizes_and_ranges():
    cases = W.batched_cases()
    assert len(cases) == 64
    sizes = {c["grid"]["nx"] for c in cases}
    nvs = {c["vmesh"]["nv"] for c in cases}
    assert sizes <= set(range(64, 257, 16)) and len(sizes) > 6
    assert nvs <= set(range(16, 41, 2)) and len(nvs) > 6
    for c in cases:
        f = c["fields"]
        assert c["grid"]["nx"] == c["grid"]["ny"]
        assert f["rho"].min() >= 0.5 - 1e-12 and f["rho"].max() <= 1.5 + 1e-12
        assert f["T"].min() >= 0.5 - 1e-12 and f["T"].max() <= 2.0 + 1e-12
        assert np.ptp(f["eps"]) == 0 and 1e-4 <= f["eps"][0, 0] <= 1e-1
        assert not f["ux"].any() and not f["uy"].any() and f["kin"].all()
    cells = sum(c["grid"]["nx"] ** 2 for c in cases)
    elements = sum(c["grid"]["nx"] ** 2 * c["vmesh"]["nv"] ** 2 for c in cases)
    assert cells == 2060800 and elements == 1843343360


def test_blob_sine_and_learned_recipes():
    b = W.gaussian_blob(nx=64, ny=64)
    assert b["fields"]["rho"].max() == pytest.approx(1.5, abs=0.01) and b["fields"]["rho"].min() >= 1.0
    assert np.all(b["fields"]["ux"] == 0.3) and np.all(b["fields"]["T"] == 1.0)
    s = W.sine_periodic()
    assert s["fields"]["rho"].min() >= 0.8 and s["fields"]["rho"].max() <= 1.2
    assert s["dt"] == pytest.approx(0.5 / 32 / 6.0)
    base = W.riemann_quadrants(nx=64, ny=64, seed=1)
    lw = W.learned_switch_case(nx=64, ny=64, seed=1)
    ratio = lw["fields"]["rho"] / base["fields"]["rho"]
    assert ratio.min() >= 1.0 and ratio.max() == pytest.approx(1.5, abs=0.02)
    iy, ix = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert abs((ix + 0.5) / 64 - 0.3) < 0.02 and abs((iy + 0.5) / 64 - 0.7) < 0.02
    assert lw["params"]["switch"] == "learned"


def test_tests_3_and_4_recipes_match_the_paper_setup():
    """Sizes, time steps, boundary conditions and thresholds of Tests 3-4 as
    printed in Sec. 4.2.1-4.2.2, and the initial states' jumps."""
    kh, sb = W.kelvin_helmholtz(), W.shock_bubble()
    assert (kh["grid"]["nx"], kh["grid"]["ny"], sb["grid"]["nx"], sb["grid"]["ny"]) == (150, 75, 150, 50)
    assert (kh["grid"]["bc_x"], kh["grid"]["bc_y"]) == ("periodic", "outflow")
    assert kh["steps"] == 4080 and sb["steps"] == 1200
    assert abs(kh["dt"] - 0.5 / 150 / 8) < 1e-15 and abs(sb["dt"] - 0.5 / 50 / 8) < 1e-15
    assert kh["params"]["eta_factor"] == 4.0 and sb["params"]["eta_factor"] == 0.5
    f = kh["fields"]
    assert set(np.unique(f["rho"])) == {1.0, 2.0} and np.allclose(f["rho"] * f["T"], 1.0)
    assert np.abs(f["uy"]).max() <= 0.01 and kh["fields"]["kin"].all()
    g = sb["fields"]
    left = g["ux"] > 0
    assert np.allclose(g["rho"][left], 16 / 7) and np.allclose((g["rho"] * g["T"])[left], 4.75)
    assert 2.4 < g["rho"].max() < 2.5  # the bubble's peak 1 + 1.5 exp(-16 d^2) near its centre
