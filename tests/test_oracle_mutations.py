"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle (in a temporary directory, on the CPU), runs the pin
that should catch it against the copy, and requires that pin to fail; the
unmutated copy must pass the same pins.  The repository's oracle is never
modified."""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file under oracle/, text, replacement, pin file, -k expression, the mistake)
MUTATIONS = [
    ("kinetic.py", "+ beta * Theta", "- beta * Theta", "test_oracle_collision.py", "stability_function",
     "ES tensor with the wrong sign of beta"),
    ("kinetic.py", "f = (fstar + h[..., None, None] * Gh) / (1.0 + h)[..., None, None]",
     "f = (fstar + h[..., None, None] * Gh) / (1.0 + 0.9 * h)[..., None, None]", "test_oracle_collision.py",
     "implicit_stage_residual", "implicit relaxation not solving its equation"),
    ("transport.py", "un * (E + P)]), np.abs", "un * E]), np.abs", "test_oracle_transport.py", "sod",
     "energy flux without the pressure work"),
    ("transport.py", "np.clip(idx, 0, m - 1)", "(idx % m)", "test_oracle_transport.py", "sod",
     "outflow ghost cells wrapped periodically"),
    ("scheme.py", "g -= dt * tab.bt[i] * Ls[i][kin]", "g -= dt * tab.b[i] * Ls[i][kin]", "test_oracle_scheme.py",
     "explicit_rk", "final transport weighted by the implicit weights"),
    ("scheme.py", "(2.0 / 3.0) * div[..., None, None]", "(1.0) * div[..., None, None]", "test_oracle_scheme.py",
     "compression", "criterion without the 2/3 trace part of D(u)"),
    ("scheme.py", "L1[st.kin] = w * np.sum", "L1[st.kin] = np.sum", "test_oracle_scheme.py", "l1_deviation",
     "L1 deviation without the quadrature weight"),
    ("scheme.py", "f_i[buf] = _mhat_of_U(prob, U_i[:, buf])", "f_i[buf] = _mhat_of_U(prob, U_n[:, buf])",
     "test_oracle_scheme.py", "second_order_pairs_converge", "buffer cells not coupled at every stage"),
    ("cnn.py", "mh = m / (1 - b1 ** t)", "mh = m", "test_oracle_cnn.py", "adam", "Adam without bias correction"),
    ("scheme.py", "f[up] = _mhat_of_U(prob, U[:, up])", "f[up] = 1.001 * _mhat_of_U(prob, U[:, up])",
     "test_oracle_scheme.py", "conversions", "fluid-to-kinetic conversion off in normalisation"),
    ("transport.py", "psi = np.stack([np.ones_like(VX), VX, VY, 0.5 * (VX * VX + VY * VY)])",
     "psi = np.stack([np.ones_like(VX), VX, VY, 0.5 * (VX * VX)])", "test_oracle_scheme.py",
     "conservative_interface", "interface energy flux missing the v_y^2 part"),
    ("transport.py", "a = np.maximum(am, ap)", "a = 0.5 * np.maximum(am, ap)", "test_oracle_transport.py",
     "dissipation", "Euler flux with half the Lax-Friedrichs speed"),
    ("transport.py", "np.abs(un) + np.sqrt(GAMMA * np.maximum(P, 0.0) / rho)",
     "np.sqrt(GAMMA * np.maximum(P, 0.0) / rho)", "test_oracle_transport.py",
     "dissipation", "Euler flux speed without the flow speed |u_n|"),
    ("transport.py", "np.sqrt(GAMMA * np.maximum(P, 0.0) / rho)", "np.sqrt(GAMMA * np.abs(P) / rho)",
     "test_oracle_transport.py", "without_pressure", "sound speed of a face state with negative pressure from |P|"),
    ("walls.py", "return g[..., ::-1] if axis == 0 else g[..., ::-1, :]", "return g", "test_oracle_walls.py",
     "symmetry", "wall mirror images of f without the specular reflection"),
    ("walls.py", "pm = 2 * a + sg - p", "pm = 2 * a - p", "test_oracle_walls.py", "symmetry",
     "wall mirror image one cell off"),
    ("walls.py", "out[..., 1 + axis] *= -1.0", "out[..., 1 + axis] *= 1.0", "test_oracle_walls.py", "symmetry",
     "Euler mirror state keeping the normal momentum"),
]


@pytest.fixture(scope="module")
def sandbox(tmp_path_factory):
    """A copy of the oracle, the generators and the pin tests."""
    base = tmp_path_factory.mktemp("mut")
    for d in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(base, d),
                        ignore=shutil.ignore_patterns("__pycache__"))
    tests = os.path.join(base, "tests")
    os.makedirs(tests)
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f.endswith(".py") and (f.startswith("test_oracle_") and f != "test_oracle_mutations.py"
                                  or not f.startswith("test_")):
            shutil.copy(os.path.join(ROOT, "tests", f), tests)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tests, "golden"))
    return str(base)


def _run_pin(base, pin, kexpr):
    env = dict(os.environ, PYTHONPATH=base, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pin), "-q", "-x", "-k", kexpr,
                        "-p", "no:cacheprovider"], cwd=base, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-1500:]


def test_unmutated_copy_passes_the_pins(sandbox):
    for pin, kexpr in sorted({(m[3], m[4]) for m in MUTATIONS}):
        rc, out = _run_pin(sandbox, pin, kexpr)
        assert rc == 0, (pin, kexpr, out)


@pytest.mark.parametrize("fname,old,new,pin,kexpr,what", MUTATIONS, ids=[m[5] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(sandbox, fname, old, new, pin, kexpr, what):
    path = os.path.join(sandbox, "oracle", fname)
    src = open(path).read()
    assert src.count(old) == 1, "mutation site not unique: " + old
    try:
        open(path, "w").write(src.replace(old, new))
        rc, out = _run_pin(sandbox, pin, kexpr)
    finally:
        open(path, "w").write(src)
    assert rc == 1, "%s: pin %s -k %s did not fail\n%s" % (what, pin, kexpr, out)
