"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/esbgk.h declares; host-only entry points behave (no GPU needed)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "esbgk.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esbgk_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2512_03586_gb300 import build as B
    return B.build()


def test_library_exports_every_declared_symbol(libpath):
    names = declared_functions()
    assert "esbgk_step" in names and "esbgk_relax_cells" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (esbgk_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert getattr(lib, n) is not None


def test_python_binding_declares_every_symbol(libpath):
    from paper_2512_03586_gb300 import _abi
    assert sorted(_abi.DECLARED) == declared_functions()


def test_host_only_entry_points(libpath):
    from paper_2512_03586_gb300 import _abi
    assert _abi.esbgk_version() >= 100
    g = _abi.Grid(128, 128, 0.0, 1.0, 0.0, 1.0, 1, 1)
    v = _abi.VMesh(32, 8.0)
    p = _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, _abi.FP32)
    nb = _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p))
    # six f arrays of nc * nv^2 floats plus O(nc) per-cell arrays
    f_bytes = 128 * 128 * 32 * 32 * 4
    assert 6 * f_bytes <= nb <= 6 * f_bytes + 400 * 128 * 128 + (1 << 20)
    p64 = _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, _abi.FP64)
    assert _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p64)) > nb
    for bad in (_abi.Grid(0, 4, 0, 1, 0, 1, 0, 0), _abi.Grid(4, 4, 1, 0, 0, 1, 0, 0), _abi.Grid(4, 4, 0, 1, 0, 1, 7, 0)):
        assert _abi.esbgk_workspace_bytes(ctypes.byref(bad), ctypes.byref(v), ctypes.byref(p)) == 0
    for badp in (_abi.Params(-0.6, 1.0, 1.0, 1e-3, 1e-6, 1, 0, 1), _abi.Params(-0.5, 0.0, 1.0, 1e-3, 1e-6, 1, 0, 1),
                 _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, 9)):
        assert _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(v), ctypes.byref(badp)) == 0
    assert _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(_abi.VMesh(65, 8.0)), ctypes.byref(p)) == 0
    # two nodes per direction cannot carry the quadratic projection; three can
    assert _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(_abi.VMesh(2, 8.0)), ctypes.byref(p)) == 0
    assert _abi.esbgk_workspace_bytes(ctypes.byref(g), ctypes.byref(_abi.VMesh(3, 8.0)), ctypes.byref(p)) > 0
    # NULL arguments are rejected before any device call
    out = ctypes.c_void_p()
    assert _abi.esbgk_create(None, None, None, None, 0, None, ctypes.byref(out)) == _abi.E_ARG
    assert _abi.esbgk_step(None, 1e-3, None) == _abi.E_ARG
    assert _abi.esbgk_relax_cells(None, None, 1, 8, 1.0, -0.5, 0, None, None, None) == _abi.E_ARG
    _abi.esbgk_destroy(None)
    # the batch's schedule, form and learned-switch entry points on a null batch
    i32 = ctypes.c_int32()
    assert _abi.esbgk_batch_schedule(None, None, None, None, None, 0, ctypes.byref(i32)) == _abi.E_ARG
    assert _abi.esbgk_batch_set_form(None, 16, 0) == _abi.E_ARG
    assert _abi.esbgk_batch_set_switch_params(None, 0, None) == _abi.E_ARG
    assert _abi.esbgk_batch_switch_stats(None, 0, None, None, None, None) == _abi.E_ARG
    assert _abi.esbgk_tiles(None, 1) == _abi.E_ARG


def test_oracle_and_library_share_no_code():
    """The CPU oracle and the CUDA path are independent: neither imports the other."""
    pkg = os.path.join(ROOT, "paper_2512_03586_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, re.M), f
                assert "oracle/" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2512_03586_gb300" not in txt, f


@pytest.mark.parametrize("name", ["ars233", "imex_euler", "ars222", "ssp2_332"])
def test_packed_tableau_carries_the_oracle_coefficients(libpath, name):
    """The binding's tableaux and the oracle's are written separately; the
    esbgk_tableau the binding packs (rows of stride 4) holds the oracle's
    coefficients."""
    import numpy as np
    import oracle as O
    import paper_2512_03586_gb300 as G
    ref = {"ars233": O.ARS233, "imex_euler": O.IMEX_EULER, "ars222": O.ARS222, "ssp2_332": O.SSP2_332}[name]
    t = G.make_tableau(name)
    s = len(ref.b)
    assert t.s == s
    At = np.array([[t.At[i * 4 + j] for j in range(s)] for i in range(s)])
    A = np.array([[t.A[i * 4 + j] for j in range(s)] for i in range(s)])
    np.testing.assert_allclose(At, ref.At, rtol=0, atol=1e-15)
    np.testing.assert_allclose(A, ref.A, rtol=0, atol=1e-15)
    np.testing.assert_allclose(list(t.bt)[:s], ref.bt, rtol=0, atol=1e-15)
    np.testing.assert_allclose(list(t.b)[:s], ref.b, rtol=0, atol=1e-15)


def test_relax_cells_argument_checks_and_empty_input(libpath):
    """esbgk_relax_cells checks its arguments and returns for n = 0 before any
    device call (the host buffers below are never dereferenced)."""
    import numpy as np
    from paper_2512_03586_gb300 import _abi
    buf = np.zeros(16)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    d = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    call = _abi.esbgk_relax_cells
    assert call(p, d, 0, 16, 6.0, -0.5, _abi.FP64, p, p, None) == 0
    assert call(p, d, -1, 16, 6.0, -0.5, _abi.FP64, p, p, None) == _abi.E_ARG
    assert call(p, d, 0, 2, 6.0, -0.5, _abi.FP64, p, p, None) == _abi.E_ARG      # N_v = 2: singular projection
    assert call(p, d, 0, 65, 6.0, -0.5, _abi.FP64, p, p, None) == _abi.E_ARG
    assert call(p, d, 0, 16, 0.0, -0.5, _abi.FP64, p, p, None) == _abi.E_ARG
    assert call(p, d, 0, 16, 6.0, -0.6, _abi.FP64, p, p, None) == _abi.E_ARG     # beta below -1/2
    assert call(p, d, 0, 16, 6.0, -0.5, 9, p, p, None) == _abi.E_ARG             # unknown precision
    assert call(None, d, 0, 16, 6.0, -0.5, _abi.FP64, p, p, None) == _abi.E_ARG


def test_batch_workspace_bytes_host_checks(libpath):
    """The batched workspace holds every case's own workspace plus descriptor
    tables (a learned-switch case's includes its network buffers); one
    precision per batch, every case valid."""
    from paper_2512_03586_gb300 import _abi
    G2 = _abi.Grid * 2
    V2 = _abi.VMesh * 2
    P2 = _abi.Params * 2
    g = G2(_abi.Grid(64, 64, 0, 1, 0, 1, 0, 0), _abi.Grid(96, 80, 0, 1, 0, 1, 1, 1))
    v = V2(_abi.VMesh(16, 8.0), _abi.VMesh(24, 8.0))
    p = P2(_abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, _abi.FP32), _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, _abi.FP32))
    total = _abi.esbgk_batch_workspace_bytes(2, g, v, p)
    singles = sum(_abi.esbgk_workspace_bytes(ctypes.byref(g[i]), ctypes.byref(v[i]), ctypes.byref(p[i])) for i in range(2))
    assert singles <= total <= singles + (1 << 22)
    assert _abi.esbgk_batch_workspace_bytes(0, g, v, p) == 0
    mixed = P2(p[0], _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 1, 0, _abi.FP64))
    assert _abi.esbgk_batch_workspace_bytes(2, g, v, mixed) == 0                  # one precision per batch
    learned = P2(p[0], _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 2, 0, _abi.FP32))
    assert _abi.esbgk_batch_workspace_bytes(2, g, v, learned) > total             # network buffers of case 1
    assert _abi.esbgk_batch_workspace_bytes(2, g, V2(v[0], _abi.VMesh(2, 8.0)), p) == 0


def test_noalloc_entry_host_checks(libpath):
    """esbgk_kinetic_steps_noalloc rejects bad arguments (E_ARG) and problems
    larger than its static scratch (E_TOO_LARGE) before any device call."""
    import numpy as np
    import paper_2512_03586_gb300 as G
    from paper_2512_03586_gb300 import _abi
    g = _abi.Grid(8, 8, 0, 1, 0, 1, 0, 0)
    v = _abi.VMesh(8, 6.0)
    p = _abi.Params(-0.5, 1.0, 1.0, 1e-3, 1e-6, 0, 0, _abi.FP32)
    tab = G.make_tableau("ars233")
    buf = np.zeros(16)
    d = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    vp = buf.ctypes.data_as(ctypes.c_void_p)
    call = _abi.esbgk_kinetic_steps_noalloc
    R = ctypes.byref
    assert call(R(g), R(v), R(p), 0.0, R(tab), 1, d, vp, d, None) == _abi.E_ARG          # dt <= 0
    assert call(R(g), R(v), R(p), float("inf"), R(tab), 1, d, vp, d, None) == _abi.E_ARG
    assert call(R(g), R(v), R(p), 1e-3, R(tab), -1, d, vp, d, None) == _abi.E_ARG        # nsteps < 0
    assert call(R(g), R(v), R(p), 1e-3, None, 1, d, vp, d, None) == _abi.E_ARG
    assert call(R(g), R(v), R(p), 1e-3, R(tab), 1, None, vp, d, None) == _abi.E_ARG
    assert call(R(g), R(_abi.VMesh(2, 6.0)), R(p), 1e-3, R(tab), 1, d, vp, d, None) == _abi.E_ARG
    bad = G.make_tableau("ars233")
    bad.s = 5                                                                             # more stages than fit
    assert call(R(g), R(v), R(p), 1e-3, R(bad), 1, d, vp, d, None) == _abi.E_ARG
    upper = G.make_tableau("ars233")
    upper.At[0 * 4 + 1] = 0.3                                                             # explicit part not strictly lower
    assert call(R(g), R(v), R(p), 1e-3, R(upper), 1, d, vp, d, None) == _abi.E_ARG
    neg = G.make_tableau("ars233")
    neg.A[1 * 4 + 1] = -0.1                                                               # negative implicit diagonal
    assert call(R(g), R(v), R(p), 1e-3, R(neg), 1, d, vp, d, None) == _abi.E_ARG
    huge = _abi.Grid(2048, 2048, 0, 1, 0, 1, 0, 0)
    assert call(R(huge), R(_abi.VMesh(32, 8.0)), R(p), 1e-3, R(tab), 1, d, vp, d, None) == _abi.E_TOO_LARGE
