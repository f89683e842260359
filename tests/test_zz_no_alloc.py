"""The allocation-free entry point esbgk_kinetic_steps_noalloc.

It exists for callers that cannot allocate device memory -- a solver embedded
in a host application that owns every device allocation through its own pool
or budget, or a loop that must never enter the allocator: its intermediate
arrays live in a static device array of the library instead of a workspace.
This file is collected last so that a run stopping at the first failure has
already run every other test; it builds its own state and passes alone or
after the rest.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# the parity bars of the storage types: FP64 to rounding, FP32 1e-5, BF16 1e-3
TOL = {"fp64": 1e-10, "fp32": 1e-5, "bf16": 1e-3}


def _structs(G, wl, prec):
    abi = G._lib()
    g, v, p = wl["grid"], wl["vmesh"], wl["params"]
    grid = abi.Grid(g["nx"], g["ny"], g["x0"], g["x1"], g["y0"], g["y1"], G.BC[g["bc_x"]], G.BC[g["bc_y"]])
    vm = abi.VMesh(v["nv"], v["vmax"])
    par = abi.Params(p["beta"], p["tau"], p["eta_factor"], p["delta"], p["cweno_eps"], G.SWITCH[p["switch"]],
                     G.COUPLING[p["coupling"]], G.PREC[prec])
    return abi, grid, vm, par


def _call(abi, grid, vm, par, dt, tab, n, eps, f, U, stream):
    return abi.esbgk_kinetic_steps_noalloc(ctypes.byref(grid), ctypes.byref(vm), ctypes.byref(par), dt,
                                           ctypes.byref(tab), n, ctypes.cast(eps.data_ptr(), abi.D),
                                           ctypes.c_void_p(f.data_ptr()), ctypes.cast(U.data_ptr(), abi.D),
                                           ctypes.c_void_p(stream.cuda_stream))


def _workspace_run(G, wl, prec, scheme, f_in, n):
    """What one allocation-free call promises to equal: a fresh context
    (esbgk_create on a workspace), esbgk_set_f of the call's input f, n steps."""
    fl = wl["fields"]
    ref = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec=prec)
    ref.set_state(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["eps"], fl["kin"])
    if f_in is not None:
        ref.set_f(f_in)
    f0 = ref.f()
    for _ in range(n):
        ref.step(wl["dt"], scheme)
    out = (f0, ref.f(), ref.cons())
    ref.close()
    return out


def _two_calls_match_workspace(wl, scheme, prec, n1, n2):
    """Two allocation-free calls in a row (n1, then n2 steps) from the initial
    f; after each, f and U are compared with the workspace entry points run
    from that call's input f."""
    import torch
    import paper_2512_03586_gb300 as G

    fl = wl["fields"]
    f0, _, _ = _workspace_run(G, wl, prec, scheme, None, 0)
    abi, grid, vm, par = _structs(G, wl, prec)
    tab = G.make_tableau(scheme)
    tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[prec]
    # f0 came out of the library's storage type, so the conversion back is exact
    f = torch.tensor(f0, dtype=torch.float64).to(tdt).cuda().contiguous()
    eps = torch.tensor(fl["eps"].reshape(-1), dtype=torch.float64, device="cuda")
    # U is an output: start it with garbage so that a read before the first write shows
    U = torch.full((4, f0.shape[0] * f0.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    f_in = f0
    for call, n in enumerate((n1, n2)):
        _, f_ref, U_ref = _workspace_run(G, wl, prec, scheme, f_in, n)
        r = _call(abi, grid, vm, par, wl["dt"], tab, n, eps, f, U, stream)
        assert r == 0, abi.STATUS_NAMES.get(r, r)
        fg = f.double().cpu().numpy().reshape(f_ref.shape)
        Ug = U.cpu().numpy().reshape(U_ref.shape)
        assert np.abs(fg - f_ref).sum() / np.abs(f_ref).sum() <= TOL[prec], (prec, call)
        assert np.abs(Ug - U_ref).sum() / np.abs(U_ref).sum() <= TOL[prec], (prec, call)
        f_in = fg


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("scheme", ["imex_euler", "ars233"])
def test_noalloc_matches_workspace_entry_point_two_calls(scheme, prec):
    wl = W.sine_periodic(scheme=scheme)  # 32^2 cells, 16^2 velocities: fits the static scratch
    _two_calls_match_workspace(wl, scheme, prec, 3, 4)


def test_noalloc_size_limit_depends_on_storage():
    """48^2 cells x 24^2 velocities: five FP32 arrays (26.5 MB) fit the 32 MiB
    scratch and run at parity; in FP64 (53 MB) the same problem is refused
    before any device work."""
    import torch
    import paper_2512_03586_gb300 as G
    wl = W.gaussian_blob(nx=48, ny=48, nv=24)
    _two_calls_match_workspace(wl, "ars233", "fp32", 1, 1)
    abi, grid, vm, par = _structs(G, wl, "fp64")
    tab = G.make_tableau("ars233")
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    r = _call(abi, grid, vm, par, wl["dt"], tab, 1, dummy, dummy, dummy, torch.cuda.current_stream())
    assert r == abi.E_TOO_LARGE


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    import paper_2512_03586_gb300 as G
    wl = W.gaussian_blob(nx=128, ny=128, nv=32)  # 5 f arrays of 128 MiB in FP64: far above 32 MiB
    abi, grid, vm, par = _structs(G, wl, "fp64")
    tab = G.make_tableau("ars233")
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    p = ctypes.cast(dummy.data_ptr(), abi.D)
    r = abi.esbgk_kinetic_steps_noalloc(ctypes.byref(grid), ctypes.byref(vm), ctypes.byref(par), wl["dt"],
                                        ctypes.byref(tab), 1, p, ctypes.c_void_p(dummy.data_ptr()), p, None)
    assert r == abi.E_TOO_LARGE
