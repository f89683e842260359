"""The allocation-free entry point esbgk_kinetic_steps_noalloc.

It exists for callers that may not allocate device memory (inside stream
capture, under a caller-owned memory pool or budget): its intermediate arrays
live in a static device array of the library instead of a workspace.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it builds its own state and passes alone or after the rest.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _structs(G, wl, prec):
    abi = G._lib()
    g, v, p = wl["grid"], wl["vmesh"], wl["params"]
    grid = abi.Grid(g["nx"], g["ny"], g["x0"], g["x1"], g["y0"], g["y1"], G.BC[g["bc_x"]], G.BC[g["bc_y"]])
    vm = abi.VMesh(v["nv"], v["vmax"])
    par = abi.Params(p["beta"], p["tau"], p["eta_factor"], p["delta"], p["cweno_eps"], G.SWITCH[p["switch"]],
                     G.COUPLING[p["coupling"]], G.PREC[prec])
    return abi, grid, vm, par


@pytest.mark.parametrize("scheme", ["imex_euler", "ars233"])
def test_noalloc_matches_workspace_entry_point_two_calls(scheme):
    import torch
    import paper_2512_03586_gb300 as G

    prec = "fp64"
    wl = W.sine_periodic(scheme=scheme)  # 32^2 cells, 16^2 velocities: fits the static scratch
    fl = wl["fields"]
    n1, n2 = 3, 4

    # reference: the workspace-based entry points, 7 steps
    ref = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec=prec)
    ref.set_state(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["eps"], fl["kin"])
    f0 = ref.f()
    checkpoints = {}
    for k in range(1, n1 + n2 + 1):
        ref.step(wl["dt"], scheme)
        if k in (n1, n1 + n2):
            checkpoints[k] = (ref.f(), ref.cons())

    # allocation-free path: same initial f, two calls in a row (3 + 4 steps)
    abi, grid, vm, par = _structs(G, wl, prec)
    tab = G.make_tableau(scheme)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda").contiguous()
    eps = torch.tensor(fl["eps"].reshape(-1), dtype=torch.float64, device="cuda")
    # U is an output: start it with garbage so that a read before the first write shows
    U = torch.full((4, f0.shape[0] * f0.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    done = 0
    for n in (n1, n2):
        r = abi.esbgk_kinetic_steps_noalloc(ctypes.byref(grid), ctypes.byref(vm), ctypes.byref(par), wl["dt"],
                                            ctypes.byref(tab), n, ctypes.cast(eps.data_ptr(), abi.D),
                                            ctypes.c_void_p(f.data_ptr()), ctypes.cast(U.data_ptr(), abi.D),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert r == 0, abi.STATUS_NAMES.get(r, r)
        done += n
        f_ref, U_ref = checkpoints[done]
        fg = f.cpu().numpy().reshape(f_ref.shape)
        Ug = U.cpu().numpy().reshape(U_ref.shape)
        assert np.abs(fg - f_ref).sum() / np.abs(f_ref).sum() <= 1e-10
        assert np.abs(Ug - U_ref).sum() / np.abs(U_ref).sum() <= 1e-10


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
