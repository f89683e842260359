"""Write the oracle's record of the full-size precision-form run.

The run: 256x256 periodic cells on [0,1]^2, 48^2 velocities on [-8,8]^2, a
Gaussian density blob (amplitude 0.5, width 0.1) on the uniform flow
u = (0.3, 0), T = 1, eps = 1e-3, every cell kinetic, ARS(2,3,3) at CFL 0.5,
100 steps (``workloads.gaussian_blob``).  Only ``oracle`` (FP64 numpy)
computes; ``workloads`` draws the inputs.

The oracle advances the whole grid; this script only spreads that work over
processes.  One ARS(2,3,3) step of a cell depends on the cells within 6 of it
along each axis (pinned in tests/test_oracle_scheme.py), so each process
advances the periodic window of its slab of rows plus 6 rows on each side
(``oracle.advance`` on that window, a periodic grid of the same cell size)
and keeps the slab's rows; the slabs together are the global step.

Stored in ``blob256_ars233_100.npz`` beside this script:
  U_<n>    float64 (4, ny, nx)  conserved fields after n steps, n in CHECKPOINTS;
  mass     float64 (steps+1,)   total mass after each step.

Usage: python tests/golden/make_blob_run.py [steps] [processes]
(about an hour and a half on 8 cores, 30 GB of memory)
"""

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "blob256_ars233_100.npz")
CHECKPOINTS = (1, 100)
HALO = 6  # rows a step depends on, each side


def _slab_step(args):
    """Advance rows [j0, j1) of the global state by one step: the oracle on
    the periodic window of rows j0-HALO .. j1+HALO-1."""
    j0, j1, f_win, U_win, eps_win, kin_win, grid, vmesh, params, dt = args
    import oracle as O
    P = O.Problem(**grid, **vmesh, **params)
    st = O.State(f=f_win, U=U_win, kin=kin_win, eps=eps_win)
    out = O.advance(P, st, dt, O.ARS233)
    return j0, out.f[HALO:HALO + (j1 - j0)], out.U[:, HALO:HALO + (j1 - j0)]


def main(steps=100, procs=8):
    import oracle as O
    import workloads as W
    wl = W.gaussian_blob()
    g = wl["grid"]
    ny, nx = g["ny"], g["nx"]
    P = O.Problem(**g, **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **wl["fields"])
    rows = ny // procs
    assert rows * procs == ny and rows >= HALO
    dy = (g["y1"] - g["y0"]) / ny
    wgrid = dict(g, ny=rows + 2 * HALO, y0=0.0, y1=(rows + 2 * HALO) * dy)
    mass = [O.totals(P, st)[0]]
    snaps = {}
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for n in range(steps):
            jobs = []
            for p in range(procs):
                j0, j1 = p * rows, (p + 1) * rows
                jj = np.arange(j0 - HALO, j1 + HALO) % ny
                jobs.append((j0, j1, st.f[jj], st.U[:, jj], st.eps[jj], st.kin[jj], wgrid, wl["vmesh"],
                             wl["params"], wl["dt"]))
            f_new = np.empty_like(st.f)
            U_new = np.empty_like(st.U)
            for j0, f_s, U_s in pool.imap_unordered(_slab_step, jobs):
                f_new[j0:j0 + rows] = f_s
                U_new[:, j0:j0 + rows] = U_s
            st = O.State(f=f_new, U=U_new, kin=st.kin, eps=st.eps)
            mass.append(O.totals(P, st)[0])
            if n + 1 in CHECKPOINTS:
                snaps["U_%d" % (n + 1)] = st.U.copy()
            print("step %d  %.0f s" % (n + 1, time.time() - t0), flush=True)
    np.savez_compressed(OUT, mass=np.array(mass), **snaps)
    print("wrote", OUT)


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:3]))
