"""Write the oracle's records of Tests 5 and 6 (Sec. 4.2.3-4.2.4) at the paper's size.

The runs: flow rho = 1, u = (2, 0), p = 1 on [0,1]^2 (78 x 78 cells, outflow
edges) toward a solid cylinder of radius 1/12 (Test 5) or a rectangle of
10 x 4 cells (Test 6) centred at (2/5, 1/2), specular walls (reading R24),
32^2 velocities on [-8,8]^2, eps = 1e-6, eta = 10 eps, delta = 1e-3, the plain
switch, ARS(2,3,3) with dt = 0.5 dx / 8 to t_end = 0.15 (188 steps), starting
all fluid (``workloads.obstacle_flow``).  Only ``oracle`` (FP64 numpy)
computes; ``workloads`` draws the inputs.

Stored in ``obstacle78_<kind>_188.npz`` beside this script:
  flags        uint8 (steps, ny*nx/8)  the regime map the oracle chooses before
               each step, bit-packed row-major (solid cells are never kinetic);
  near64       int32 (k, 2)            (step, cell) pairs whose indicator lies
               within 1e-6 (relative) of its threshold (lambda_A vs eta, or the
               L1 deviation vs delta in a cell that was kinetic);
  near32       int32 (k, 2)            the same within 1e-3 (FP32 storage);
  U_<n>        float64 (4, ny, nx)     conserved fields after n steps, at n in
               CHECKPOINTS (solid cells hold their initial state);
  kin_count    int32 (steps,)          kinetic cells per step.

Usage: python tests/golden/make_obstacle_runs.py [cylinder|rectangle] [steps]
(~10 s per step on one core).
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

CHECKPOINTS = (94, 188)


def out_path(kind):
    return os.path.join(HERE, "obstacle78_%s_188.npz" % kind)


def main(kind, steps=188):
    wl = W.obstacle_flow(kind)
    solid = wl["solid"]
    fluid = ~solid
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"], solid=solid)
    st = O.init_state(P, **wl["fields"])
    flags, near64, near32, kin_count = [], [], [], []
    snaps = {}
    t0 = time.time()
    for n in range(steps):
        lam, l1 = O.regime_indicators(P, st)
        eta = P.eta_factor * st.eps
        new = ((lam > eta) | (st.kin & (l1 > P.delta))) & fluid
        flags.append(np.packbits(new.ravel()))
        d_lam = np.abs(lam - eta)
        d_l1 = np.abs(l1 - P.delta)
        for rel, out in ((1e-6, near64), (1e-3, near32)):
            near = ((d_lam <= rel * eta) | (st.kin & (d_l1 <= rel * P.delta))) & fluid
            out.extend((n, int(c)) for c in np.flatnonzero(near.ravel()))
        st = O.convert(P, st, new)
        kin_count.append(int(new.sum()))
        st = O.advance(P, st, wl["dt"], O.ARS233)
        if not np.isfinite(st.U[:, fluid]).all():
            raise FloatingPointError("non-finite state after step %d" % (n + 1))
        if n + 1 in CHECKPOINTS:
            snaps["U_%d" % (n + 1)] = st.U.copy()
        rho = st.U[0][fluid]
        print("step %d kinetic %d min rho %.4f  %.0f s" % (n + 1, kin_count[-1], rho.min(), time.time() - t0),
              flush=True)
    np.savez_compressed(
        out_path(kind), flags=np.array(flags, np.uint8),
        near64=np.array(near64, np.int32).reshape(-1, 2),
        near32=np.array(near32, np.int32).reshape(-1, 2),
        kin_count=np.array(kin_count, np.int32), **snaps)
    print("wrote", out_path(kind))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "cylinder", int(sys.argv[2]) if len(sys.argv) > 2 else 188)
