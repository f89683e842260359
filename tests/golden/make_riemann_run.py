"""Write the oracle's record of the coupled four-quadrant Riemann run at full size.

The run: 128x128 cells on [0,1]^2 (outflow), 32^2 velocities on [-8,8]^2, the
plain switch with eta = eps and delta = 1e-3, ARS(2,3,3) at CFL 0.5, 200 steps
from the seed-0 data of ``workloads.riemann_quadrants`` (starting all fluid).
Only ``oracle`` (FP64 numpy) computes; ``workloads`` draws the inputs.

Stored in ``riemann128_ars233_200.npz`` beside this script:
  flags        uint8 (steps, ny*nx/8)  the regime map the oracle chooses before
               each step (Algorithm 1's regime update), bit-packed row-major;
  near64       int32 (k, 2)            (step, cell) pairs whose indicator lies
               within 1e-6 (relative) of its threshold (lambda_A vs eta, or the
               L1 deviation vs delta in a cell that was kinetic): a library in
               FP64 may decide these differently;
  near32       int32 (k, 2)            the same within 1e-3, for FP32 storage
               (the criterion is evaluated in float32 there);
  U_<n>        float64 (4, ny, nx)     conserved fields after n steps, at
               n in CHECKPOINTS;
  kin_count    int32 (steps,)          kinetic cells per step.

Usage: python tests/golden/make_riemann_run.py [steps]   (~25 s per step on one core)
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "riemann128_ars233_200.npz")
CHECKPOINTS = (100, 200)


def main(steps=200):
    wl = W.riemann_quadrants(seed=0, steps=steps)
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **wl["fields"])
    flags, near64, near32, kin_count = [], [], [], []
    snaps = {}
    t0 = time.time()
    for n in range(steps):
        lam, l1 = O.regime_indicators(P, st)
        eta = P.eta_factor * st.eps
        new = (lam > eta) | (st.kin & (l1 > P.delta))
        flags.append(np.packbits(new.ravel()))
        d_lam = np.abs(lam - eta)
        d_l1 = np.abs(l1 - P.delta)
        for rel, out in ((1e-6, near64), (1e-3, near32)):
            near = (d_lam <= rel * eta) | (st.kin & (d_l1 <= rel * P.delta))
            out.extend((n, int(c)) for c in np.flatnonzero(near.ravel()))
        st = O.convert(P, st, new)
        kin_count.append(int(new.sum()))
        st = O.advance(P, st, wl["dt"], O.ARS233)
        if n + 1 in CHECKPOINTS:
            snaps["U_%d" % (n + 1)] = st.U.copy()
        print("step %d kinetic %d  %.0f s" % (n + 1, kin_count[-1], time.time() - t0), flush=True)
    np.savez_compressed(
        OUT, flags=np.array(flags, np.uint8),
        near64=np.array(near64, np.int32).reshape(-1, 2),
        near32=np.array(near32, np.int32).reshape(-1, 2),
        kin_count=np.array(kin_count, np.int32), **snaps)
    print("wrote", OUT)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 200)
