"""Acceptance bars of the switch network's gradients (test helper).

The GPU stores the activations a1, a2 and the back-propagated dz2, dz1 in
bf16 (8 significant bits: a relative rounding of at most 2^-9) and accumulates
in float32.  What the bf16 storage alone does to a gradient on given inputs is
computed by the FP64 oracle with the same roundings applied where the GPU
stores (g_emu); the exact float64 network gives g_exact.  A GPU gradient
g_gpu then differs from g_emu by float32 accumulation only (a few 1e-4 of a
block's largest entry, and a rare one-ulp flip of a bf16 value on a rounding
boundary), so by the triangle inequality, per block and per element,

    |g_gpu - g_exact| <= |g_emu - g_exact| + ACC * max|g_exact|,

and per block ||g_gpu - g_exact|| <= ||g_emu - g_exact|| + ACC ||g_exact||.
ACC = 2e-3 covers the accumulation part with a margin.
"""

import numpy as np

ACC = 2e-3
BLOCKS = ("W1", "b1", "W2", "b2", "w3", "b3")


def check(g_test, g_exact, g_emu, unpack):
    """Blocks of g_test outside the bars: {name: (block error, bound,
    worst element excess)}; empty when every block passes."""
    t, e, m = unpack(g_test), unpack(g_exact), unpack(g_emu)
    bad = {}
    for name in BLOCKS:
        ne = np.linalg.norm(e[name])
        err = np.linalg.norm(t[name] - e[name]) / ne
        bound = np.linalg.norm(m[name] - e[name]) / ne + ACC
        scale = np.max(np.abs(e[name]))
        excess = np.max(np.abs(t[name] - e[name]) - (np.abs(m[name] - e[name]) + ACC * scale)) / scale
        if err > bound or excess > 0:
            bad[name] = (err, bound, excess)
    return bad
