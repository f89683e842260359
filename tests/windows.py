"""Periodic windows of a workload (test helper, no method arithmetic): the
(2R+1) x (2R+1) cells around cell (j0, i0), wrapped at the periodic edges, on a
grid with the same cell size."""

import numpy as np


def window(wl, j0, i0, R):
    g = wl["grid"]
    assert g["bc_x"] == g["bc_y"] == "periodic"
    nx, ny = g["nx"], g["ny"]
    jj = np.arange(j0 - R, j0 + R + 1) % ny
    ii = np.arange(i0 - R, i0 + R + 1) % nx
    dx, dy = (g["x1"] - g["x0"]) / nx, (g["y1"] - g["y0"]) / ny
    out = dict(wl)
    out["grid"] = dict(g, nx=2 * R + 1, ny=2 * R + 1, x0=0.0, x1=(2 * R + 1) * dx, y0=0.0, y1=(2 * R + 1) * dy)
    out["fields"] = {k: v[np.ix_(jj, ii)] for k, v in wl["fields"].items()}
    return out
