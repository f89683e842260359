"""CUDA-graph replay of repeated steps (esbgk_step on a non-default stream)
gives bit-identical results to plain launches: the graph holds the same
launches with the same arguments."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,prec", [("ars233", "fp32"), ("imex_euler", "fp64"), ("ars233", "fp64")])
def test_graph_replay_is_bitwise_identical(scheme, prec):
    import torch
    import paper_2512_03586_gb300 as G
    wl = W.riemann_quadrants(nx=24, ny=20, nv=16, seed=5, scheme=scheme)
    f = wl["fields"]
    out = []
    for graphs in (True, False):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec=prec, stream=stream)
            s.graphs(graphs)
            s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
            for _ in range(8):
                s.step(wl["dt"], scheme)
            s.sync()
            out.append((s.cons(), s.flags(), s.f(), s.counters()))
    (U1, k1, f1, c1), (U2, k2, f2, c2) = out
    np.testing.assert_array_equal(U1, U2)
    np.testing.assert_array_equal(k1, k2)
    np.testing.assert_array_equal(f1[k1], f2[k2])
    assert c1 == c2
