"""Batched form: many independent problems advanced by one launch per kernel.

Every case of a batch must reproduce the same problem advanced alone: the
batched kernels run the single-problem per-cell code, but they are separate
kernels, so the compiler may contract a few products into FMAs differently
and the results agree to rounding, not bit for bit.  Per field, the relative
L1 difference must stay within TOL_BATCH and the regime maps must be
identical, for mixed grid sizes, velocity grids (vector and scalar node
groups), switches and tableaux, with and without CUDA-graph replay.  One small
batch is also checked directly against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

# batch vs single problem: rounding differences only (FP64: a few ulp,
# FP32 / BF16 storage: the storage rounding of f can flip)
TOL_BATCH = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 1e-3}


def _mixed_cases():
    """Uneven sizes, N_v even/odd (every per-cell form: groups of 4 or 2
    nodes, one or two cells per warp, scalar), plain and frozen switches,
    all-kinetic, hybrid and initially all-fluid maps.  Every
    velocity grid resolves the thermal speed of its data (dv <= sqrt(T)
    in most cells), so that rounding differences are not amplified by an
    ill-conditioned moment system."""
    out = []
    out.append(W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3))               # plain, starts fluid
    out += W.batched_cases(n_cases=2, seed0=11, sizes=[16, 24], nvs=[12, 16])  # plain, all kinetic
    for k, nv in enumerate((18, 26, 20)):   # 2-node groups (two / one cell per warp), straddling 4-node groups
        out += W.batched_cases(n_cases=1, seed0=30 + k, sizes=[12, 20], nvs=[nv])
    out.append(W.sine_periodic(nx=10, ny=14, nv=15, scheme="ars233"))        # frozen, odd N_v
    hyb = W.gaussian_blob(nx=18, ny=12, nv=8, vmax=4.0)
    rng = np.random.default_rng(5)
    hyb["fields"]["kin"] = rng.random((12, 18)) < 0.4                          # frozen hybrid map
    out.append(hyb)
    return out


def _single(wl, prec):
    import paper_2512_03586_gb300 as G
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec=prec)
    f = wl["fields"]
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    return s


def _batch(cases, prec, stream=None):
    import paper_2512_03586_gb300 as G
    b = G.BatchSolver([(c["grid"], c["vmesh"], c["params"]) for c in cases], prec=prec, stream=stream)
    for i, c in enumerate(cases):
        f = c["fields"]
        b.set_state(i, f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    return b


def _compare(b, singles, prec):
    for i, s in enumerate(singles):
        Ub, Us = b.cons(i), s.cons()
        r = np.abs(Us[0]).sum()
        for q in range(4):
            scale = np.abs(Us[3]).sum() if q == 3 else r
            err = np.abs(Ub[q] - Us[q]).sum() / scale
            assert err <= TOL_BATCH[prec], "case %d field %d: %.3e" % (i, q, err)
        np.testing.assert_array_equal(b.flags(i), s.flags(), err_msg="case %d flags" % i)


@pytest.mark.parametrize("prec,tableau,graph", [("fp64", "ars233", True), ("fp32", "ars233", True),
                                                ("fp32", "imex_euler", True), ("fp64", "ars233", False),
                                                ("bf16", "ars233", True)])
def test_batch_equals_single_cases(prec, tableau, graph):
    import torch
    cases = _mixed_cases()
    for c in cases:
        c["scheme"] = tableau
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, prec, stream=stream)
        singles = [_single(c, prec) for c in cases]
        dts = np.array([c["dt"] for c in cases])
        for _ in range(5):
            for s, c in zip(singles, cases):
                s.step(c["dt"], tableau)
            b.step(dts, tableau, graph=graph)
        b.sync()
        _compare(b, singles, prec)
        cb = b.counters()
        cs = [s.counters() for s in singles]
        assert cb["kinetic_cell_updates"] == sum(c["kinetic_cell_updates"] for c in cs)
        assert cb["kinetic_cells"] == sum(c["kinetic_cells"] for c in cs)
        assert cb["steps"] == 5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_mixed_moment_sums_equal_single_cases(prec):
    """Cases with compensated and plain moment sums in one batch: the batched
    launches take the kernels whose sums follow each case's parameter, and
    every case matches the same problem advanced alone (compensated cases by
    the single-problem kernels with run-time sums, plain ones by the kernels
    with the compensation compiled out)."""
    import torch
    cases = _mixed_cases()
    for k, c in enumerate(cases):
        c["params"] = dict(c["params"], moment_sums="compensated" if k % 2 == 0 else "plain")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, prec, stream=stream)
        singles = [_single(c, prec) for c in cases]
        dts = np.array([c["dt"] for c in cases])
        for _ in range(5):
            for s, c in zip(singles, cases):
                s.step(c["dt"], "ars233")
            b.step(dts, "ars233", graph=True)
        b.sync()
        _compare(b, singles, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_with_largest_velocity_grid(prec):
    """A case at the largest accepted N_v = 64 (4096 nodes: the widest shared
    f* arrays of the batched kernels) beside a small two-cells-per-warp case."""
    import torch
    big = W.gaussian_blob(nx=5, ny=3, nv=64, steps=2)
    small = W.riemann_quadrants(nx=12, ny=10, nv=12, seed=4)
    cases = [big, small]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, prec, stream=stream)
        singles = [_single(c, prec) for c in cases]
        dts = np.array([c["dt"] for c in cases])
        for _ in range(3):
            for s, c in zip(singles, cases):
                s.step(c["dt"], "ars233")
            b.step(dts, "ars233")
        b.sync()
        _compare(b, singles, prec)


def test_batch_on_default_stream_runs_without_graph():
    cases = _mixed_cases()[:3]
    b = _batch(cases, "fp64")
    singles = [_single(c, "fp64") for c in cases]
    dts = np.array([c["dt"] for c in cases])
    for _ in range(3):
        b.step(dts, "ars233", graph=True)  # legacy stream: plain launches
        for s, c in zip(singles, cases):
            s.step(c["dt"], "ars233")
    _compare(b, singles, "fp64")


def test_batch_autotune_keeps_results():
    import torch
    cases = W.batched_cases(n_cases=6, seed0=20, sizes=[16, 32, 48], nvs=[16, 20, 24])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, "fp32", stream=stream)
        dts = np.array([c["dt"] for c in cases])
        threads, ctas = b.autotune(dts)
        assert threads in (32, 64, 128) and ctas in (0, 2, 4, 8)
        sch = b.schedule()
        assert (sch["threads"], sch["ctas_per_sm"]) == (threads, ctas)
        assert sorted(sch["forms"]) == [16, 20, 24]
        assert set(sch["forms"].values()) <= set(b.FORMS)
        n_tuned = b.counters()["steps"]
        assert n_tuned > 0
        b.step(dts)
        singles = [_single(c, "fp32") for c in cases]
        for s, c in zip(singles, cases):
            for _ in range(n_tuned + 1):
                s.step(c["dt"], "ars233")
        # whatever forms were chosen, the results are the single runs'
        _compare(b, singles, "fp32")
        # a later batch of the same velocity grids starts from the chosen schedule
        b2 = _batch(cases, "fp32", stream=stream)
        assert b2.schedule() == sch


@pytest.mark.parametrize("form", ["default", "one_cell_per_warp", "scalar"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_every_per_cell_form_keeps_results(form, prec):
    """Each per-cell form the autotuner may choose gives the single-problem
    results (N_v = 12: two cells per warp by default; N_v = 26 and 18: the
    straddling forms)."""
    import torch
    cases = W.batched_cases(n_cases=3, seed0=40, sizes=[16, 24], nvs=[12, 18, 26])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, prec, stream=stream)
        for nv in sorted({c["vmesh"]["nv"] for c in cases}):
            b.set_form(nv, form)
        assert set(b.schedule()["forms"].values()) == {form}
        dts = np.array([c["dt"] for c in cases])
        for _ in range(3):
            b.step(dts)
        singles = [_single(c, prec) for c in cases]
        for s, c in zip(singles, cases):
            for _ in range(3):
                s.step(c["dt"], "ars233")
        _compare(b, singles, prec)


def test_batch_matches_oracle_small():
    import torch
    w1 = W.riemann_quadrants(nx=16, ny=12, nv=12, seed=1)
    w1["params"] = dict(w1["params"], switch="frozen")
    w1["fields"]["kin"] = np.random.default_rng(2).random((12, 16)) < 0.5
    w2 = W.gaussian_blob(nx=10, ny=8, nv=16, steps=2)
    cases = [w1, w2]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, "fp64", stream=stream)
        dts = np.array([c["dt"] for c in cases])
        for _ in range(2):
            b.step(dts)
        b.sync()
    for i, wl in enumerate(cases):
        P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
        st = O.init_state(P, **wl["fields"])
        for _ in range(2):
            st = O.step(P, st, wl["dt"], O.ARS233)
        U = b.cons(i)
        r = np.abs(st.U[0]).sum()
        for q in range(4):
            scale = np.abs(st.U[3]).sum() if q == 3 else r
            assert np.abs(U[q] - st.U[q]).sum() / scale <= 1e-10, (i, q)


def test_batch_rejects_bad_input():
    import paper_2512_03586_gb300 as G
    w = W.sine_periodic(nx=4, ny=4, nv=8)
    with pytest.raises(ValueError):
        G.BatchSolver([])
    b = G.BatchSolver([(w["grid"], w["vmesh"], w["params"])], prec="fp64")
    with pytest.raises(G.Error):  # no state yet
        b.step(w["dt"])
    out = np.empty(4 * 16)
    assert b._abi.esbgk_batch_get_cons(b._b, 5, out.ctypes.data_as(b._abi.D)) == b._abi.E_ARG
    assert b._abi.esbgk_batch_get_cons(b._b, -1, out.ctypes.data_as(b._abi.D)) == b._abi.E_ARG


def test_batch_learned_switch_equals_single_contexts():
    """Learned-switch cases in a batch (with a plain-switch case beside them):
    the criterion runs batched, each network in its own launches of the same
    step; flags, judge statistics and fields equal the single contexts' runs
    with the same network (FP64 storage: fields to 1e-12)."""
    import torch
    from paper_2512_03586_gb300 import switch_train as T
    theta = T.init_params(5)
    theta[-1] = -0.5  # head bias: part of the cells predicted kinetic
    cases = [W.riemann_quadrants(nx=24, ny=20, nv=16, seed=3), W.riemann_quadrants(nx=32, ny=16, nv=12, seed=4),
             W.riemann_quadrants(nx=20, ny=20, nv=16, seed=5)]
    for c in cases[:2]:
        c["params"] = dict(c["params"], switch="learned")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch(cases, "fp64", stream=stream)
        for i in range(2):
            b.set_switch_params(i, theta)
        singles = [_single(c, "fp64") for c in cases]
        for s in singles[:2]:
            s.set_switch_params(theta)
        dts = np.array([c["dt"] for c in cases])
        for _ in range(5):
            b.step(dts)
            for s, c in zip(singles, cases):
                s.step(c["dt"], "ars233")
            for i, s in enumerate(singles):
                np.testing.assert_array_equal(b.flags(i), s.flags())
        _compare(b, singles, "fp64")
        for i in range(2):
            assert b.switch_stats(i) == singles[i].switch_stats()
        assert b.switch_stats(0)["predicted"] > 0


def test_batch_learned_case_without_parameters_is_refused():
    import torch
    import paper_2512_03586_gb300 as G
    c = W.riemann_quadrants(nx=8, ny=8, nv=8, seed=1)
    c["params"] = dict(c["params"], switch="learned")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = _batch([c], "fp64", stream=stream)
        with pytest.raises(G.Error):
            b.step(np.array([c["dt"]]))
