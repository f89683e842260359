"""GB300 (sm_103a) library for the coupled IMEX domain-decomposition method of
the ES-BGK model (Caparello & Tenna, arXiv 2512.03586).

The compute path is libesbgk.so (hand-written CUDA behind the C ABI of
include/esbgk.h).  This package only marshals arguments: PyTorch provides the
device workspace and the stream, numpy the host arrays.  Every entry point
loads libesbgk.so on first use and raises ImportError when it has not been
built -- there is no CPU fallback.
"""

import ctypes
import importlib

import numpy as np


def _lib():
    """The ctypes binding of libesbgk.so; raises ImportError when the library
    has not been built (no fallback)."""
    return importlib.import_module(__name__ + "._abi")


class Error(RuntimeError):
    """A negative esbgk_status returned by the library."""

    NAMES = {0: "OK", -1: "E_ARG", -2: "E_WORKSPACE", -3: "E_CUDA", -4: "E_NONREALIZABLE",
             -5: "E_TIMEOUT", -6: "E_STATE", -7: "E_TOO_LARGE"}

    def __init__(self, code, msg="", bad_cell=-1):
        self.code = code
        self.bad_cell = bad_cell
        super().__init__("%s (%d): %s" % (self.NAMES.get(code, "?"), code, msg))


BC = {"periodic": 0, "outflow": 1}
SWITCH = {"frozen": 0, "plain": 1, "learned": 2}
CNN_PARAMS, CNN_CHANNELS = 10753, 16
COUPLING = {"stage": 0, "step": 1}
INTERFACE = {"own": 0, "conservative": 1}
TAU_MODEL = {"constant": 0, "density": 1}
MOMENT_SUMS = {"plain": 0, "compensated": 1}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}

__all__ = ["Solver", "BatchSolver", "SwitchNet", "make_tableau", "ARS233", "IMEX_EULER", "relax_cells", "Error"]

_ALPHA = (3.0 + 3.0 ** 0.5) / 6.0
#: ARS(2,3,3) (Sec. 3.4): explicit (At, bt), implicit (A, b), alpha = (3+sqrt 3)/6.
ARS233 = dict(
    At=[[0.0, 0.0, 0.0], [_ALPHA, 0.0, 0.0], [_ALPHA - 1.0, 2.0 - 2.0 * _ALPHA, 0.0]],
    bt=[0.0, 0.5, 0.5],
    A=[[0.0, 0.0, 0.0], [0.0, _ALPHA, 0.0], [0.0, 1.0 - 2.0 * _ALPHA, _ALPHA]],
    b=[0.0, 0.5, 0.5])
#: First-order IMEX (Filbet-Jin) in ARS(1,1,1) form: f^{n+1} = relax(f^n - dt L(f^n)).
IMEX_EULER = dict(At=[[0.0, 0.0], [1.0, 0.0]], bt=[1.0, 0.0], A=[[0.0, 0.0], [0.0, 1.0]], b=[0.0, 1.0])
#: Second-order pairs: ARS(2,2,2) (Ascher, Ruuth, Spiteri 1997; gamma = 1 - 1/sqrt 2,
#: delta = 1 - 1/(2 gamma)) and IMEX-SSP2(3,3,2) (Pareschi, Russo 2005; implicit first stage).
_GAMMA = 1.0 - 2.0 ** -0.5
_DELTA = 1.0 - 0.5 / _GAMMA
ARS222 = dict(At=[[0.0, 0.0, 0.0], [_GAMMA, 0.0, 0.0], [_DELTA, 1.0 - _DELTA, 0.0]], bt=[_DELTA, 1.0 - _DELTA, 0.0],
              A=[[0.0, 0.0, 0.0], [0.0, _GAMMA, 0.0], [0.0, 1.0 - _GAMMA, _GAMMA]], b=[0.0, 1.0 - _GAMMA, _GAMMA])
SSP2_332 = dict(At=[[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5, 0.5, 0.0]], bt=[1.0 / 3.0] * 3,
                A=[[0.25, 0.0, 0.0], [0.0, 0.25, 0.0], [1.0 / 3.0] * 3], b=[1.0 / 3.0] * 3)
TABLEAUX = {"ars233": ARS233, "imex_euler": IMEX_EULER, "ars222": ARS222, "ssp2_332": SSP2_332}


def make_tableau(t):
    """esbgk_tableau from a name ('ars233', 'imex_euler', 'ars222', 'ssp2_332') or a dict At, bt, A, b."""
    if isinstance(t, str):
        t = TABLEAUX[t]
    At, A = np.asarray(t["At"], float), np.asarray(t["A"], float)
    bt, b = np.asarray(t["bt"], float), np.asarray(t["b"], float)
    s = len(b)
    out = _lib().Tableau()
    out.s = s
    for i in range(s):
        out.bt[i] = bt[i]
        out.b[i] = b[i]
        for j in range(s):
            out.At[i * 4 + j] = At[i, j]
            out.A[i * 4 + j] = A[i, j]
    return out


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _structs(_abi, grid, vmesh, params, prec):
    g = _abi.Grid(int(grid["nx"]), int(grid["ny"]), float(grid.get("x0", 0.0)), float(grid.get("x1", 1.0)),
                  float(grid.get("y0", 0.0)), float(grid.get("y1", 1.0)), BC[grid.get("bc_x", "periodic")],
                  BC[grid.get("bc_y", "periodic")])
    v = _abi.VMesh(int(vmesh["nv"]), float(vmesh["vmax"]))
    p = params
    q = _abi.Params(float(p.get("beta", -0.5)), float(p.get("tau", 1.0)), float(p.get("eta_factor", 1.0)),
                    float(p.get("delta", 1e-3)), float(p.get("cweno_eps", 1e-6)),
                    SWITCH[p.get("switch", "frozen")], COUPLING[p.get("coupling", "stage")], PREC[prec],
                    INTERFACE[p.get("interface", "own")], TAU_MODEL[p.get("tau_model", "constant")],
                    MOMENT_SUMS[p.get("moment_sums", "plain")])
    return g, v, q


class Solver:
    """One problem on one GPU: wraps esbgk_create / esbgk_* on a torch workspace.

    grid: nx, ny, x0, x1, y0, y1, bc_x, bc_y ('periodic' | 'outflow')
    vmesh: nv, vmax
    params: beta, tau, eta_factor, delta, cweno_eps, switch ('frozen' | 'plain'),
            coupling ('stage' | 'step'), interface ('own' | 'conservative'),
            tau_model ('constant' | 'density'),
            moment_sums ('plain' | 'compensated': FP32/BF16 moment sums);
            prec: 'fp64' | 'fp32' | 'bf16'.
    """

    def __init__(self, grid, vmesh, params, prec="fp64", device=None, stream=None):
        import torch
        _abi = _lib()
        self._abi = _abi
        self.torch = torch
        self.grid, self.vmesh, self.params = _structs(_abi, grid, vmesh, params, prec)
        self.nx, self.ny, self.nv = self.grid.nx, self.grid.ny, self.vmesh.nv
        self.nc = self.nx * self.ny
        nbytes = _abi.esbgk_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.vmesh), ctypes.byref(self.params))
        if nbytes == 0:
            raise Error(-1, "invalid grid/velocity mesh/parameters")
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            r = _abi.esbgk_create(ctypes.byref(self.grid), ctypes.byref(self.vmesh), ctypes.byref(self.params),
                                  ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ctx))
        if r != 0:
            raise Error(r, "esbgk_create")
        self.workspace_bytes = nbytes

    # -- helpers ------------------------------------------------------------
    def _check(self, r, what):
        if r != 0:
            buf = ctypes.create_string_buffer(512)
            bad = ctypes.c_longlong(-1)
            self._abi.esbgk_last_error(self._ctx, buf, 512, ctypes.byref(bad))
            raise Error(r, "%s: %s" % (what, buf.value.decode(errors="replace")), bad.value)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._abi.esbgk_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ----------------------------------------------------------------
    def set_state(self, rho, ux, uy, T, eps, kin=None):
        n = self.nc
        arrs = [_f64(a, n) for a in (rho, ux, uy, T, eps)]
        k = None if kin is None else np.ascontiguousarray(np.asarray(kin).reshape(-1), dtype=np.uint8)
        r = self._abi.esbgk_set_state(self._ctx, *[_dptr(a) for a in arrs], None if k is None else _u8ptr(k))
        self._check(r, "set_state")

    def set_f(self, f):
        f = _f64(f, self.nc * self.nv * self.nv)
        self._check(self._abi.esbgk_set_f(self._ctx, _dptr(f)), "set_f")

    def f(self):
        out = np.empty((self.ny, self.nx, self.nv, self.nv))
        self._check(self._abi.esbgk_get_f(self._ctx, _dptr(out)), "get_f")
        return out

    def regime_update(self):
        self._check(self._abi.esbgk_regime_update(self._ctx), "regime_update")

    def set_flags(self, kin):
        k = np.ascontiguousarray(np.asarray(kin).reshape(-1), dtype=np.uint8)
        self._check(self._abi.esbgk_set_flags(self._ctx, _u8ptr(k)), "set_flags")

    def set_solid(self, solid):
        """Solid obstacles with specular walls: a bool mask (ny, nx), or None
        to remove them (call after set_state)."""
        if solid is None:
            self._check(self._abi.esbgk_set_solid(self._ctx, None), "set_solid")
            return
        m = np.ascontiguousarray(np.asarray(solid).reshape(-1), dtype=np.uint8)
        self._check(self._abi.esbgk_set_solid(self._ctx, _u8ptr(m)), "set_solid")

    def flags(self):
        out = np.empty((self.ny, self.nx), np.uint8)
        self._check(self._abi.esbgk_get_flags(self._ctx, _u8ptr(out)), "get_flags")
        return out.astype(bool)

    def indicators(self):
        lam = np.empty((self.ny, self.nx))
        l1 = np.empty((self.ny, self.nx))
        self._check(self._abi.esbgk_get_indicators(self._ctx, _dptr(lam), _dptr(l1)), "get_indicators")
        return lam, l1

    def advance(self, dt, tableau="ars233"):
        t = tableau if isinstance(tableau, self._abi.Tableau) else make_tableau(tableau)
        self._check(self._abi.esbgk_advance(self._ctx, float(dt), ctypes.byref(t)), "advance")

    def step(self, dt, tableau="ars233"):
        t = tableau if isinstance(tableau, self._abi.Tableau) else make_tableau(tableau)
        self._check(self._abi.esbgk_step(self._ctx, float(dt), ctypes.byref(t)), "step")

    def moments(self, out=None):
        """(rho, u_x, u_y, T) as a (4, ny, nx) float64 array (written into `out`
        when given: C-contiguous float64, e.g. pinned host memory)."""
        if out is None:
            out = np.empty((4, self.ny, self.nx))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 4 * self.nc
        o = out.reshape(4, -1)
        self._check(self._abi.esbgk_get_moments(self._ctx, *[_dptr(o[q]) for q in range(4)]), "get_moments")
        return out

    def cons(self):
        out = np.empty((4, self.ny, self.nx))
        self._check(self._abi.esbgk_get_cons(self._ctx, _dptr(out)), "get_cons")
        return out

    def totals(self):
        out = np.empty(4)
        self._check(self._abi.esbgk_totals(self._ctx, _dptr(out)), "totals")
        return out

    def counters(self):
        u, s, k, b = (ctypes.c_longlong() for _ in range(4))
        self._check(self._abi.esbgk_counters(self._ctx, ctypes.byref(u), ctypes.byref(s), ctypes.byref(k),
                                             ctypes.byref(b)), "counters")
        return dict(kinetic_cell_updates=u.value, steps=s.value, kinetic_cells=k.value, buffer_fills=b.value)

    def graphs(self, enable=True):
        """Enable or disable CUDA-graph replay of repeated steps."""
        self._check(self._abi.esbgk_graphs(self._ctx, int(bool(enable))), "graphs")

    def kinetic_form(self):
        """(nodes per vector group, kinetic cells per warp) of the specialised
        stage launches: the per-cell form chosen for this velocity grid."""
        w, p = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._abi.esbgk_kinetic_form(self._ctx, ctypes.byref(w), ctypes.byref(p)), "kinetic form")
        return w.value, p.value

    def tiles(self, enable=True):
        """Enable or disable the tiled stage kernel (every cell kinetic,
        regime frozen); off by default."""
        self._check(self._abi.esbgk_tiles(self._ctx, int(bool(enable))), "tiles")

    def tiled(self):
        """Whether the next step's stage launches take the tiled kernel."""
        t = ctypes.c_int32()
        self._check(self._abi.esbgk_tiled(self._ctx, ctypes.byref(t)), "tiled")
        return bool(t.value)

    def timing(self, enable=True):
        """Bracket every library kernel with CUDA events on the stream."""
        self._check(self._abi.esbgk_timing(self._ctx, int(bool(enable))), "timing")

    def timing_read(self):
        """{kernel class: (milliseconds, launches)} since the last read."""
        n = len(self._abi.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(self._abi.esbgk_timing_read(self._ctx, ms, cnt, n), "timing_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self._abi.KERNEL_CLASSES)}

    def sync(self):
        self._check(self._abi.esbgk_sync(self._ctx), "sync")

    # -- learned switch --------------------------------------------------------
    def set_switch_params(self, theta):
        """Network parameters (CNN_PARAMS float32) of a 'learned' switch."""
        th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(-1))
        assert th.size == CNN_PARAMS
        self._check(self._abi.esbgk_set_switch_params(self._ctx, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "set_switch_params")

    def switch_stats(self):
        j, p, m, e = (ctypes.c_longlong() for _ in range(4))
        self._check(self._abi.esbgk_switch_stats(self._ctx, ctypes.byref(j), ctypes.byref(p), ctypes.byref(m),
                                                 ctypes.byref(e)), "switch_stats")
        return dict(judged=j.value, predicted=p.value, missed=m.value, extra=e.value)

    def features(self, out=None):
        """Network features of the current state as a (ny, nx, 16) bf16
        device tensor (written into `out` when given)."""
        torch = self.torch
        if out is None:
            out = torch.empty((self.ny, self.nx, CNN_CHANNELS), dtype=torch.bfloat16, device=self.device)
        assert out.dtype == torch.bfloat16 and out.is_contiguous() and out.numel() == self.nc * CNN_CHANNELS
        self._check(self._abi.esbgk_features(self._ctx, ctypes.c_void_p(out.data_ptr())), "features")
        return out


class SwitchNet:
    """Training and evaluation of the learned-switch network (esbgk_cnn_*) on
    batches of up to max_images images of H x W cells: features (n, H, W, 16)
    bf16 and labels (n, H, W) uint8, torch device tensors."""

    def __init__(self, max_images, H, W, device=None, stream=None):
        import torch
        _abi = _lib()
        self._abi = _abi
        self.torch = torch
        self.max_images, self.H, self.W = int(max_images), int(H), int(W)
        nbytes = _abi.esbgk_cnn_workspace_bytes(self.max_images, self.H, self.W)
        if nbytes == 0:
            raise Error(-1, "invalid network batch shape")
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._c = ctypes.c_void_p()
        r = _abi.esbgk_cnn_create(self.max_images, self.H, self.W, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._c))
        if r != 0:
            raise Error(r, "esbgk_cnn_create")

    def close(self):
        if getattr(self, "_c", None) and self._c.value:
            self._abi.esbgk_cnn_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _fptr(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

    def _chk(self, r, what):
        if r != 0:
            raise Error(r, what)

    def _xy(self, x, y=None):
        torch = self.torch
        assert x.dtype == torch.bfloat16 and x.is_contiguous() and x.shape[1:] == (self.H, self.W, CNN_CHANNELS)
        n = x.shape[0]
        assert 1 <= n <= self.max_images
        if y is not None:
            assert y.dtype == torch.uint8 and y.is_contiguous() and tuple(y.shape) == (n, self.H, self.W)
        return n

    def set_params(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(-1))
        assert th.size == CNN_PARAMS
        self._chk(self._abi.esbgk_cnn_set_params(self._c, self._fptr(th)), "set_params")

    def params(self):
        out = np.empty(CNN_PARAMS, np.float32)
        self._chk(self._abi.esbgk_cnn_get_params(self._c, self._fptr(out)), "get_params")
        return out

    def forward(self, x):
        """Logits (n, H, W) float32 device tensor."""
        n = self._xy(x)
        out = self.torch.empty((n, self.H, self.W), dtype=self.torch.float32, device=self.device)
        self._chk(self._abi.esbgk_cnn_forward(self._c, ctypes.c_void_p(x.data_ptr()), n,
                                              ctypes.c_void_p(out.data_ptr())), "forward")
        return out

    def gradient(self, x, y, pos_weight):
        """(loss, gradient (CNN_PARAMS,) float32) without an update."""
        n = self._xy(x, y)
        g = np.empty(CNN_PARAMS, np.float32)
        L = ctypes.c_float()
        self._chk(self._abi.esbgk_cnn_gradient(self._c, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                               n, float(pos_weight), ctypes.byref(L), self._fptr(g)), "gradient")
        return L.value, g

    def train_step(self, x, y, pos_weight, lr, want_loss=False):
        n = self._xy(x, y)
        L = ctypes.c_float()
        self._chk(self._abi.esbgk_cnn_train_step(self._c, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                                 n, float(pos_weight), float(lr),
                                                 ctypes.byref(L) if want_loss else None), "train_step")
        return L.value if want_loss else None

    def sync(self):
        self._chk(self._abi.esbgk_cnn_sync(self._c), "sync")


class BatchSolver:
    """n independent problems advanced together (esbgk_batch_*): one launch per
    kernel per step over all cases, replayed as a CUDA graph on a non-default
    stream.  cases: list of (grid, vmesh, params) dicts as for Solver; all
    share `prec`."""

    def __init__(self, cases, prec="fp64", device=None, stream=None):
        import torch
        _abi = _lib()
        self._abi = _abi
        n = len(cases)
        if n < 1:
            raise ValueError("need at least one case")
        self.n = n
        G = (_abi.Grid * n)()
        V = (_abi.VMesh * n)()
        Pp = (_abi.Params * n)()
        self.shapes = []
        for i, (grid, vmesh, params) in enumerate(cases):
            G[i], V[i], Pp[i] = _structs(_abi, grid, vmesh, params, prec)
            self.shapes.append((G[i].nx, G[i].ny, V[i].nv))
        self._G, self._V, self._P = G, V, Pp
        nbytes = _abi.esbgk_batch_workspace_bytes(n, G, V, Pp)
        if nbytes == 0:
            raise Error(-1, "invalid batch description")
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            r = _abi.esbgk_batch_create(n, G, V, Pp, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._b))
        if r != 0:
            raise Error(r, "esbgk_batch_create")
        self.workspace_bytes = nbytes

    def _check(self, r, what):
        if r != 0:
            buf = ctypes.create_string_buffer(512)
            at = ctypes.c_int32(-1)
            self._abi.esbgk_batch_last_error(self._b, buf, 512, ctypes.byref(at))
            raise Error(r, "%s (case %d): %s" % (what, at.value, buf.value.decode(errors="replace")))

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._abi.esbgk_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dt(self, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (self.n,)))
        return d

    def set_state(self, i, rho, ux, uy, T, eps, kin=None):
        nx, ny, _ = self.shapes[i]
        arrs = [_f64(a, nx * ny) for a in (rho, ux, uy, T, eps)]
        k = None if kin is None else np.ascontiguousarray(np.asarray(kin).reshape(-1), dtype=np.uint8)
        self._check(self._abi.esbgk_batch_set_state(self._b, i, *[_dptr(a) for a in arrs],
                                                    None if k is None else _u8ptr(k)), "set_state")

    def step(self, dt, tableau="ars233", graph=True):
        """One step of every case; dt is a scalar or one value per case."""
        t = tableau if isinstance(tableau, self._abi.Tableau) else make_tableau(tableau)
        d = self._dt(dt)
        self._check(self._abi.esbgk_batch_step(self._b, _dptr(d), ctypes.byref(t), int(bool(graph))), "step")

    def autotune(self, dt, tableau="ars233"):
        """Pick the stage launch shape, then each velocity grid's per-cell
        form (advances the batch); returns (threads, ctas_per_sm).  The full
        schedule: schedule()."""
        t = tableau if isinstance(tableau, self._abi.Tableau) else make_tableau(tableau)
        d = self._dt(dt)
        th, ct = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._abi.esbgk_batch_autotune(self._b, _dptr(d), ctypes.byref(t), ctypes.byref(th),
                                                   ctypes.byref(ct)), "autotune")
        return th.value, ct.value

    FORMS = ("default", "one_cell_per_warp", "scalar")

    def schedule(self):
        """The current schedule: {'threads', 'ctas_per_sm', 'forms': {N_v: form name}}."""
        th, ct, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._abi.esbgk_batch_schedule(self._b, ctypes.byref(th), ctypes.byref(ct), None, None, 0,
                                                   ctypes.byref(n)), "schedule")
        nv = (ctypes.c_int32 * max(n.value, 1))()
        fm = (ctypes.c_int32 * max(n.value, 1))()
        self._check(self._abi.esbgk_batch_schedule(self._b, None, None, nv, fm, n.value, None), "schedule")
        return {"threads": th.value, "ctas_per_sm": ct.value,
                "forms": {int(nv[i]): self.FORMS[fm[i]] for i in range(n.value)}}

    def set_switch_params(self, i, theta):
        """Network parameters (CNN_PARAMS float32) of learned-switch case i."""
        th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(-1))
        assert th.size == CNN_PARAMS
        self._check(self._abi.esbgk_batch_set_switch_params(self._b, int(i),
                                                            th.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "set_switch_params")

    def switch_stats(self, i):
        j, p, m, e = (ctypes.c_longlong() for _ in range(4))
        self._check(self._abi.esbgk_batch_switch_stats(self._b, int(i), ctypes.byref(j), ctypes.byref(p),
                                                       ctypes.byref(m), ctypes.byref(e)), "switch_stats")
        return dict(judged=j.value, predicted=p.value, missed=m.value, extra=e.value)

    def set_form(self, nv, form):
        """Per-cell form of the cases with nv velocity nodes per direction
        ('default', 'one_cell_per_warp', 'scalar' or 0..2)."""
        f = self.FORMS.index(form) if isinstance(form, str) else int(form)
        self._check(self._abi.esbgk_batch_set_form(self._b, int(nv), f), "set_form")

    def moments(self, i, out=None):
        nx, ny, _ = self.shapes[i]
        if out is None:
            out = np.empty((4, ny, nx))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 4 * nx * ny
        o = out.reshape(4, -1)
        self._check(self._abi.esbgk_batch_get_moments(self._b, i, *[_dptr(o[q]) for q in range(4)]), "get_moments")
        return out

    def cons(self, i):
        nx, ny, _ = self.shapes[i]
        out = np.empty((4, ny, nx))
        self._check(self._abi.esbgk_batch_get_cons(self._b, i, _dptr(out)), "get_cons")
        return out

    def flags(self, i):
        nx, ny, _ = self.shapes[i]
        out = np.empty((ny, nx), np.uint8)
        self._check(self._abi.esbgk_batch_get_flags(self._b, i, _u8ptr(out)), "get_flags")
        return out.astype(bool)

    def counters(self):
        u, e, s, k = (ctypes.c_longlong() for _ in range(4))
        self._check(self._abi.esbgk_batch_counters(self._b, ctypes.byref(u), ctypes.byref(e), ctypes.byref(s),
                                                   ctypes.byref(k)), "counters")
        return dict(kinetic_cell_updates=u.value, element_updates=e.value, steps=s.value, kinetic_cells=k.value)

    def timing(self, enable=True):
        """Bracket every batched launch with CUDA events (steps then run
        without graph replay)."""
        self._check(self._abi.esbgk_batch_timing(self._b, int(bool(enable))), "timing")

    def timing_read(self):
        """{kernel class: (milliseconds, launches)} since the last read."""
        n = len(self._abi.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(self._abi.esbgk_batch_timing_read(self._b, ms, cnt, n), "timing_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self._abi.KERNEL_CLASSES)}

    def sync(self):
        self._check(self._abi.esbgk_batch_sync(self._b), "sync")


def relax_cells(fstar, h, vmax, beta=-0.5, prec="fp64", stream=None):
    """esbgk_relax_cells on torch device tensors: fstar (n, nv, nv) of the
    storage dtype of `prec`, h (n,) float64.  Returns (f, G_hat) tensors."""
    import torch
    _abi = _lib()
    n, nv, nv2 = fstar.shape
    assert nv == nv2 and fstar.is_cuda and fstar.is_contiguous()
    h = h.to(torch.float64).contiguous()
    f = torch.empty_like(fstar)
    g = torch.empty_like(fstar)
    st = stream if stream is not None else torch.cuda.current_stream(fstar.device)
    r = _abi.esbgk_relax_cells(ctypes.c_void_p(fstar.data_ptr()), ctypes.cast(h.data_ptr(), _abi.D), n, nv,
                               float(vmax), float(beta), PREC[prec], ctypes.c_void_p(f.data_ptr()),
                               ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise Error(r, "esbgk_relax_cells")
    return f, g


def wait_probe(arrive, polls=1 << 12, stream=None):
    """esbgk_wait_probe: one CTA waits on a barrier with the library's bounded
    wait; arrive=False withholds the arrival.  Returns the status code (0 =
    OK; -5 = E_TIMEOUT when the wait ran out) -- failure detection without a
    GPU fault."""
    import torch
    _abi = _lib()
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(_abi.esbgk_wait_probe(int(bool(arrive)), int(polls), ctypes.c_void_p(st.cuda_stream)))
