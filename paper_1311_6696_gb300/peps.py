"""ctypes binding of the C ABI declared in include/peps.h (argument marshalling only).

Every computation runs in ``libpeps.so``; this module converts arguments,
checks status codes and raises :class:`PepsError` with the library's message.
If the library is missing, importing this module raises -- there is no
Python fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpeps.so")

OK, EINVAL, ENOMEM, ECUDA, ECONVERGE, ETIMEOUT = range(6)
F64, F32 = 0, 1
SVD, VAR = 0, 1
PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "tf32x3": 3, "bf16x3": 4}
KIND = {"site": 0, "hbond": 1, "vbond": 2}
MODE = {"svd": SVD, "var": VAR}

EXPORTS = [
    "peps_env_full", "peps_env_cluster", "peps_expect_local", "peps_env_rho", "peps_norm",
    "peps_env_ln_norm", "peps_env_free", "peps_last_error", "peps_profile_enable",
    "peps_profile_reset", "peps_profile_count", "peps_profile_name", "peps_profile_read",
    "peps_cu0_noalloc", "peps_closure_data", "peps_mlp_param_count", "peps_mlp_init",
    "peps_mlp_loss_grad", "peps_mlp_train", "peps_mlp_predict", "peps_plan_create", "peps_plan_run",
    "peps_plan_env", "peps_plan_launches", "peps_plan_free", "peps_plan_tune",
    "peps_set_iteration_caps", "peps_wait_selftest", "peps_boundary_fidelity", "peps_env_cluster_range",
    "peps_ipeps_cluster", "peps_bond_update", "peps_bond_update_cluster", "peps_mlp_train_state",
    "peps_mlp_save", "peps_mlp_load", "peps_env_save", "peps_env_load",
]
CLOSURE_WIDTH = 256


class PepsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"peps error {code}: {msg}")
        self.code = code


class Lattice(C.Structure):
    _fields_ = [("Ly", C.c_int), ("Lx", C.c_int), ("d", C.c_int), ("D", C.c_int),
                ("dtype", C.c_int), ("A", C.c_void_p), ("on_device", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("chi", C.c_int), ("mode", C.c_int), ("sweeps", C.c_int), ("precision", C.c_int),
                ("n", C.c_int), ("closure", C.c_int), ("closure_weights", C.c_void_p),
                ("seed", C.c_ulonglong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.peps_env_full.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.POINTER(P), P]
    lib.peps_env_cluster.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.POINTER(P), P]
    lib.peps_expect_local.argtypes = [P, C.POINTER(Lattice), C.c_int, P, P, P]
    lib.peps_env_rho.argtypes = [P, C.c_int, P, P]
    lib.peps_norm.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.POINTER(C.c_double),
                              C.POINTER(C.c_int), P]
    lib.peps_env_ln_norm.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int), P]
    lib.peps_env_free.argtypes = [P]
    lib.peps_env_free.restype = None
    lib.peps_last_error.restype = C.c_char_p
    lib.peps_profile_enable.argtypes = [C.c_int]
    lib.peps_profile_enable.restype = None
    lib.peps_profile_reset.restype = None
    lib.peps_profile_name.restype = C.c_char_p
    lib.peps_profile_read.argtypes = [C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.peps_cu0_noalloc.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
    lib.peps_closure_data.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), P, P, C.c_longlong,
                                      C.POINTER(C.c_longlong), P]
    lib.peps_mlp_param_count.argtypes = [C.c_int, C.c_int, C.c_int]
    lib.peps_mlp_param_count.restype = C.c_longlong
    lib.peps_mlp_init.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_ulonglong, P]
    lib.peps_mlp_loss_grad.argtypes = [P, P, P, C.c_longlong, C.c_int, C.c_int, C.c_int,
                                       C.POINTER(C.c_double), P, P]
    lib.peps_mlp_train.argtypes = [P, P, P, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_float, C.c_float, C.c_ulonglong, C.POINTER(C.c_double), P]
    lib.peps_mlp_predict.argtypes = [P, P, C.c_longlong, C.c_int, C.c_int, C.c_int, P, P]
    lib.peps_plan_create.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.c_int, C.POINTER(P), P]
    lib.peps_plan_tune.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.c_int, C.POINTER(P),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), P]
    lib.peps_plan_run.argtypes = [P, P]
    lib.peps_plan_env.argtypes = [P]
    lib.peps_plan_env.restype = P
    lib.peps_plan_launches.argtypes = [P]
    lib.peps_plan_launches.restype = C.c_longlong
    lib.peps_plan_free.argtypes = [P]
    lib.peps_plan_free.restype = None
    lib.peps_set_iteration_caps.argtypes = [C.c_int, C.c_int]
    lib.peps_wait_selftest.argtypes = [C.c_int, P]
    lib.peps_boundary_fidelity.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.c_int, C.c_int,
                                           C.POINTER(C.c_double), P]
    lib.peps_env_cluster_range.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.c_longlong, C.c_longlong,
                                           C.POINTER(P), P]
    lib.peps_ipeps_cluster.argtypes = [P, C.c_int, C.c_int, C.c_int, C.POINTER(Opts), P, P, P, P, P]
    lib.peps_bond_update.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), P, P, C.c_int, C.c_int, P, P, P]
    lib.peps_bond_update_cluster.argtypes = [C.POINTER(Lattice), C.POINTER(Opts), C.c_int, P, P, C.c_int,
                                             C.c_int, P, P, P]
    lib.peps_mlp_train_state.argtypes = [P, P, P, C.POINTER(C.c_longlong), P, P, C.c_longlong, C.c_int, C.c_int,
                                         C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_ulonglong,
                                         C.POINTER(C.c_double), P]
    lib.peps_mlp_save.argtypes = [C.c_char_p, P, P, P, C.c_longlong, C.c_int, C.c_int, C.c_int, P]
    lib.peps_mlp_load.argtypes = [C.c_char_p, P, P, P, C.POINTER(C.c_longlong), C.c_int, C.c_int, C.c_int, P]
    lib.peps_env_save.argtypes = [P, C.c_char_p, P]
    lib.peps_env_load.argtypes = [C.c_char_p, C.POINTER(P), P]
    return lib


lib = _load()


def _check(rc: int):
    if rc != OK:
        raise PepsError(rc, lib.peps_last_error().decode(errors="replace"))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)     # torch.cuda.Stream


class _Input:
    """Keeps the array alive and describes it as a peps_lattice."""

    def __init__(self, A):
        try:
            import torch
        except ImportError:          # numpy-only use
            torch = None
        if torch is not None and isinstance(A, torch.Tensor):
            assert A.dim() == 7 and A.is_contiguous(), "A must be contiguous (Ly,Lx,d,D,D,D,D)"
            assert A.dtype in (torch.float64, torch.float32)
            self.keep = A
            ptr, dev = A.data_ptr(), int(A.is_cuda)
            dt = F64 if A.dtype == torch.float64 else F32
        else:
            A = np.ascontiguousarray(A)
            if A.dtype not in (np.float64, np.float32):
                A = A.astype(np.float64)
            assert A.ndim == 7, "A must have shape (Ly,Lx,d,D,D,D,D)"
            self.keep = A
            ptr, dev = A.ctypes.data, 0
            dt = F64 if A.dtype == np.float64 else F32
        Ly, Lx, d, D = (int(v) for v in A.shape[:4])
        self.lat = Lattice(Ly, Lx, d, D, dt, ptr, dev)


def _opts(chi, mode, sweeps, precision, n, seed, closure_weights=None):
    learned = closure_weights is not None
    return Opts(int(chi), MODE[mode] if isinstance(mode, str) else int(mode), int(sweeps),
                PREC[precision] if isinstance(precision, str) else int(precision), int(n),
                1 if learned else 0, int(closure_weights.data_ptr()) if learned else None, int(seed))


class Env:
    """A device-resident environment handle (freed with the object)."""

    def __init__(self, handle, shape, stream, owner=None):
        self._h = handle
        self.Ly, self.Lx, self.d = shape
        self._stream = stream
        self._owner = owner          # a Plan owns its env handle

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_owner", None) is None:
            lib.peps_env_free(h)
        self._h = None

    def free(self):
        self.__del__()

    def _count(self, kind):
        return {"site": self.Ly * self.Lx, "hbond": self.Ly * (self.Lx - 1),
                "vbond": (self.Ly - 1) * self.Lx}[kind]

    def expect(self, kind: str, op) -> np.ndarray:
        """<O> = Tr(rho O) / Tr(rho) at every site / bond (row-major)."""
        op = np.ascontiguousarray(op, dtype=np.float64)
        out = np.zeros(self._count(kind))
        _check(lib.peps_expect_local(self._h, None, KIND[kind], op.ctypes.data, out.ctypes.data,
                                     _stream_ptr(self._stream)))
        return out

    def rho(self, kind: str) -> np.ndarray:
        k = self.d if kind == "site" else self.d * self.d
        out = np.zeros((self._count(kind), k, k))
        _check(lib.peps_env_rho(self._h, KIND[kind], out.ctypes.data, _stream_ptr(self._stream)))
        return out

    def ln_norm(self):
        ln = C.c_double()
        sg = C.c_int()
        _check(lib.peps_env_ln_norm(self._h, C.byref(ln), C.byref(sg), _stream_ptr(self._stream)))
        return ln.value, sg.value


def _set_device(device):
    if device is None:
        return
    import torch
    torch.cuda.set_device(device)


def env_full(A, chi: int, mode="svd", sweeps: int = 2, precision="fp64", seed: int = 0,
             stream=None, device=None) -> Env:
    """Full (sandwich) environments of every site; see peps_env_full."""
    _set_device(device)
    inp = _Input(A)
    o = _opts(chi, mode, sweeps, precision, 1, seed)
    h = C.c_void_p()
    _check(lib.peps_env_full(C.byref(inp.lat), C.byref(o), C.byref(h), _stream_ptr(stream)))
    return Env(h.value, (inp.lat.Ly, inp.lat.Lx, inp.lat.d), stream)


def env_cluster(A, n: int, chi: int, mode="svd", sweeps: int = 2, precision="fp64", seed: int = 0,
                stream=None, device=None, closure_weights=None, anchors=None) -> Env:
    """Cluster environments (window n x n around every site); see peps_env_cluster.
    closure_weights: a float32 CUDA tensor of learned-closure weights (width 256).
    anchors: (begin, end) -- only the windows of anchors y*Lx+x in [begin, end)
    (peps_env_cluster_range)."""
    _set_device(device)
    inp = _Input(A)
    o = _opts(chi, mode, sweeps, precision, n, seed, closure_weights)
    h = C.c_void_p()
    if anchors is None:
        _check(lib.peps_env_cluster(C.byref(inp.lat), C.byref(o), C.byref(h), _stream_ptr(stream)))
    else:
        a0, a1 = (int(v) for v in anchors)
        _check(lib.peps_env_cluster_range(C.byref(inp.lat), C.byref(o), a0, a1, C.byref(h), _stream_ptr(stream)))
    return Env(h.value, (inp.lat.Ly, inp.lat.Lx, inp.lat.d), stream)


class Plan:
    """A recorded environment computation (CUDA graph); see peps_plan_create.
    A must be a contiguous CUDA tensor; overwrite it in place between runs."""

    def __init__(self, A, chi: int, mode="svd", sweeps: int = 2, precision="fp64", seed: int = 0,
                 cluster_n: int | None = None, closure_weights=None, stream=None, device=None,
                 tune: bool = False):
        _set_device(device)
        self._inp = _Input(A)
        assert self._inp.lat.on_device, "a plan needs the lattice on the device"
        self._w = closure_weights
        o = _opts(chi, mode, sweeps, precision, cluster_n or 1, seed, closure_weights)
        self._stream = stream
        h = C.c_void_p()
        self.lanes = self.qr_cluster = None
        if tune:      # launch configuration chosen by measurement (peps_plan_tune)
            nl, qc = C.c_int(), C.c_int()
            _check(lib.peps_plan_tune(C.byref(self._inp.lat), C.byref(o), int(cluster_n is not None),
                                      C.byref(h), C.byref(nl), C.byref(qc), _stream_ptr(stream)))
            self.lanes, self.qr_cluster = nl.value, qc.value
        else:
            _check(lib.peps_plan_create(C.byref(self._inp.lat), C.byref(o), int(cluster_n is not None),
                                        C.byref(h), _stream_ptr(stream)))
        self._h = h.value
        self.launches = int(lib.peps_plan_launches(self._h))

    @property
    def env(self) -> Env:
        """The plan's environment (contents of the last run); keeps the plan alive."""
        lat = self._inp.lat
        return Env(lib.peps_plan_env(self._h), (lat.Ly, lat.Lx, lat.d), self._stream, owner=self)

    def run(self, stream=None) -> Env:
        _check(lib.peps_plan_run(self._h, _stream_ptr(stream if stream is not None else self._stream)))
        return self.env

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.peps_plan_free(h)
            self._h = None

    def free(self):
        self.__del__()


def norm(A, chi: int, mode="svd", sweeps: int = 2, precision="fp64", seed: int = 0,
         stream=None, device=None):
    """(ln|<psi|psi>|, sign) by the top-down sweep; see peps_norm."""
    _set_device(device)
    inp = _Input(A)
    o = _opts(chi, mode, sweeps, precision, 1, seed)
    ln = C.c_double()
    sg = C.c_int()
    _check(lib.peps_norm(C.byref(inp.lat), C.byref(o), C.byref(ln), C.byref(sg), _stream_ptr(stream)))
    return ln.value, sg.value


def boundary_fidelity(A, delta: int, chi: int, chi_ref: int, mode="var", sweeps: int = 2, precision="fp64",
                      seed: int = 0, stream=None, device=None) -> float:
    """1 - f of the left-most column's environment with a cluster of delta
    columns at bond chi against the full contraction at chi_ref; see
    peps_boundary_fidelity."""
    _set_device(device)
    inp = _Input(A)
    o = _opts(chi, mode, sweeps, precision, 1, seed)
    out = C.c_double()
    _check(lib.peps_boundary_fidelity(C.byref(inp.lat), C.byref(o), int(delta), int(chi_ref), C.byref(out),
                                      _stream_ptr(stream)))
    return out.value


def ipeps_cluster(A, n: int, chi: int, mode="var", sweeps: int = 2, precision="fp64", seed: int = 0,
                  stream=None, device=None) -> dict:
    """Density matrices of one site and its right / down bonds of the infinite
    PEPS with the single tensor A (d, D, D, D, D), from the infinite CU_0
    boundaries and an n x n cluster at bond chi; see peps_ipeps_cluster."""
    _set_device(device)
    try:
        import torch
    except ImportError:
        torch = None
    if torch is not None and isinstance(A, torch.Tensor):
        assert A.dim() == 5 and A.dtype == torch.float64 and A.is_contiguous()
        keep, ptr, on_dev = A, A.data_ptr(), int(A.is_cuda)
    else:
        keep = np.ascontiguousarray(A, dtype=np.float64)
        assert keep.ndim == 5
        ptr, on_dev = keep.ctypes.data, 0
    d, D = int(keep.shape[0]), int(keep.shape[1])
    assert tuple(keep.shape[1:]) == (D,) * 4, "every leg of A must have dimension D"
    o = _opts(chi, mode, sweeps, precision, n, seed)
    rs = np.zeros((d, d))
    rh = np.zeros((d * d, d * d))
    rv = np.zeros((d * d, d * d))
    sg = np.zeros((4, D, D))
    _check(lib.peps_ipeps_cluster(ptr, d, D, on_dev, C.byref(o), rs.ctypes.data, rh.ctypes.data, rv.ctypes.data,
                                  sg.ctypes.data, _stream_ptr(stream)))
    return dict(rho_site=rs, rho_h=rh, rho_v=rv, sigma=sg)


def cu0_noalloc(A_dev, sigma_dev, stream=None):
    """Top-down CU_0 boundaries into a caller-owned device tensor, with no
    device allocation (see peps_cu0_noalloc).  A_dev: contiguous float64 CUDA
    tensor (Ly,Lx,d,D,D,D,D); sigma_dev: float64 CUDA tensor (Ly,Lx,D,D)."""
    import torch
    # The C side reads and writes these buffers by the sizes alone, so every
    # property it relies on is checked here, before anything is launched.
    if A_dev.dim() != 7:
        raise ValueError(f"A must have 7 dimensions (Ly,Lx,d,D,D,D,D), got {tuple(A_dev.shape)}")
    Ly, Lx, d, D = (int(v) for v in A_dev.shape[:4])
    if tuple(A_dev.shape[3:]) != (D,) * 4:
        raise ValueError(f"A's four virtual legs must all have dimension D={D}, got {tuple(A_dev.shape)}")
    if tuple(sigma_dev.shape) != (Ly, Lx, D, D):
        raise ValueError(f"sigma must have shape {(Ly, Lx, D, D)}, got {tuple(sigma_dev.shape)}")
    for name, t in (("A", A_dev), ("sigma", sigma_dev)):
        if t.dtype != torch.float64:
            raise TypeError(f"{name} must be float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t in (("A", A_dev), ("sigma", sigma_dev)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")
    _check(lib.peps_cu0_noalloc(A_dev.data_ptr(), Ly, Lx, d, D, sigma_dev.data_ptr(), _stream_ptr(stream)))


def set_iteration_caps(cu0_half_sweeps: int = 0, jacobi_sweeps: int = 0):
    """Caps of the CU_0 half-sweeps and the Jacobi sweeps (0: default); see
    peps_set_iteration_caps."""
    _check(lib.peps_set_iteration_caps(int(cu0_half_sweeps), int(jacobi_sweeps)))


def wait_selftest(budget_us: int = 2000, stream=None):
    """Runs the bounded-wait self-test (raises PepsError with ETIMEOUT)."""
    _check(lib.peps_wait_selftest(int(budget_us), _stream_ptr(stream)))


# ---------------------------------------------------------------- learned closure
def closure_data(A, chi: int, mode="svd", precision="fp64", stream=None):
    """(X, Y) float32 CUDA tensors of closure features and labels for lattice A."""
    import torch
    inp = _Input(A)
    o = _opts(chi, mode, 2, precision, 1, 0)
    cnt = C.c_longlong()
    _check(lib.peps_closure_data(C.byref(inp.lat), C.byref(o), None, None, 0, C.byref(cnt), _stream_ptr(stream)))
    d, D = inp.lat.d, inp.lat.D
    F = d * D ** 4 + 2 * D * D
    X = torch.zeros((cnt.value, F), dtype=torch.float32, device="cuda")
    Y = torch.zeros((cnt.value, D * D), dtype=torch.float32, device="cuda")
    _check(lib.peps_closure_data(C.byref(inp.lat), C.byref(o), X.data_ptr(), Y.data_ptr(), cnt.value,
                                 C.byref(cnt), _stream_ptr(stream)))
    return X, Y


def mlp_param_count(d: int, D: int, width: int = CLOSURE_WIDTH) -> int:
    return int(lib.peps_mlp_param_count(d, D, width))


def mlp_init(d: int, D: int, width: int = CLOSURE_WIDTH, seed: int = 0, stream=None):
    import torch
    w = torch.zeros(mlp_param_count(d, D, width), dtype=torch.float32, device="cuda")
    _check(lib.peps_mlp_init(w.data_ptr(), d, D, width, int(seed), _stream_ptr(stream)))
    return w


def mlp_loss_grad(w, X, Y, d: int, D: int, width: int = CLOSURE_WIDTH, stream=None):
    import torch
    g = torch.zeros_like(w)
    loss = C.c_double()
    _check(lib.peps_mlp_loss_grad(w.data_ptr(), X.data_ptr(), Y.data_ptr(), X.shape[0], d, D, width,
                                  C.byref(loss), g.data_ptr(), _stream_ptr(stream)))
    return loss.value, g


def mlp_train(w, X, Y, d: int, D: int, width: int = CLOSURE_WIDTH, steps: int = 200, batch: int = 256,
              lr: float = 1e-3, weight_decay: float = 1e-4, seed: int = 0, stream=None) -> float:
    loss = C.c_double()
    _check(lib.peps_mlp_train(w.data_ptr(), X.data_ptr(), Y.data_ptr(), X.shape[0], d, D, width, steps, batch,
                              lr, weight_decay, int(seed), C.byref(loss), _stream_ptr(stream)))
    return loss.value


class AdamState:
    """AdamW moments and step count of a closure network, held by the caller
    so that training can be split over calls and checkpointed."""

    def __init__(self, w):
        import torch
        self.m = torch.zeros_like(w)
        self.v = torch.zeros_like(w)
        self.step = 0


def mlp_train_state(w, state: AdamState, X, Y, d: int, D: int, width: int = CLOSURE_WIDTH, steps: int = 200,
                    batch: int = 256, lr: float = 1e-3, weight_decay: float = 1e-4, seed: int = 0,
                    stream=None) -> float:
    """mlp_train continuing from ``state`` (updated in place); see peps_mlp_train_state."""
    loss = C.c_double()
    step = C.c_longlong(state.step)
    _check(lib.peps_mlp_train_state(w.data_ptr(), state.m.data_ptr(), state.v.data_ptr(), C.byref(step),
                                    X.data_ptr(), Y.data_ptr(), X.shape[0], d, D, width, steps, batch, lr,
                                    weight_decay, int(seed), C.byref(loss), _stream_ptr(stream)))
    state.step = step.value
    return loss.value


def mlp_save(path: str, w, d: int, D: int, width: int = CLOSURE_WIDTH, state: AdamState | None = None,
             stream=None):
    """Weights (and optimizer state) to a checkpoint file; see peps_mlp_save."""
    _check(lib.peps_mlp_save(os.fsencode(path), w.data_ptr(), state.m.data_ptr() if state else None,
                             state.v.data_ptr() if state else None, state.step if state else 0, d, D, width,
                             _stream_ptr(stream)))


def mlp_load(path: str, w, d: int, D: int, width: int = CLOSURE_WIDTH, state: AdamState | None = None,
             stream=None):
    """Weights (and optimizer state) from a checkpoint file into ``w`` / ``state``; see peps_mlp_load."""
    step = C.c_longlong(0)
    _check(lib.peps_mlp_load(os.fsencode(path), w.data_ptr(), state.m.data_ptr() if state else None,
                             state.v.data_ptr() if state else None, C.byref(step), d, D, width,
                             _stream_ptr(stream)))
    if state is not None:
        state.step = step.value


def env_save(env, path: str, stream=None):
    """An environment's results to a checkpoint file; see peps_env_save."""
    _check(lib.peps_env_save(env._h, os.fsencode(path), _stream_ptr(stream)))


def env_load(path: str, stream=None) -> "Env":
    """A new environment handle from a checkpoint file; see peps_env_load."""
    h = C.c_void_p()
    _check(lib.peps_env_load(os.fsencode(path), C.byref(h), _stream_ptr(stream)))
    with open(path, "rb") as f:
        hdr = json.loads(f.read(512).decode().strip())
    return Env(h.value, (hdr["Ly"], hdr["Lx"], hdr["d"]), stream)


def mlp_predict(w, X, d: int, D: int, width: int = CLOSURE_WIDTH, stream=None):
    import torch
    out = torch.zeros((X.shape[0], D * D), dtype=torch.float32, device="cuda")
    _check(lib.peps_mlp_predict(w.data_ptr(), X.data_ptr(), X.shape[0], d, D, width, out.data_ptr(),
                                _stream_ptr(stream)))
    return out


# ---------------------------------------------------------------- instrumentation
def profile_enable(mask: int = -1):
    lib.peps_profile_enable(int(mask))


def profile_reset():
    lib.peps_profile_reset()


def profile_read() -> dict:
    out = {}
    for i in range(lib.peps_profile_count()):
        n = C.c_longlong()
        ms = C.c_double()
        fl = C.c_double()
        by = C.c_double()
        _check(lib.peps_profile_read(i, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
        out[lib.peps_profile_name(i).decode()] = dict(launches=n.value, ms=ms.value,
                                                       flops=fl.value, bytes=by.value)
    return out


def class_index(name: str) -> int:
    for i in range(lib.peps_profile_count()):
        if lib.peps_profile_name(i).decode() == name:
            return i
    raise KeyError(name)


def bond_update(A, gate, bonds, chi: int, mode="var", sweeps: int = 2, precision="fp64", seed: int = 0,
                iters: int = 8, out=None, stream=None, device=None, delta=None):
    """The tensor update (Section 2) of every bond in ``bonds`` ((kind, y, x):
    kind 0 = (y,x)-(y,x+1), 1 = (y,x)-(y+1,x); no shared sites), all from the
    environment of the input state: the full one (delta None, see
    peps_bond_update) or the cluster of size delta (see
    peps_bond_update_cluster).  A: contiguous CUDA tensor (Ly,Lx,d,D,D,D,D);
    out: a tensor like A (default: A itself, updated in place).  Returns
    (out, cost) with cost[i] = |psi - G phi|^2_N / |G phi|^2_N of bond i."""
    import torch
    _set_device(device)
    assert isinstance(A, torch.Tensor) and A.is_cuda, "A must be a CUDA tensor"
    inp = _Input(A)
    if out is None:
        out = A
    assert isinstance(out, torch.Tensor) and out.is_cuda and out.is_contiguous()
    assert out.shape == A.shape and out.dtype == A.dtype, "out must be shaped and typed like A"
    d = int(A.shape[2])
    g = np.ascontiguousarray(gate, dtype=np.float64)
    assert g.shape == (d * d, d * d), "gate must be (d*d, d*d)"
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 3))
    cost = np.zeros(len(b))
    o = _opts(chi, mode, sweeps, precision, 1, seed)
    if delta is None:
        _check(lib.peps_bond_update(C.byref(inp.lat), C.byref(o), g.ctypes.data, b.ctypes.data, int(len(b)),
                                    int(iters), out.data_ptr(), cost.ctypes.data, _stream_ptr(stream)))
    else:
        _check(lib.peps_bond_update_cluster(C.byref(inp.lat), C.byref(o), int(delta), g.ctypes.data,
                                            b.ctypes.data, int(len(b)), int(iters), out.data_ptr(),
                                            cost.ctypes.data, _stream_ptr(stream)))
    return out, cost


def trotter_sets(Ly: int, Lx: int):
    """Four bond sets with no shared site (horizontal even / odd columns,
    vertical even / odd rows), the first-order Trotter order."""
    sets = []
    for par in (0, 1):
        sets.append([(0, y, x) for y in range(Ly) for x in range(par, Lx - 1, 2)])
    for par in (0, 1):
        sets.append([(1, y, x) for y in range(par, Ly - 1, 2) for x in range(Lx)])
    return [s for s in sets if s]


def evolve(A, gate, steps: int, chi: int, mode="var", sweeps: int = 2, precision="fp64", seed: int = 0,
           iters: int = 8, stream=None, device=None, delta=None):
    """``steps`` Trotter steps in place on the CUDA tensor A, every set of
    trotter_sets updated from its own environment (the parallel schedule):
    the full update (delta None) or the cluster update CU_delta.  Returns A."""
    Ly, Lx = int(A.shape[0]), int(A.shape[1])
    for _ in range(steps):
        for s in trotter_sets(Ly, Lx):
            bond_update(A, gate, s, chi, mode, sweeps, precision, seed, iters, stream=stream, device=device,
                        delta=delta)
    return A
