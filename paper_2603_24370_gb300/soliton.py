"""Thin Python binding of the C-ABI in ``include/soliton.h`` (argument marshalling only).

Every step of the relaxation runs in the CUDA kernels of ``libsoliton.so``; this
module converts arguments (numpy arrays / torch tensors / pointers), checks the
return codes and raises ``SolitonError`` with the library's message. There is no
CPU fallback: without the compiled library every call raises.

The functions keep the C names: ``ss_create_grid``, ``ss_set_theory``,
``ss_init_ansatz``, ``ss_set_fields``, ``ss_get_fields``, ``ss_get_velocity``,
``ss_force``, ``ss_step``, ``ss_minimise``, ``ss_observables``, ``ss_destroy``.
``Solver`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

SS_OK = 0
SS_ERR_ARG = -1
SS_ERR_STATE = -2
SS_ERR_CUDA = -3
SS_ERR_TIMEOUT = -4
SS_ERR_NONFINITE = -5
SS_ERR_NOT_CONVERGED = -6
SS_ERR_NOMEM = -7

SS_FP32 = 1        # compensated FP32 fields (value + remainder planes)
SS_FP64 = 2
SS_FP32_PLAIN = 3  # one FP32 plane per component
SS_ABELIAN_HIGGS = 1
SS_CHIRAL_MAGNET = 2
SS_BABY_SKYRME = 3
SS_BEC = 4
SS_SID = 5
SS_METHOD_ANF = 0       # arrested Newton flow (default)
SS_METHOD_GRADIENT = 1  # gradient descent phi <- phi - dtau G

_ERR_NAMES = {
    SS_ERR_ARG: "SS_ERR_ARG", SS_ERR_STATE: "SS_ERR_STATE", SS_ERR_CUDA: "SS_ERR_CUDA",
    SS_ERR_TIMEOUT: "SS_ERR_TIMEOUT", SS_ERR_NONFINITE: "SS_ERR_NONFINITE",
    SS_ERR_NOT_CONVERGED: "SS_ERR_NOT_CONVERGED", SS_ERR_NOMEM: "SS_ERR_NOMEM",
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsoliton.so")


class SolitonError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class ss_soliton(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("charge", ctypes.c_int),
                ("size", ctypes.c_double), ("phase", ctypes.c_double)]


class ss_status(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("grad_max", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("arrests", ctypes.c_longlong), ("converged", ctypes.c_int), ("arrested", ctypes.c_int),
                ("energy_change", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ss_batch_item(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int),
                ("solitons", ctypes.POINTER(ss_soliton)), ("n_solitons", ctypes.c_int)]


class ss_obs(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("charge", ctypes.c_double), ("flux", ctypes.c_double),
                ("grad_max", ctypes.c_double), ("grad_max_raw", ctypes.c_double), ("norm_dev", ctypes.c_double),
                ("steps", ctypes.c_longlong), ("atoms", ctypes.c_double), ("angular_momentum", ctypes.c_double),
                ("chemical_potential", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load ``libsoliton.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        pd = ctypes.POINTER(ctypes.c_double)
        sig = {
            "ss_last_error": ([], ctypes.c_char_p),
            "ss_version": ([], i),
            "ss_create_grid": ([ctypes.POINTER(vp), i, i, d, d, i, vp], i),
            "ss_set_theory": ([vp, i, pd, i], i),
            "ss_init_ansatz": ([vp, ctypes.POINTER(ss_soliton), i], i),
            "ss_set_fields": ([vp, vp, i], i),
            "ss_get_fields": ([vp, vp, i], i),
            "ss_get_velocity": ([vp, vp, i], i),
            "ss_get_remainder": ([vp, vp, i], i),
            "ss_force": ([vp, vp, i, pd, pd], i),
            "ss_step": ([vp, i, ctypes.POINTER(ss_status)], i),
            "ss_minimise": ([vp, d, ll, ctypes.POINTER(ss_status)], i),
            "ss_observables": ([vp, ctypes.POINTER(ss_obs)], i),
            "ss_profile_stages": ([vp, i, ctypes.POINTER(ctypes.c_float)], i),
            "ss_observables_noalloc": ([i, pd, i, vp, i, i, d, d, i, vp, vp], i),
            "ss_batch_create": ([ctypes.POINTER(vp), i, i, ctypes.POINTER(ss_batch_item), i, vp], i),
            "ss_batch_size": ([vp], i),
            "ss_batch_step": ([vp, i, ctypes.POINTER(ss_status)], i),
            "ss_batch_minimise": ([vp, d, ll, ctypes.POINTER(ss_status)], i),
            "ss_batch_get_fields": ([vp, i, vp, i], i),
            "ss_batch_set_fields": ([vp, i, vp, i], i),
            "ss_batch_autotune": ([vp, i, ctypes.POINTER(ctypes.c_int)], i),
            "ss_autotune": ([vp, i, ctypes.POINTER(ctypes.c_int)], i),
            "ss_batch_set_launch": ([vp, i, ctypes.POINTER(ctypes.c_int)], i),
            "ss_set_launch": ([vp, i, ctypes.POINTER(ctypes.c_int)], i),
            "ss_batch_set_method": ([vp, i, d], i),
            "ss_set_method": ([vp, i, d], i),
            "ss_batch_observables": ([vp, i, ctypes.POINTER(ss_obs)], i),
            "ss_batch_destroy": ([vp], i),
            "ss_destroy": ([vp], i),
            # learned initialiser (soliton_net.h)
            "ss_net_create": ([ctypes.POINTER(vp), i, i, i, ctypes.c_ulonglong, vp], i),
            "ss_net_destroy": ([vp], i),
            "ss_net_last_error": ([], ctypes.c_char_p),
            "ss_net_num_params": ([vp], ll),
            "ss_net_get_params": ([vp, vp], i),
            "ss_net_set_params": ([vp, vp], i),
            "ss_net_save": ([vp, ctypes.c_char_p], i),
            "ss_net_load": ([vp, ctypes.c_char_p], i),
            "ss_net_pack": ([vp, vp, pd, i, vp], i),
            "ss_net_forward": ([vp, vp, pd, i, vp], i),
            "ss_net_gradients": ([vp, vp, pd, vp, i, vp, pd], i),
            "ss_net_train_step": ([vp, vp, pd, vp, i, ctypes.c_float, pd], i),
            "ss_net_predict": ([vp, vp, pd, i, vp], i),
            "ss_net_apply_gradients": ([vp, vp, ctypes.c_float], i),
            "ss_net_get_optimizer_state": ([vp, vp, vp, ctypes.POINTER(ll)], i),
            "ss_conv3x3": ([vp, i, i, i, i, vp, i, vp, i, vp, vp], i),
            "ss_conv3x3_wgrad": ([vp, vp, i, i, i, i, i, vp, vp], i),
            "ss_wait_selftest": ([i, vp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load_library().ss_last_error().decode(errors="replace")


def _check(rc: int, allow=()):
    if rc != SS_OK and rc not in allow:
        raise SolitonError(rc, last_error())
    return rc


def _ptr(arr, dtype):
    """(pointer, is_device) of a contiguous numpy array or torch tensor of ``dtype``."""
    if hasattr(arr, "data_ptr"):  # torch tensor
        import torch
        want = torch.float32 if dtype == np.float32 else torch.float64
        if arr.dtype != want or not arr.is_contiguous():
            raise ValueError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(arr.data_ptr()), 1 if arr.is_cuda else 0
    if not isinstance(arr, np.ndarray) or arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"]:
        raise ValueError(f"array must be a C-contiguous numpy {np.dtype(dtype).name} array")
    return ctypes.c_void_p(arr.ctypes.data), 0


# ---------------------------------------------------------------- C names
def ss_create_grid(nx: int, ny: int, dx: float, dy: float, precision: int = SS_FP32, stream=None):
    lib = load_library()
    ctx = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.ss_create_grid(ctypes.byref(ctx), nx, ny, dx, dy, precision, s))
    return ctx


def ss_set_theory(ctx, theory: int, params) -> None:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
    _check(load_library().ss_set_theory(ctx, theory, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size))


def ss_init_ansatz(ctx, solitons) -> None:
    rows = np.asarray(solitons, dtype=np.float64).reshape(-1, 5)
    arr = (ss_soliton * max(len(rows), 1))()
    for k, (x, y, q, size, ph) in enumerate(rows):
        if q != int(q):
            raise ValueError("soliton charges must be integers")
        arr[k] = ss_soliton(x, y, int(q), size, ph)
    _check(load_library().ss_init_ansatz(ctx, arr, len(rows)))


def ss_set_fields(ctx, fields, dtype) -> None:
    p, dev = _ptr(fields, dtype)
    _check(load_library().ss_set_fields(ctx, p, dev))


def ss_get_fields(ctx, out) -> None:
    p, dev = _ptr(out, np.float32 if _dtype_of(out) == np.float32 else np.float64)
    _check(load_library().ss_get_fields(ctx, p, dev))


def ss_get_remainder(ctx, out) -> None:
    p, dev = _ptr(out, np.float32 if _dtype_of(out) == np.float32 else np.float64)
    _check(load_library().ss_get_remainder(ctx, p, dev))


def ss_get_velocity(ctx, out) -> None:
    p, dev = _ptr(out, np.float32 if _dtype_of(out) == np.float32 else np.float64)
    _check(load_library().ss_get_velocity(ctx, p, dev))


def ss_force(ctx, out):
    p, dev = _ptr(out, np.float32 if _dtype_of(out) == np.float32 else np.float64)
    e, g = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ss_force(ctx, p, dev, ctypes.byref(e), ctypes.byref(g)))
    return e.value, g.value


def ss_step(ctx, n_steps: int, allow=()) -> dict:
    st = ss_status()
    rc = _check(load_library().ss_step(ctx, int(n_steps), ctypes.byref(st)), allow)
    d = st.as_dict()
    d["rc"] = rc
    return d


def ss_minimise(ctx, tol: float, max_steps: int, allow=(SS_ERR_NOT_CONVERGED,)) -> dict:
    st = ss_status()
    rc = _check(load_library().ss_minimise(ctx, float(tol), int(max_steps), ctypes.byref(st)), allow)
    d = st.as_dict()
    d["rc"] = rc
    return d


def ss_observables(ctx) -> dict:
    o = ss_obs()
    _check(load_library().ss_observables(ctx, ctypes.byref(o)))
    return o.as_dict()


def ss_profile_stages(ctx, n_steps: int) -> list[float]:
    """Mean device milliseconds of the step's two kernels (pass 1: RK stages 1-2 +
    reductions + arrest decision; pass 2: RK stages 3-4 + combination) over n_steps
    real flow steps; under gradient descent [descent kernel, 0.0]."""
    ms = (ctypes.c_float * 2)()
    _check(load_library().ss_profile_stages(ctx, int(n_steps), ms))
    return [float(x) for x in ms]


def ss_observables_noalloc(theory: int, params, fields, nx: int, ny: int, dx: float, dy: float, precision: int,
                           out, stream=None) -> None:
    """Observables of a device field into a device buffer of 6 doubles, with no
    allocation (see include/soliton.h). ``fields`` and ``out`` are CUDA tensors or
    device addresses; the call is asynchronous on ``stream``."""
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
    f = ctypes.c_void_p(fields.data_ptr() if hasattr(fields, "data_ptr") else int(fields))
    o = ctypes.c_void_p(out.data_ptr() if hasattr(out, "data_ptr") else int(out))
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load_library().ss_observables_noalloc(theory, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, f,
                                                 nx, ny, dx, dy, precision, o, s))


def ss_destroy(ctx) -> None:
    if ctx is not None:
        _check(load_library().ss_destroy(ctx))


def _dtype_of(a):
    if hasattr(a, "data_ptr"):
        import torch
        return np.float32 if a.dtype == torch.float32 else np.float64
    return a.dtype.type


# ---------------------------------------------------------------- batches
def _soliton_array(solitons):
    rows = np.asarray(solitons, dtype=np.float64).reshape(-1, 5)
    arr = (ss_soliton * max(len(rows), 1))()
    for k, (x, y, q, size, ph) in enumerate(rows):
        if q != int(q):
            raise ValueError("soliton charges must be integers")
        arr[k] = ss_soliton(x, y, int(q), size, ph)
    return arr, len(rows)


def ss_batch_create(theory: int, precision: int, problems, stream=None):
    """``problems``: objects with nx, ny, dx, dy, params, solitons (e.g. inputs.Problem)."""
    keep = []
    items = (ss_batch_item * len(problems))()
    for k, pr in enumerate(problems):
        prm = np.ascontiguousarray(np.asarray(pr.params, dtype=np.float64).reshape(-1))
        sol, ns = _soliton_array(pr.solitons)
        keep += [prm, sol]
        items[k] = ss_batch_item(pr.nx, pr.ny, pr.dx, pr.dy, prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 prm.size, sol, ns)
    b = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load_library().ss_batch_create(ctypes.byref(b), theory, precision, items, len(problems), s))
    return b


def _statuses(arr):
    return [arr[k].as_dict() for k in range(len(arr))]


def ss_batch_step(b, n_steps: int, allow=()):
    n = load_library().ss_batch_size(b)
    st = (ss_status * n)()
    rc = _check(load_library().ss_batch_step(b, int(n_steps), st), allow)
    return rc, _statuses(st)


def ss_batch_minimise(b, tol: float, max_steps: int, allow=(SS_ERR_NOT_CONVERGED,)):
    n = load_library().ss_batch_size(b)
    st = (ss_status * n)()
    rc = _check(load_library().ss_batch_minimise(b, float(tol), int(max_steps), st), allow)
    return rc, _statuses(st)


def ss_batch_get_fields(b, item: int, out) -> None:
    p, dev = _ptr(out, np.float32 if _dtype_of(out) == np.float32 else np.float64)
    _check(load_library().ss_batch_get_fields(b, int(item), p, dev))


def ss_batch_set_fields(b, item: int, fields) -> None:
    p, dev = _ptr(fields, np.float32 if _dtype_of(fields) == np.float32 else np.float64)
    _check(load_library().ss_batch_set_fields(b, item, p, dev))


def ss_batch_autotune(b, trial_steps: int = 8) -> dict:
    c = (ctypes.c_int * 3)()
    _check(load_library().ss_batch_autotune(b, trial_steps, c))
    return {"tile_shape": c[0], "blocks": [c[1], c[2]]}


def ss_autotune(ctx, trial_steps: int = 8) -> dict:
    c = (ctypes.c_int * 3)()
    _check(load_library().ss_autotune(ctx, trial_steps, c))
    return {"tile_shape": c[0], "blocks": [c[1], c[2]]}


def _blocks(blocks):
    if blocks is None:
        return None
    arr = (ctypes.c_int * 2)(int(blocks[0]), int(blocks[1]))
    return arr


def ss_batch_set_launch(b, tile_shape: int, blocks=None) -> None:
    _check(load_library().ss_batch_set_launch(b, tile_shape, _blocks(blocks)))


def ss_set_launch(ctx, tile_shape: int, blocks=None) -> None:
    _check(load_library().ss_set_launch(ctx, tile_shape, _blocks(blocks)))


def ss_batch_set_method(b, method: int, step_factor: float = 0.0) -> None:
    _check(load_library().ss_batch_set_method(b, int(method), float(step_factor)))


def ss_set_method(ctx, method: int, step_factor: float = 0.0) -> None:
    _check(load_library().ss_set_method(ctx, int(method), float(step_factor)))


def ss_batch_observables(b, item: int) -> dict:
    o = ss_obs()
    _check(load_library().ss_batch_observables(b, int(item), ctypes.byref(o)))
    return o.as_dict()


def ss_batch_destroy(b) -> None:
    if b is not None:
        _check(load_library().ss_batch_destroy(b))


# ---------------------------------------------------------------- convenience
class Solver:
    """One relaxation problem on the GPU: a context plus its shape and dtype."""

    def __init__(self, theory: int, params, nx: int, ny: int, dx: float, dy: float, precision: int = SS_FP32,
                 stream=None):
        self.theory, self.nx, self.ny, self.dx, self.dy = theory, nx, ny, dx, dy
        self.precision = precision
        self.C = {SS_ABELIAN_HIGGS: 4, SS_BEC: 2, SS_SID: 6}.get(theory, 3)
        self.dtype = np.float64 if precision == SS_FP64 else np.float32
        self.ctx = None
        self.ctx = ss_create_grid(nx, ny, dx, dy, precision, stream)
        try:
            ss_set_theory(self.ctx, theory, params)
        except Exception:
            ctx, self.ctx = self.ctx, None  # the destructor must not release it again
            ss_destroy(ctx)
            raise

    @property
    def shape(self):
        return (self.C, self.ny, self.nx)

    def init_ansatz(self, solitons):
        ss_init_ansatz(self.ctx, solitons)

    def set_fields(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=self.dtype)
        ss_set_fields(self.ctx, f, self.dtype)

    def fields(self, out=None):
        out = np.empty(self.shape, dtype=self.dtype) if out is None else out
        ss_get_fields(self.ctx, out)
        return out

    def remainder(self):
        """Rounding remainder of a compensated FP32 field (zeros otherwise)."""
        out = np.empty(self.shape, dtype=self.dtype)
        ss_get_remainder(self.ctx, out)
        return out

    def exact_fields(self):
        """value + remainder in FP64: the field the flow holds."""
        return self.fields().astype(np.float64) + self.remainder().astype(np.float64)

    def velocity(self):
        out = np.empty(self.shape, dtype=self.dtype)
        ss_get_velocity(self.ctx, out)
        return out

    def force(self):
        out = np.empty(self.shape, dtype=self.dtype)
        e, g = ss_force(self.ctx, out)
        return out, e, g

    def step(self, n: int, allow=()):
        return ss_step(self.ctx, n, allow)

    def autotune(self, trial_steps: int = 8) -> dict:
        """Pick the fastest tile shape and pass grids (the flow restarts from rest)."""
        return ss_autotune(self.ctx, trial_steps)

    def set_launch(self, tile_shape: int, blocks=None) -> None:
        ss_set_launch(self.ctx, tile_shape, blocks)

    def set_method(self, method: int, step_factor: float = 0.0) -> None:
        """SS_METHOD_ANF or SS_METHOD_GRADIENT (dtau = step_factor x the stability
        limit, 0.8 when <= 0); the flow restarts from the current field at rest."""
        ss_set_method(self.ctx, method, step_factor)

    def minimise(self, tol: float, max_steps: int):
        return ss_minimise(self.ctx, tol, max_steps)

    def observables(self):
        return ss_observables(self.ctx)

    def close(self):
        if self.ctx is not None:
            ss_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned initialiser
def _dev(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not hasattr(t, "data_ptr") or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _net_check(rc: int):
    if rc != SS_OK:
        raise SolitonError(rc, load_library().ss_net_last_error().decode(errors="replace"))


def _couplings(c, batch):
    if c is None:
        return None
    arr = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    if arr.size < batch:
        raise ValueError("one coupling value per problem is required")
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ss_net_create(theory: int, size: int, max_batch: int, seed: int = 0, stream=None):
    h = ctypes.c_void_p()
    _net_check(load_library().ss_net_create(ctypes.byref(h), theory, size, max_batch, seed, _stream_ptr(stream)))
    return h


def ss_net_destroy(net) -> None:
    if net:
        load_library().ss_net_destroy(net)


def ss_net_num_params(net) -> int:
    return int(load_library().ss_net_num_params(net))


def ss_net_get_params(net) -> np.ndarray:
    out = np.empty(ss_net_num_params(net), dtype=np.float32)
    _net_check(load_library().ss_net_get_params(net, ctypes.c_void_p(out.ctypes.data)))
    return out


def ss_net_set_params(net, theta) -> None:
    a = np.ascontiguousarray(theta, dtype=np.float32)
    if a.size != ss_net_num_params(net):
        raise ValueError("wrong number of parameters")
    _net_check(load_library().ss_net_set_params(net, ctypes.c_void_p(a.ctypes.data)))


def ss_net_save(net, path: str) -> None:
    _net_check(load_library().ss_net_save(net, os.fsencode(path)))


def ss_net_load(net, path: str) -> None:
    _net_check(load_library().ss_net_load(net, os.fsencode(path)))


def ss_net_pack(net, fields, couplings, batch: int, input_nhwc) -> None:
    keep = _couplings(couplings, batch)
    _net_check(load_library().ss_net_pack(net, _dev(fields), keep[1] if keep else None, batch, _dev(input_nhwc)))


def ss_net_forward(net, ansatz, couplings, batch: int, out=None) -> None:
    keep = _couplings(couplings, batch)
    _net_check(load_library().ss_net_forward(net, _dev(ansatz), keep[1] if keep else None, batch, _dev(out)))


def ss_net_gradients(net, ansatz, couplings, relaxed, batch: int, grad_out=None) -> float:
    keep = _couplings(couplings, batch)
    loss = ctypes.c_double()
    _net_check(load_library().ss_net_gradients(net, _dev(ansatz), keep[1] if keep else None, _dev(relaxed), batch,
                                               _dev(grad_out), ctypes.byref(loss)))
    return loss.value


def ss_net_train_step(net, ansatz, couplings, relaxed, batch: int, lr: float) -> float:
    keep = _couplings(couplings, batch)
    loss = ctypes.c_double()
    _net_check(load_library().ss_net_train_step(net, _dev(ansatz), keep[1] if keep else None, _dev(relaxed), batch,
                                                lr, ctypes.byref(loss)))
    return loss.value


def ss_net_apply_gradients(net, grad, lr: float) -> None:
    _net_check(load_library().ss_net_apply_gradients(net, _dev(grad), lr))


def ss_net_get_optimizer_state(net):
    """(m, v, updates taken) of the network's Adam state, m and v as host float32 arrays."""
    n = ss_net_num_params(net)
    m = np.empty(n, dtype=np.float32)
    v = np.empty(n, dtype=np.float32)
    t = ctypes.c_longlong()
    _net_check(load_library().ss_net_get_optimizer_state(net, ctypes.c_void_p(m.ctypes.data),
                                                         ctypes.c_void_p(v.ctypes.data), ctypes.byref(t)))
    return m, v, int(t.value)


def ss_net_predict(net, ansatz, couplings, batch: int, init) -> None:
    keep = _couplings(couplings, batch)
    _net_check(load_library().ss_net_predict(net, _dev(ansatz), keep[1] if keep else None, batch, _dev(init)))


def ss_conv3x3(x, w, bias, mode: int, out, stream=None) -> None:
    N, H, W, Cin = x.shape
    Cout = w.shape[0]
    _net_check(load_library().ss_conv3x3(_dev(x), N, H, W, Cin, _dev(w), Cout, _dev(bias), mode, _dev(out),
                                         _stream_ptr(stream)))


def ss_conv3x3_wgrad(dy, x, dw, stream=None) -> None:
    N, H, W, Cin = x.shape
    Cout = dy.shape[3]
    _net_check(load_library().ss_conv3x3_wgrad(_dev(dy), _dev(x), N, H, W, Cout, Cin, _dev(dw),
                                               _stream_ptr(stream)))


def ss_wait_selftest(limit_us: int, stream=None) -> int:
    """Return code of the bounded-wait self-test (SS_ERR_TIMEOUT when it works)."""
    return int(load_library().ss_wait_selftest(limit_us, _stream_ptr(stream)))
