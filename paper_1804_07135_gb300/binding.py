"""ctypes binding of libss (include/ss.h): the same entry points, argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only converts numpy arrays and
torch tensors to pointers and raises ``SsError`` on a non-zero status.  There is no CPU fallback:
if the library cannot be built or loaded, ``load()`` raises.

Arrays crossing the boundary are ``[image][site][3]`` float32/float64, site index
``(z*ny + y)*nx + x``; numpy arrays and CPU tensors are host memory, CUDA tensors device memory.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SS_OK, SS_ERR_INVALID_ARG, SS_ERR_CUDA, SS_ERR_OOM, SS_ERR_NONFINITE, SS_ERR_TIMEOUT, SS_ERR_STATE = range(7)
SS_DTYPE_F32, SS_DTYPE_F64 = 0, 1
SS_PREC_FP32, SS_PREC_FP64 = 0, 1
SS_DIPOLE_OFF, SS_DIPOLE_DIRECT, SS_DIPOLE_FFT = 0, 1, 2
SS_INT_EULER, SS_INT_DOPRI5, SS_INT_DOPRI5_IMAGE, SS_INT_RKF45, SS_INT_RKF45_IMAGE = 0, 1, 2, 3, 4
SS_INTERP_LINEAR, SS_INTERP_SPLINE = 0, 1
SS_DYN_STRING, SS_DYN_LLG = 0, 1
_STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID_ARG", 2: "SS_ERR_CUDA", 3: "SS_ERR_OOM", 4: "SS_ERR_NONFINITE",
           5: "SS_ERR_TIMEOUT", 6: "SS_ERR_STATE"}


class SsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class ss_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("precision", ctypes.c_int), ("dipole", ctypes.c_int),
                ("reparam_every", ctypes.c_int), ("stream", ctypes.c_void_p)]


class ss_string_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("J", ctypes.c_double),
                ("D", ctypes.c_double), ("K", ctypes.c_double), ("w", ctypes.c_double), ("n_images", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# device allocator callbacks (ss_set_allocator)
SS_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
SS_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None  # keeps the installed callbacks alive

# name -> (restype, argtypes); mirrors include/ss.h
_SIGNATURES = {
    "ss_default_opts": (None, [ctypes.POINTER(ss_opts)]),
    "ss_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ss_opts),
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "ss_create_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ss_string_desc), ctypes.POINTER(ss_opts),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "ss_set_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "ss_get_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "ss_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ss_set_integrator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "ss_set_reparam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "ss_set_allocator": (ctypes.c_int, [SS_ALLOC_FN, SS_FREE_FN, ctypes.c_void_p]),
    "ss_set_dynamics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "ss_climbing_image": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ss_integrator_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "ss_energies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ss_step_energies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ss_barrier": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int)]),
    "ss_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "ss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ss_energy_terms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ss_time_kernels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "ss_field_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "ss_launch_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ss_num_strings": (ctypes.c_int, [ctypes.c_void_p]),
    "ss_string_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ss_string_desc)]),
    "ss_kernels_per_iteration": (ctypes.c_int, [ctypes.c_void_p]),
    "ss_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ss_destroy": (None, [ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libss.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libss.so is not built ({_build.LIB}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, ctx=None):
    if status != SS_OK:
        msg = _lib.ss_last_error(ctx)
        raise SsError(status, msg.decode() if msg else "")


# ---- marshalling ------------------------------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _dtype_code(x) -> int:
    if _is_torch(x):
        import torch
        if x.dtype == torch.float32:
            return SS_DTYPE_F32
        if x.dtype == torch.float64:
            return SS_DTYPE_F64
    else:
        if x.dtype == np.float32:
            return SS_DTYPE_F32
        if x.dtype == np.float64:
            return SS_DTYPE_F64
    raise TypeError(f"spin arrays must be float32 or float64, got {x.dtype}")


def _pointer(x, writable: bool = False):
    """(pointer, dtype code, on_device) of a contiguous numpy array or torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), _dtype_code(x), int(x.is_cuda)
    if not isinstance(x, np.ndarray) or not x.flags.c_contiguous:
        raise ValueError("array must be a C-contiguous numpy array")
    if writable and not x.flags.writeable:
        raise ValueError("output array is read-only")
    return ctypes.c_void_p(x.ctypes.data), _dtype_code(x), 0


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(x.size)


def ss_default_opts() -> ss_opts:
    load()
    o = ss_opts()
    _lib.ss_default_opts(ctypes.byref(o))
    return o


def make_opts(dt=0.1, precision=SS_PREC_FP32, dipole=SS_DIPOLE_FFT, reparam_every=1, stream=None) -> ss_opts:
    o = ss_default_opts()
    o.dt = float(dt)
    o.precision = int(precision)
    o.dipole = int(dipole)
    o.reparam_every = int(reparam_every)
    o.stream = stream
    return o


def ss_create(nx, ny, nz, J, D, K, w_dip, n_images, opts: ss_opts | None = None):
    load()
    ctx = ctypes.c_void_p()
    st = _lib.ss_create(int(nx), int(ny), int(nz), float(J), float(D), float(K), float(w_dip), int(n_images),
                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(ctx))
    _check(st, None)
    return ctx


def ss_create_batch(descs, opts: ss_opts | None = None):
    load()
    arr = (ss_string_desc * len(descs))()
    for i, d in enumerate(descs):
        if isinstance(d, ss_string_desc):
            arr[i] = d
        else:
            nx, ny, nz, J, D, K, w, n = d
            arr[i] = ss_string_desc(int(nx), int(ny), int(nz), float(J), float(D), float(K), float(w), int(n))
    ctx = ctypes.c_void_p()
    st = _lib.ss_create_batch(len(descs), arr, ctypes.byref(opts) if opts is not None else None, ctypes.byref(ctx))
    _check(st, None)
    return ctx


def ss_destroy(ctx) -> None:
    if ctx is not None and _lib is not None:
        _lib.ss_destroy(ctx)


def ss_string_info(ctx, string: int) -> ss_string_desc:
    d = ss_string_desc()
    _check(_lib.ss_string_info(ctx, int(string), ctypes.byref(d)), ctx)
    return d


def ss_launch_config(ctx, string: int = 0) -> dict:
    out = (ctypes.c_int * 8)()
    _check(_lib.ss_launch_config(ctx, int(string), out), ctx)
    keys = ("Px", "Py", "rows_xfwd", "rows_xinv", "threads_xfwd", "threads_yz", "threads_xinv", "energy_partials")
    return dict(zip(keys, list(out)))


def ss_num_strings(ctx) -> int:
    return int(_lib.ss_num_strings(ctx))


def ss_kernels_per_iteration(ctx) -> int:
    return int(_lib.ss_kernels_per_iteration(ctx))


def ss_last_error(ctx=None) -> str:
    load()
    m = _lib.ss_last_error(ctx)
    return m.decode() if m else ""


def _expect_size(ctx, string, x, per_image: bool = True, n_images=None):
    d = ss_string_info(ctx, string)
    n = (n_images if n_images is not None else d.n_images) * d.nx * d.ny * d.nz * 3
    if _numel(x) != n:
        raise ValueError(f"expected {n} values ([images][sites][3]), got {_numel(x)}")
    return d


def ss_set_path(ctx, string: int, spins) -> None:
    _expect_size(ctx, string, spins)
    p, dt, dev = _pointer(spins)
    _check(_lib.ss_set_path(ctx, int(string), p, dt, dev), ctx)


def ss_get_path(ctx, string: int, out) -> None:
    _expect_size(ctx, string, out)
    p, dt, dev = _pointer(out, writable=True)
    _check(_lib.ss_get_path(ctx, int(string), p, dt, dev), ctx)


def ss_step(ctx, n_iter: int) -> None:
    _check(_lib.ss_step(ctx, int(n_iter)), ctx)


def ss_set_integrator(ctx, kind: int, rtol: float = 1e-6, atol: float = 1e-8) -> None:
    _check(_lib.ss_set_integrator(ctx, int(kind), float(rtol), float(atol)), ctx)


def ss_set_allocator(alloc, free, user=None) -> None:
    """Install device allocator callbacks (SS_ALLOC_FN / SS_FREE_FN instances, or both null) for
    contexts created afterwards; the caller keeps the callback objects alive."""
    _check(_lib.ss_set_allocator(alloc, free, user))


def use_torch_allocator() -> None:
    """Contexts created from now on take their device memory from PyTorch's caching allocator
    (on the context's opts.stream) and give it back to it in ss_destroy."""
    global _allocator_refs
    import torch

    def _alloc(nbytes, device, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), int(device), int(stream or 0))
        except Exception:  # out of memory: the library reports SS_ERR_OOM
            return None

    def _free(ptr, nbytes, device, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (SS_ALLOC_FN(_alloc), SS_FREE_FN(_free))
    ss_set_allocator(refs[0], refs[1], None)
    _allocator_refs = refs


def use_cuda_malloc() -> None:
    """Contexts created from now on allocate with cudaMalloc again."""
    global _allocator_refs
    ss_set_allocator(SS_ALLOC_FN(), SS_FREE_FN(), None)
    _allocator_refs = None


def ss_set_reparam(ctx, interp: int = SS_INTERP_LINEAR, climb: bool = False) -> None:
    _check(_lib.ss_set_reparam(ctx, int(interp), int(bool(climb))), ctx)


def ss_set_dynamics(ctx, kind: int = SS_DYN_STRING, alpha: float = 0.0) -> None:
    _check(_lib.ss_set_dynamics(ctx, int(kind), float(alpha)), ctx)


def ss_climbing_image(ctx, string: int) -> int:
    k = ctypes.c_int()
    _check(_lib.ss_climbing_image(ctx, int(string), ctypes.byref(k)), ctx)
    return int(k.value)


def ss_integrator_state(ctx, string: int, image: int = -1) -> tuple[float, int, int]:
    """(carried step, accepted attempts, rejected attempts) of the adaptive integrator: the string's
    smallest step and summed counts (image = -1), or those of the system holding `image`."""
    h = ctypes.c_double()
    a, r = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.ss_integrator_state(ctx, int(string), int(image), ctypes.byref(h), ctypes.byref(a), ctypes.byref(r)),
           ctx)
    return float(h.value), int(a.value), int(r.value)


def ss_energies(ctx, string: int) -> np.ndarray:
    d = ss_string_info(ctx, string)
    out = np.zeros(d.n_images)
    _check(_lib.ss_energies(ctx, int(string), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return out


def ss_step_energies(ctx, string: int) -> np.ndarray:
    d = ss_string_info(ctx, string)
    out = np.zeros(d.n_images)
    _check(_lib.ss_step_energies(ctx, int(string), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return out


def ss_barrier(ctx, string: int) -> tuple[float, int]:
    dE = ctypes.c_double()
    k = ctypes.c_int()
    _check(_lib.ss_barrier(ctx, int(string), ctypes.byref(dE), ctypes.byref(k)), ctx)
    return float(dE.value), int(k.value)


def ss_field(ctx, string: int, out) -> None:
    _expect_size(ctx, string, out)
    p, dt, dev = _pointer(out, writable=True)
    _check(_lib.ss_field(ctx, int(string), p, dt, dev), ctx)


def ss_grad(ctx, string: int, image: int, dE_ds=None) -> np.ndarray:
    """Fills dE_ds ([N][3], optional) with dE/ds of one image; returns (dE/dJ, dE/dD, dE/dK, dE/dw)."""
    terms = np.zeros(4)
    if dE_ds is not None:
        _expect_size(ctx, string, dE_ds, n_images=1)
        p, dt, dev = _pointer(dE_ds, writable=True)
    else:
        p, dt, dev = None, SS_DTYPE_F64, 0
    _check(_lib.ss_grad(ctx, int(string), int(image), p, dt, dev,
                        terms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return terms


def ss_energy_terms(ctx, string: int) -> np.ndarray:
    """[n_images][4] = (dE/dJ, dE/dD, dE/dK, dE/dw) of every image, from one evaluation."""
    d = ss_string_info(ctx, string)
    out = np.zeros((d.n_images, 4))
    _check(_lib.ss_energy_terms(ctx, int(string), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return out


def ss_time_kernels(ctx, reps: int = 10) -> np.ndarray:
    """Mean milliseconds per timing entry of one iteration, in launch order (see include/ss.h: xfwd, yz,
    xinv, arc per size group on the Euler path; the stages of one attempt round under a Runge-Kutta
    integrator)."""
    out = np.zeros(4096)
    n = ctypes.c_int()
    _check(_lib.ss_time_kernels(ctx, int(reps), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(out),
                                ctypes.byref(n)), ctx)
    if n.value > len(out):
        raise SsError(SS_ERR_INVALID_ARG, f"{n.value} timing entries exceed the binding's buffer")
    return out[: n.value].copy()


def ss_field_noalloc(nx, ny, nz, J, D, K, w_dip, n_images, spins, field, stream=None) -> None:
    """Effective field without any device allocation (see include/ss.h): spins and field are CUDA
    float32 tensors of n_images * nx * ny * nz * 3 values.  Raises SsError on a non-zero status."""
    load()
    n = int(n_images) * int(nx) * int(ny) * int(nz) * 3
    for name, x in (("spins", spins), ("field", field)):
        if not _is_torch(x) or not x.is_cuda or _dtype_code(x) != SS_DTYPE_F32 or not x.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if _numel(x) != n:
            raise ValueError(f"{name} must hold {n} values")
    st = _lib.ss_field_noalloc(int(nx), int(ny), int(nz), float(J), float(D), float(K), float(w_dip), int(n_images),
                               ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(field.data_ptr()),
                               ctypes.c_void_p(stream) if stream else None)
    if st != SS_OK:
        raise SsError(st, "ss_field_noalloc failed")


# ---- a small owning wrapper ---------------------------------------------------------------------------

class StringMethod:
    """Owns one ss_ctx.  ``strings`` is a list of (nx, ny, nz, J, D, K, w, n_images) tuples."""

    def __init__(self, strings, dt=0.1, precision=SS_PREC_FP32, dipole=SS_DIPOLE_FFT, reparam_every=1,
                 stream=None):
        load()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        self.opts = make_opts(dt, precision, dipole, reparam_every, stream)
        self.ctx = ss_create_batch(list(strings), self.opts)
        self.strings = [ss_string_info(self.ctx, i) for i in range(ss_num_strings(self.ctx))]

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ss_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def shape(self, string=0):
        d = self.strings[string]
        return (d.n_images, d.nx * d.ny * d.nz, 3)

    def set_path(self, string, spins):
        ss_set_path(self.ctx, string, spins)

    def get_path(self, string=0, dtype=np.float64):
        out = np.zeros(self.shape(string), dtype=dtype)
        ss_get_path(self.ctx, string, out)
        return out

    def step(self, n_iter):
        ss_step(self.ctx, n_iter)

    def set_integrator(self, kind, rtol=1e-6, atol=1e-8):
        ss_set_integrator(self.ctx, kind, rtol, atol)

    def integrator_state(self, string=0, image=-1):
        return ss_integrator_state(self.ctx, string, image)

    def set_reparam(self, interp=SS_INTERP_LINEAR, climb=False):
        ss_set_reparam(self.ctx, interp, climb)

    def climbing_image(self, string=0):
        return ss_climbing_image(self.ctx, string)

    def set_dynamics(self, kind=SS_DYN_STRING, alpha=0.0):
        ss_set_dynamics(self.ctx, kind, alpha)

    def energies(self, string=0):
        return ss_energies(self.ctx, string)

    def step_energies(self, string=0):
        return ss_step_energies(self.ctx, string)

    def barrier(self, string=0):
        return ss_barrier(self.ctx, string)

    def relax(self, tol=1e-6, check_every=100, max_iter=100000):
        """Iterate until every string's barrier changes by at most `tol` (in units of J) between two
        checks `check_every` iterations apart (Sec. III repeats the two steps until the string
        converges; the paper states no criterion), or until max_iter iterations.  Returns
        (iterations done, converged, {string: [barrier at each check]})."""
        if check_every < 1 or max_iter < 0 or not tol >= 0:
            raise ValueError("check_every >= 1, max_iter >= 0 and tol >= 0 are required")
        n = ss_num_strings(self.ctx)
        history = {i: [self.barrier(i)[0]] for i in range(n)}
        done = 0
        while done < max_iter:
            k = min(check_every, max_iter - done)
            self.step(k)
            done += k
            converged = True
            for i in range(n):
                dE = self.barrier(i)[0]
                converged &= abs(dE - history[i][-1]) <= tol
                history[i].append(dE)
            if converged:
                return done, True, history
        return done, False, history

    def field(self, string=0, dtype=np.float64):
        out = np.zeros(self.shape(string), dtype=dtype)
        ss_field(self.ctx, string, out)
        return out

    def energy_terms(self, string=0):
        return ss_energy_terms(self.ctx, string)

    def grad(self, string, image, want_ds=True, dtype=np.float64):
        ds = np.zeros(self.shape(string)[1:], dtype=dtype) if want_ds else None
        terms = ss_grad(self.ctx, string, image, ds)
        return ds, terms

    def kernels_per_iteration(self):
        return ss_kernels_per_iteration(self.ctx)

    def launch_config(self, string=0):
        return ss_launch_config(self.ctx, string)

    def time_kernels(self, reps=10):
        return ss_time_kernels(self.ctx, reps)
