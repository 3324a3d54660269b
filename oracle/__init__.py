"""FP64 CPU oracle for the simplified string method (arXiv:1804.07135), plain C behind ctypes.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
are the only callers.  Nothing here is shared with, or imported by, the CUDA path.

Every wrapper takes and returns numpy float64 arrays in the layout ``[image][site][3]`` (or
``[site][3]`` for one image), with site index ``(z*ny + y)*nx + x``.  Units are reduced: energies
in units of J's unit, lengths in lattice constants, ``h = -dE/ds``, ``w = mu0 |S|^2 / (4 pi a^3)``.

Parity status: see the header of ``ssm_oracle.c``; the barrier value itself is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleModel(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("J", ctypes.c_double), ("D", ctypes.c_double), ("K", ctypes.c_double),
                ("w", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ssm_oracle.c with gcc (-O2, IEEE arithmetic, OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        i = ctypes.c_int
        dp = P(d)
        mp = P(OracleModel)
        sig = {
            "or_dipole_tensor": (None, [d, d, d, dp]),
            "or_energy_terms": (None, [mp, dp, dp]),
            "or_field": (i, [mp, i, dp, dp]),
            "or_dipole_field": (i, [mp, dp, dp]),
            "or_field_at": (i, [mp, dp, i, P(i), dp]),
            "or_energy_from_field": (d, [i, dp, dp]),
            "or_step": (None, [i, d, dp, dp]),
            "or_reparam": (None, [i, i, dp, dp, dp]),
            "or_string_run": (i, [mp, i, i, d, dp, dp]),
            "or_reparam_v": (None, [i, i, dp, dp, i, i, dp]),
            "or_string_run_v": (i, [mp, i, i, d, i, i, dp, dp, P(ctypes.c_int)]),
            "or_string_run_rk": (i, [mp, i, i, d, d, d, i, dp, dp, dp, P(ctypes.c_long)]),
            "or_llg_run": (i, [mp, i, i, d, d, dp, dp]),
            "or_llg_run_rk": (i, [mp, i, i, d, d, d, d, i, dp, dp, dp, P(ctypes.c_long)]),
            "or_dp_tableau": (None, [dp, dp, dp]),
            "or_rkf_tableau": (None, [dp, dp, dp]),
            "or_string_run_rk_method": (i, [mp, i, i, d, d, d, i, i, dp, dp, dp, P(ctypes.c_long)]),
            "or_barrier": (d, [i, dp, P(i)]),
            "or_energy_param_grad": (None, [mp, dp, dp]),
            "or_max_threads": (i, []),
            "or_set_threads": (None, [i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def model(nx, ny, nz, J=1.0, D=0.0, K=0.0, w=0.0) -> OracleModel:
    return OracleModel(int(nx), int(ny), int(nz), float(J), float(D), float(K), float(w))


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_max_threads())


def dipole_tensor(r) -> np.ndarray:
    """Eq. 7 at offset r (lattice units): (xx, yy, zz, xy, xz, yz)."""
    out = np.zeros(6)
    _load().or_dipole_tensor(float(r[0]), float(r[1]), float(r[2]), _ptr(out))
    return out


def energy_terms(m: OracleModel, s) -> dict:
    """Eq. 1 term by term: exchange, dmi, anisotropy, dipole, total."""
    s = _f64(s)
    out = np.zeros(5)
    _load().or_energy_terms(ctypes.byref(m), _ptr(s), _ptr(out))
    return dict(zip(("exchange", "dmi", "anisotropy", "dipole", "total"), out.tolist()))


def field(m: OracleModel, s) -> np.ndarray:
    """Eqs. 2-7: h = -dE/ds for one image [N,3] or a batch [K,N,3]."""
    s = _f64(s)
    n_img = 1 if s.ndim == 2 else s.shape[0]
    h = np.zeros_like(s)
    if _load().or_field(ctypes.byref(m), n_img, _ptr(s), _ptr(h)) != 0:
        raise MemoryError("oracle field: out of memory")
    return h


def field_at(m: OracleModel, s, sites) -> np.ndarray:
    """Eqs. 2-7 of one image [N,3] at the given site indices -> [len(sites), 3]."""
    s = _f64(s)
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
    out = np.zeros((sites.size, 3))
    st = _load().or_field_at(ctypes.byref(m), _ptr(s), int(sites.size),
                             sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out))
    if st != 0:
        raise ValueError("oracle field_at: out of memory or site index out of range")
    return out


def dipole_field(m: OracleModel, s) -> np.ndarray:
    """Eq. 6 alone (direct O(N^2) sum) for one image."""
    s = _f64(s)
    h = np.zeros_like(s)
    if _load().or_dipole_field(ctypes.byref(m), _ptr(s), _ptr(h)) != 0:
        raise MemoryError("oracle dipole field: out of memory")
    return h


def energy_from_field(s, h) -> float:
    """Eq. 8."""
    s, h = _f64(s), _f64(h)
    return float(_load().or_energy_from_field(s.size // 3, _ptr(s), _ptr(h)))


def energies(m: OracleModel, path) -> np.ndarray:
    """Eq. 8 for every image of a [K,N,3] path."""
    path = _f64(path)
    h = field(m, path)
    return np.array([energy_from_field(path[k], h[k]) for k in range(path.shape[0])])


def step(s, h, dt: float) -> np.ndarray:
    """Eq. 10 with the force of Eq. 13: one projected Euler step + renormalisation (copy)."""
    s = _f64(s).copy()
    h = _f64(h)
    _load().or_step(s.size // 3, float(dt), _ptr(h), _ptr(s))
    return s


def reparam(path, return_alpha: bool = False):
    """Eqs. 11-12 + interpolation onto alpha_k = k/(K-1) (copy)."""
    star = _f64(path)
    K = star.shape[0]
    out = np.zeros_like(star)
    alpha = np.zeros(K)
    _load().or_reparam(K, star[0].size // 3, _ptr(star), _ptr(out), _ptr(alpha))
    return (out, alpha) if return_alpha else out


def string_run(m: OracleModel, path, n_iter: int, dt: float, with_energies: bool = True):
    """Sec. III loop: n_iter x (step all images, reparametrise).  Returns (final path, energies or None)."""
    phi = _f64(path).copy()
    K = phi.shape[0]
    e = np.zeros(K) if with_energies else None
    if _load().or_string_run(ctypes.byref(m), K, int(n_iter), float(dt), _ptr(phi),
                             _ptr(e) if with_energies else None) != 0:
        raise MemoryError("oracle string run: out of memory")
    return phi, e


def reparam_v(path, spline: bool = False, kc: int = -1, return_alpha: bool = False):
    """Reparametrisation with the variants: natural cubic spline instead of linear interpolation,
    and/or a climbing image kc splitting the string into two parts."""
    star = _f64(path)
    K = star.shape[0]
    out = np.zeros_like(star)
    alpha = np.zeros(K)
    _load().or_reparam_v(K, star[0].size // 3, _ptr(star), _ptr(out), int(bool(spline)), int(kc), _ptr(alpha))
    return (out, alpha) if return_alpha else out


def string_run_v(m: OracleModel, path, n_iter: int, dt: float, spline: bool = False, climb: bool = False,
                 with_energies: bool = True):
    """Sec. III loop (Euler step) with the spline and climbing-image variants.  Returns (final path,
    energies or None, the climbing image the next iteration would use or -1)."""
    phi = _f64(path).copy()
    K = phi.shape[0]
    e = np.zeros(K) if with_energies else None
    kc = ctypes.c_int(-1)
    if _load().or_string_run_v(ctypes.byref(m), K, int(n_iter), float(dt), int(bool(spline)), int(bool(climb)),
                               _ptr(phi), _ptr(e) if with_energies else None, ctypes.byref(kc)) != 0:
        raise MemoryError("oracle string run: out of memory")
    return phi, e, int(kc.value)


def string_run_rk(m: OracleModel, path, n_iter: int, T: float, rtol: float = 1e-6, atol: float = 1e-8,
                  step=None, with_energies: bool = True, per_image: bool = False, method: str = "dopri5"):
    """Sec. III loop with an adaptive embedded Runge-Kutta evolution over T per iteration: the
    Dormand-Prince 5(4) pair (method="dopri5") or the Runge-Kutta-Fehlberg 4(5) pair ("rkf45"); the
    whole string one ODE system (per_image=False) or every image its own (per_image=True).  Returns
    (final path, energies or None, carried step, (accepted, rejected)); with per_image the step is an
    array of K steps and the counts an array of K (accepted, rejected) rows."""
    phi = _f64(path).copy()
    K = phi.shape[0]
    n_sys = K if per_image else 1
    e = np.zeros(K) if with_energies else None
    h = np.full(n_sys, float(T)) if step is None else np.array(np.broadcast_to(np.asarray(step, float), (n_sys,)))
    counts = (ctypes.c_long * (2 * n_sys))()
    meth = {"dopri5": 0, "rkf45": 1}[method]
    rc = _load().or_string_run_rk_method(ctypes.byref(m), K, int(n_iter), float(T), float(rtol), float(atol), meth,
                                         int(bool(per_image)), _ptr(h), _ptr(phi), _ptr(e) if with_energies else None,
                                         counts)
    if rc == -1:
        raise MemoryError("oracle RK string run: out of memory")
    if rc != 0:
        raise RuntimeError("oracle RK string run: step size collapsed")
    c = np.array(counts[:], dtype=np.int64).reshape(n_sys, 2)
    if per_image:
        return phi, e, h, c
    return phi, e, float(h[0]), (int(c[0, 0]), int(c[0, 1]))


def llg_run(m: OracleModel, states, n_steps: int, dt: float, alpha: float, with_energies: bool = True):
    """Eq. 9 (reduced units) by explicit Euler steps with renormalisation, every image on its own.
    Returns (final states, energies or None)."""
    phi = _f64(states).copy()
    K = phi.shape[0]
    e = np.zeros(K) if with_energies else None
    if _load().or_llg_run(ctypes.byref(m), K, int(n_steps), float(dt), float(alpha), _ptr(phi),
                          _ptr(e) if with_energies else None) != 0:
        raise MemoryError("oracle LLG run: out of memory")
    return phi, e


def llg_run_rk(m: OracleModel, states, n_iter: int, T: float, alpha: float, rtol: float = 1e-6, atol: float = 1e-8,
               step=None, with_energies: bool = True, per_image: bool = False):
    """Eq. 9 (reduced units) with the Dormand-Prince 5(4) pair over n_iter intervals of T, no
    reparametrisation.  Returns as string_run_rk."""
    phi = _f64(states).copy()
    K = phi.shape[0]
    n_sys = K if per_image else 1
    e = np.zeros(K) if with_energies else None
    h = np.full(n_sys, float(T)) if step is None else np.array(np.broadcast_to(np.asarray(step, float), (n_sys,)))
    counts = (ctypes.c_long * (2 * n_sys))()
    rc = _load().or_llg_run_rk(ctypes.byref(m), K, int(n_iter), float(T), float(alpha), float(rtol), float(atol),
                               int(bool(per_image)), _ptr(h), _ptr(phi), _ptr(e) if with_energies else None, counts)
    if rc == -1:
        raise MemoryError("oracle LLG run: out of memory")
    if rc != 0:
        raise RuntimeError("oracle LLG run: step size collapsed")
    c = np.array(counts[:], dtype=np.int64).reshape(n_sys, 2)
    if per_image:
        return phi, e, h, c
    return phi, e, float(h[0]), (int(c[0, 0]), int(c[0, 1]))


def dp_tableau():
    """The Dormand-Prince 5(4) coefficients the oracle uses: (a[7][6], b[7], bhat[7])."""
    a, b, bh = np.zeros((7, 6)), np.zeros(7), np.zeros(7)
    _load().or_dp_tableau(_ptr(a), _ptr(b), _ptr(bh))
    return a, b, bh


def rkf_tableau():
    """The Runge-Kutta-Fehlberg 4(5) coefficients the oracle uses: (a[6][5], b4[6], b5[6])."""
    a, b4, b5 = np.zeros((6, 5)), np.zeros(6), np.zeros(6)
    _load().or_rkf_tableau(_ptr(a), _ptr(b4), _ptr(b5))
    return a, b4, b5


def barrier(energies_) -> tuple[float, int]:
    """max_k E_k - E_0, lowest index on ties."""
    e = _f64(energies_)
    k = ctypes.c_int(0)
    dE = _load().or_barrier(e.size, _ptr(e), ctypes.byref(k))
    return float(dE), int(k.value)


def energy_param_grad(m: OracleModel, s) -> np.ndarray:
    """(dE/dJ, dE/dD, dE/dK, dE/dw) of one image (Eq. 1 is linear in each)."""
    s = _f64(s)
    out = np.zeros(4)
    _load().or_energy_param_grad(ctypes.byref(m), _ptr(s), _ptr(out))
    return out
