"""FP64 CPU oracle for the PA-SFM radiation operator (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never links, loads
or calls it, and it imports nothing from the product package.

``pasfm_oracle.c`` holds the operator (forward, adjoint, pose gradient, loss
head) written pair by pair in FP64 from the paper's Appendix A closed forms
(uniform sphere; outgoing Gaussian of Eq. 1 with kernel K_G) and Eq. 1; ``rigid.py`` holds the host-side rigid-body pieces (SO(3) exponential,
Kabsch fit, RANSAC consensus with the pairwise-edge pre-check of Stage 3) and
``adam.py`` the textbook Adam step.  Parity status of every function is listed
in each module's header; all are pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pasfm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


class OracleGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_elem", ctypes.c_int32), ("n_frames", ctypes.c_int32),
                ("n_samples", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("fs", ctypes.c_double), ("t0", ctypes.c_double), ("c", ctypes.c_double),
                ("a0", ctypes.c_double), ("point_sampling", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("vol_pose", ctypes.c_double * 12),
                ("sigma", ctypes.c_double)]

KERNELS = {"sphere": 0, "gauss": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"])
    return _LIB


def load(path: str):
    """Open a compiled oracle library and declare its signatures."""
    L = ctypes.CDLL(path)
    g = ctypes.POINTER(OracleGeom)
    dp = np.ctypeslib.ndpointer(np.float64, flags="C")
    fp = np.ctypeslib.ndpointer(np.float32, flags="C")
    L.oracle_support.argtypes = [g]
    L.oracle_support.restype = ctypes.c_double
    L.oracle_pulse.argtypes = [g, ctypes.c_double, ctypes.c_int]
    L.oracle_pulse.restype = ctypes.c_double
    L.oracle_pulse_dd.argtypes = [g, ctypes.c_double, ctypes.c_int]
    L.oracle_pulse_dd.restype = ctypes.c_double
    L.oracle_element_positions.argtypes = [g, dp, dp, dp]
    L.oracle_check_geometry.argtypes = [g, dp]
    L.oracle_check_geometry.restype = ctypes.c_int64
    L.oracle_forward_rows.argtypes = [g, fp, dp, ctypes.c_void_p, ctypes.c_int64, dp]
    L.oracle_adjoint_voxels.argtypes = [g, dp, dp, ctypes.c_void_p, ctypes.c_int64, dp]
    L.oracle_pose_grad.argtypes = [g, fp, dp, dp, ctypes.c_void_p, dp, ctypes.c_void_p]
    L.oracle_element_gradient_rows.argtypes = [g, fp, dp, dp, ctypes.c_void_p, ctypes.c_int64, dp]
    L.oracle_element_gradient_bounds.argtypes = [g, fp, dp, dp, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_double, dp, dp, ctypes.c_void_p]
    L.oracle_loss.argtypes = [g, dp, dp, ctypes.c_void_p, dp]
    L.oracle_loss.restype = ctypes.c_double
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def make_geom(geom: dict, *, point_sampling: bool = False, vol_pose=None) -> OracleGeom:
    """Pack an acquisition dict (keys as produced by the input generators)."""
    g = OracleGeom()
    for k in ("nx", "ny", "nz", "n_elem", "n_frames", "n_samples"):
        setattr(g, k, int(geom[k]))
    for k in ("dx", "dy", "dz", "ox", "oy", "oz"):
        setattr(g, k, float(geom[k]))
    g.fs, g.t0, g.c, g.a0 = (float(geom["fs_mhz"]), float(geom["t0_us"]),
                             float(geom["c_mm_per_us"]), float(geom["a0_mm"]))
    g.point_sampling = int(point_sampling)
    g.kernel = KERNELS[geom.get("kernel", "sphere")]
    g.sigma = float(geom.get("sigma_mm", 0.0))
    if g.kernel == 1 and not g.sigma > 0:
        raise ValueError("the Gaussian kernel needs sigma_mm > 0")
    vp = np.eye(3, 4) if vol_pose is None else np.asarray(vol_pose, dtype=np.float64)
    for k, v in enumerate(vp.reshape(12)):
        g.vol_pose[k] = float(v)
    return g


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _opt_ptr(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def support(geom) -> float:
    """Half-width (mm) of a voxel's pulse in the distance variable: a0, or 4 sigma."""
    return lib().oracle_support(ctypes.byref(make_geom(geom)))


def pulse(geom, d, n, **kw) -> float:
    """Sample n of a unit voxel's pulse at distance d (mm)."""
    return lib().oracle_pulse(ctypes.byref(make_geom(geom, **kw)), float(d), int(n))


def pulse_dd(geom, d, n, **kw) -> float:
    return lib().oracle_pulse_dd(ctypes.byref(make_geom(geom, **kw)), float(d), int(n))


def element_positions(geom, elem, poses) -> np.ndarray:
    """x[f][j] = R_f e_j + t_f, float64 [F][E][3]."""
    F, E = int(geom["n_frames"]), int(geom["n_elem"])
    out = np.zeros((F, E, 3))
    lib().oracle_element_positions(ctypes.byref(make_geom(geom)), _f64(elem), _f64(poses), out)
    return out


def check_geometry(geom, xw, **kw) -> int:
    return int(lib().oracle_check_geometry(ctypes.byref(make_geom(geom, **kw)), _f64(xw)))


def forward(geom, p0, xw, rows=None, **kw) -> np.ndarray:
    """Signals [F][E][Nt] (or [len(rows)][Nt] for flat (f*E + j) row indices)."""
    g = make_geom(geom, **kw)
    p0 = np.ascontiguousarray(p0, dtype=np.float32)
    F, E, T = int(geom["n_frames"]), int(geom["n_elem"]), int(geom["n_samples"])
    if rows is None:
        out = np.zeros((F, E, T))
        lib().oracle_forward_rows(ctypes.byref(g), p0, _f64(xw), None, 0, out)
        return out
    r, rp = _opt_ptr(rows, np.int64)
    out = np.zeros((len(r), T))
    lib().oracle_forward_rows(ctypes.byref(g), p0, _f64(xw), rp, len(r), out)
    return out


def adjoint(geom, gsig, xw, voxels=None, **kw) -> np.ndarray:
    """Back-projection [nz][ny][nx] (or [len(voxels)] for flat voxel indices)."""
    g = make_geom(geom, **kw)
    gs = _f64(gsig)
    if voxels is None:
        out = np.zeros((int(geom["nz"]), int(geom["ny"]), int(geom["nx"])))
        lib().oracle_adjoint_voxels(ctypes.byref(g), gs, _f64(xw), None, 0, out)
        return out
    v, vp = _opt_ptr(voxels, np.int64)
    out = np.zeros(len(v))
    lib().oracle_adjoint_voxels(ctypes.byref(g), gs, _f64(xw), vp, len(v), out)
    return out


def pose_grad(geom, p0, gsig, xw, mask=None, **kw):
    """Returns (grad6 [F][6] ordered (w, v), G [F][E][3])."""
    g = make_geom(geom, **kw)
    F, E = int(geom["n_frames"]), int(geom["n_elem"])
    grad6 = np.zeros((F, 6))
    G = np.zeros((F, E, 3))
    m, mp = _opt_ptr(mask, np.uint8)
    lib().oracle_pose_grad(ctypes.byref(g), np.ascontiguousarray(p0, dtype=np.float32),
                           _f64(gsig), _f64(xw), mp, grad6, G.ctypes.data_as(ctypes.c_void_p))
    return grad6, G


def element_gradient_rows(geom, p0, gsig, xw, rows):
    """Element-position gradients [len(rows)][3] for flat (f*E + j) row indices."""
    g = make_geom(geom)
    r, rp = _opt_ptr(rows, np.int64)
    out = np.zeros((len(r), 3))
    lib().oracle_element_gradient_rows(ctypes.byref(g), np.ascontiguousarray(p0, dtype=np.float32),
                                       _f64(gsig), _f64(xw), rp, len(r), out)
    return out


def element_gradient_bounds(geom, p0, gsig, xw, rows, eps, counts=False):
    """(Gmid, Ghalf) [len(rows)][3]: every one-sided choice of the derivative at
    support-edge boundaries within eps mm of +-a0 lies in Gmid +- Ghalf.  With
    ``counts`` also the number of such boundaries per row that carry a nonzero
    term (0: the row's gradient is the strict one whatever side is taken)."""
    g = make_geom(geom)
    r, rp = _opt_ptr(rows, np.int64)
    mid = np.zeros((len(r), 3))
    half = np.zeros((len(r), 3))
    n = np.zeros(len(r), dtype=np.int64)
    lib().oracle_element_gradient_bounds(ctypes.byref(g), np.ascontiguousarray(p0, dtype=np.float32),
                                         _f64(gsig), _f64(xw), rp, len(r), float(eps), mid, half,
                                         n.ctypes.data_as(ctypes.c_void_p))
    return (mid, half, n) if counts else (mid, half)


def loss(geom, sig, meas, mask=None):
    """Returns (L, g) with g = mask (s - S) and L = 1/2 sum g^2."""
    g = make_geom(geom)
    out = np.zeros(np.shape(sig))
    m, mp = _opt_ptr(mask, np.uint8)
    L = lib().oracle_loss(ctypes.byref(g), _f64(sig), _f64(meas), mp, out)
    return L, out


def threads_used() -> int:
    """OpenMP threads the oracle runs with (OMP_NUM_THREADS, else all cores)."""
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env else os.cpu_count() or 1
