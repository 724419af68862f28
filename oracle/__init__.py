"""FP64 CPU oracle for the matvis visibility simulator (arXiv:2312.09763).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2312_09763_gb300`` and never imports it.

The arithmetic lives in ``matvis_oracle.c`` (plain C, IEEE double, compiled
with ``-ffp-contract=off``); this module only marshals numpy arrays into it.
Functions and the passages they follow:

* :func:`xeq`            -- eq. "xeq", Sec. 2.3
* :func:`rotation`       -- eq. "rotation", Sec. 2.3 (read with H = -LST)
* :func:`to_topo`        -- X_hrz = R X_eq, Sec. 2.3
* :func:`azza`           -- az = atan2(E, N), za = acos(Up) (reading; Sec. 2.4
  needs a spherical grid with the zenith as its pole)
* :func:`keys`           -- Keys (1981) cubic-convolution kernel, a = -1/2
* :func:`beam_eval`      -- analytic / gridded beams, Sec. 2.4
* :func:`count_live`     -- horizon cut of Algorithm 2 step (i)
* :func:`vis`            -- direct per-baseline sum: eq. "matvisrime" with the
  delay of eq. "matvisdelay" and C = I * identity (Sec. 2.2)
* :func:`vis_outer`      -- Z of eq. "littlez" and V = Z Z^dagger of eq. "zz"
  (Algorithm 2 steps iii-v), a small-problem cross-check of :func:`vis`
* :func:`perturb_sky`    -- Algorithm 1 (Sec. 2.3) steps (ii), (iv)-(vi):
  perturbed RA/Dec from apparent (alt, az) at a reference LST
* :func:`vis_with_beam_fn` -- :func:`vis` with the beams of a caller's model
  tabulated at the live sources (the learned beam's checker)

Parity status: pinned by closed forms and invariants only (the paper prints no
numeric visibilities); see tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "matvis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

C_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the C source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_src", ctypes.c_int64),
        ("ra", ctypes.c_void_p), ("dec", ctypes.c_void_p),
        ("flux_ref", ctypes.c_void_p), ("spec_idx", ctypes.c_void_p),
        ("nu_ref", ctypes.c_double),
        ("n_ant", ctypes.c_int32),
        ("enu", ctypes.c_void_p), ("beam_idx", ctypes.c_void_p),
        ("lat", ctypes.c_double),
        ("beam_kind", ctypes.c_int32), ("fwhm", ctypes.c_double),
        ("n_beam", ctypes.c_int32), ("n_feed", ctypes.c_int32), ("n_ax", ctypes.c_int32),
        ("n_nu", ctypes.c_int32), ("n_za", ctypes.c_int32), ("n_az", ctypes.c_int32),
        ("grid", ctypes.c_void_p),
        ("nu0", ctypes.c_double), ("dnu", ctypes.c_double),
        ("dza", ctypes.c_double), ("daz", ctypes.c_double),
        ("interp", ctypes.c_int32),
        ("stokes_quv", ctypes.c_void_p),
    ]


_lib: Optional[ctypes.CDLL] = None


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.c_void_p
        lib.orc_xeq.argtypes = [ctypes.c_int64, dp, dp, dp]
        lib.orc_rotation.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        lib.orc_to_topo.argtypes = [dp, ctypes.c_int64, dp, dp]
        lib.orc_azza.argtypes = [ctypes.c_int64, dp, dp, dp]
        lib.orc_keys.argtypes = [ctypes.c_double]
        lib.orc_keys.restype = ctypes.c_double
        lib.orc_beam_eval_many.argtypes = [P, ctypes.c_int64, dp, dp, ctypes.c_double, dp]
        lib.orc_beam_eval_many.restype = ctypes.c_int
        lib.orc_count_live.argtypes = [P, ctypes.c_double]
        lib.orc_count_live.restype = ctypes.c_int64
        lib.orc_vis.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                dp, dp, dp, ctypes.c_int]
        lib.orc_vis.restype = ctypes.c_int
        lib.orc_vis_outer.argtypes = [P, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_vis_outer.restype = ctypes.c_int
        lib.orc_coherency_sqrt.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.orc_coherency_sqrt.restype = None
        lib.orc_perturb_sky.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_perturb_sky.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Problem:
    """Inputs of one simulation (Sec. 3.1 input list), in FP64.

    beam: ``("uniform",)``, ``("gaussian", fwhm_rad)`` or
    ``("grid", values, nu0, dnu, dza, daz, interp)`` with ``values`` complex
    ``[beam][feed][ax][nu][za][az]`` and ``interp`` "cubic" | "bilinear".
    """
    ra: np.ndarray
    dec: np.ndarray
    flux_ref: np.ndarray
    enu: np.ndarray
    lat: float
    beam: tuple
    spec_idx: Optional[np.ndarray] = None
    nu_ref: float = 150e6
    beam_idx: Optional[np.ndarray] = None
    stokes_quv: Optional[np.ndarray] = None   # [3][n_src] Q, U, V (Jy at nu_ref); needs a two-axis beam
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Problem:
        ra, dec, fl = _f64(self.ra), _f64(self.dec), _f64(self.flux_ref)
        si = None if self.spec_idx is None else _f64(self.spec_idx)
        enu = _f64(self.enu).reshape(-1, 3)
        bi = None if self.beam_idx is None else np.ascontiguousarray(self.beam_idx, dtype=np.int32)
        quv = None if self.stokes_quv is None else _f64(self.stokes_quv).reshape(3, -1)
        keep = [ra, dec, fl, si, enu, bi, quv]
        p = _Problem()
        p.stokes_quv = _ptr(quv)
        p.n_src = ra.size
        p.ra, p.dec, p.flux_ref, p.spec_idx = _ptr(ra), _ptr(dec), _ptr(fl), _ptr(si)
        p.nu_ref = float(self.nu_ref)
        p.n_ant = enu.shape[0]
        p.enu, p.beam_idx = _ptr(enu), _ptr(bi)
        p.lat = float(self.lat)
        kind = self.beam[0]
        p.n_beam, p.n_feed, p.n_ax = 1, 1, 1
        if kind == "uniform":
            p.beam_kind = 0
        elif kind == "gaussian":
            p.beam_kind = 1
            p.fwhm = float(self.beam[1])
        elif kind == "grid":
            vals, nu0, dnu, dza, daz, interp = self.beam[1:7]
            g = np.ascontiguousarray(np.asarray(vals, dtype=np.complex128))
            assert g.ndim == 6
            keep.append(g)
            p.beam_kind = 2
            p.n_beam, p.n_feed, p.n_ax, p.n_nu, p.n_za, p.n_az = g.shape
            p.grid = _ptr(g)
            p.nu0, p.dnu, p.dza, p.daz = float(nu0), float(dnu), float(dza), float(daz)
            p.interp = {"cubic": 0, "bilinear": 1}[interp]
        elif kind == "table":
            # caller-evaluated beams at the live sources: complex [beam][feed][ax][n_live]
            g = np.ascontiguousarray(np.asarray(self.beam[1], dtype=np.complex128))
            assert g.ndim == 4
            keep.append(g)
            p.beam_kind = 3
            p.n_beam, p.n_feed, p.n_ax = g.shape[:3]
            p.grid = _ptr(g)
        else:
            raise ValueError(kind)
        self._keep = keep
        return p

    @property
    def n_feed(self) -> int:
        return self.beam[1].shape[1] if self.beam[0] == "grid" else 1


def xeq(ra, dec) -> np.ndarray:
    """eq. "xeq": Cartesian equatorial unit vectors, shape [n, 3]."""
    ra, dec = _f64(ra), _f64(dec)
    out = np.empty((ra.size, 3))
    _load().orc_xeq(ra.size, _ptr(ra), _ptr(dec), _ptr(out))
    return out


def rotation(lst: float, lat: float) -> np.ndarray:
    """eq. "rotation" with H = -LST: 3x3 equatorial -> ENU matrix."""
    R = np.empty(9)
    _load().orc_rotation(float(lst), float(lat), _ptr(R))
    return R.reshape(3, 3)


def to_topo(R, xyz) -> np.ndarray:
    R, xyz = _f64(R).reshape(9), _f64(xyz).reshape(-1, 3)
    out = np.empty_like(xyz)
    _load().orc_to_topo(_ptr(R), xyz.shape[0], _ptr(xyz), _ptr(out))
    return out


def azza(enu):
    enu = _f64(enu).reshape(-1, 3)
    az, za = np.empty(enu.shape[0]), np.empty(enu.shape[0])
    _load().orc_azza(enu.shape[0], _ptr(enu), _ptr(az), _ptr(za))
    return az, za


def keys(x: float) -> float:
    return _load().orc_keys(float(x))


def beam_eval(prob: Problem, az, za, nu: float) -> np.ndarray:
    """Beam components at directions: complex128 [beam][feed][ax][n]."""
    az, za = _f64(az), _f64(za)
    p = prob.c()
    nb = p.n_beam if p.beam_kind == 2 else 1
    out = np.empty((nb, p.n_feed, p.n_ax, az.size), dtype=np.complex128)
    rc = _load().orc_beam_eval_many(ctypes.byref(p), az.size, _ptr(az), _ptr(za), float(nu), _ptr(out))
    if rc:
        raise ValueError("frequency outside the beam grid")
    return out


def count_live(prob: Problem, lst: float) -> int:
    p = prob.c()
    return int(_load().orc_count_live(ctypes.byref(p), float(lst)))


def vis(prob: Problem, lst: float, nu: float, pairs=None, threads: Optional[int] = None) -> np.ndarray:
    """Direct per-baseline sum.

    pairs=None: full complex128 [N][N] with N = n_feed * n_ant.
    pairs=(a, b) index arrays: complex128 [n_pairs][n_feed][n_feed].
    """
    p = prob.c()
    nfd = p.n_feed
    nt = threads or os.cpu_count() or 1
    if pairs is None:
        out = np.empty((nfd * p.n_ant, nfd * p.n_ant), dtype=np.complex128)
        rc = _load().orc_vis(ctypes.byref(p), float(lst), float(nu), -1, None, None, _ptr(out), nt)
    else:
        pa = np.ascontiguousarray(pairs[0], dtype=np.int32)
        pb = np.ascontiguousarray(pairs[1], dtype=np.int32)
        out = np.empty((pa.size, nfd, nfd), dtype=np.complex128)
        rc = _load().orc_vis(ctypes.byref(p), float(lst), float(nu), pa.size, _ptr(pa), _ptr(pb), _ptr(out), nt)
    _raise(rc)
    return out


def _raise(rc: int):
    if rc == -1:
        raise ValueError("frequency outside the beam grid")
    if rc == -2:
        raise ValueError("bad antenna index")
    if rc == -3:
        raise ValueError("a polarised sky needs a two-axis beam")
    if rc:
        raise ValueError(f"oracle error {rc}")


def vis_outer(prob: Problem, lst: float, nu: float) -> np.ndarray:
    """Outer-product form Z Z^dagger in FP64 (small problems only)."""
    p = prob.c()
    N = p.n_feed * p.n_ant
    out = np.empty((N, N), dtype=np.complex128)
    rc = _load().orc_vis_outer(ctypes.byref(p), float(lst), float(nu), _ptr(out))
    _raise(rc)
    return out


def coherency_sqrt(I, Q, U, V) -> np.ndarray:
    """M with M M^dagger = C = [[I+Q, U+iV], [U-iV, I-Q]] (lower-triangular), complex [2][2]."""
    m = np.empty(4)
    _load().orc_coherency_sqrt(float(I), float(Q), float(U), float(V), _ptr(m))
    return np.array([[m[0], 0.0], [m[1] + 1j * m[2], m[3]]])


def live_directions(prob: Problem, lst: float):
    """(az, za) of the live sources (Up > 0), in catalogue order."""
    enu = to_topo(rotation(lst, prob.lat), xeq(prob.ra, prob.dec))
    live = enu[:, 2] > 0
    return azza(enu[live])


def vis_with_beam_fn(prob: Problem, lst: float, nu: float, beam_fn, pairs=None, threads=None) -> np.ndarray:
    """Direct per-baseline sum with the beams given by a caller's model:
    beam_fn(az, za, nu) -> complex [beam][feed][ax][n] at the live sources."""
    az, za = live_directions(prob, lst)
    table = np.asarray(beam_fn(az, za, nu), dtype=np.complex128)
    q = Problem(ra=prob.ra, dec=prob.dec, flux_ref=prob.flux_ref, enu=prob.enu, lat=prob.lat,
                beam=("table", table), spec_idx=prob.spec_idx, nu_ref=prob.nu_ref, beam_idx=prob.beam_idx,
                stokes_quv=prob.stokes_quv)
    return vis(q, lst, nu, pairs=pairs, threads=threads)


def perturb_sky(alt, az, lst_ref: float, lat: float):
    """Algorithm 1 steps (ii), (iv)-(vi): (RA', Dec') such that the rigid
    rotation at lst_ref puts each source at the given apparent (alt, az)."""
    alt, az = _f64(alt).ravel(), _f64(az).ravel()
    ra, dec = np.empty(alt.size), np.empty(alt.size)
    _load().orc_perturb_sky(alt.size, _ptr(alt), _ptr(az), float(lst_ref), float(lat), _ptr(ra), _ptr(dec))
    return ra, dec
