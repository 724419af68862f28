"""ctypes binding of the C-ABI in ``include/matvis.h`` (argument marshalling only).

Every step of the simulation runs in the CUDA library.  Output V lands in a
torch CUDA tensor (complex64 ``[n_t, n_nu, N, N]``) or, with ``host=True``,
in a numpy array written by the library's device-to-host copy.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmatvis_gb300.so")

MV_OK = 0
_STATUS = {0: "MV_OK", 1: "MV_ERR_ARG", 2: "MV_ERR_OOM", 3: "MV_ERR_CUDA", 4: "MV_ERR_STATE",
           5: "MV_ERR_DEVICE_TIMEOUT", 6: "MV_ERR_UNSUPPORTED"}
PRECISION = {"fp32": 0, "fp16x3": 2}
_CUDA_STREAM_LEGACY = 0x1
INTERP = {"cubic": 0, "bilinear": 1}

# exported symbols of include/matvis.h
EXPORTS = ["mv_default_options", "mv_create", "mv_destroy", "mv_last_error", "mv_init_sky",
           "mv_set_beam_gaussian", "mv_set_beam_grid", "mv_set_antennas", "mv_simulate",
           "mv_simulate_pairs", "mv_check_device_status", "mv_last_live_counts", "mv_last_launch_count",
           "mv_profile_enable", "mv_profile_read", "mv_horizon_cull_static", "mv_autotune",
           "mv_default_mlp_config", "mv_surrogate_create", "mv_surrogate_train", "mv_surrogate_params",
           "mv_surrogate_set_params", "mv_surrogate_eval", "mv_surrogate_grad", "mv_surrogate_save",
           "mv_surrogate_load", "mv_set_beam_surrogate", "mv_set_sky_polarisation", "mv_redundancy_plan",
           "mv_set_redundancy", "mv_simulate_unique", "mv_selftest_wait_timeout", "mv_perturb_sky",
           "mv_beam_model_bytes"]
KERNEL_KINDS = {"cull": 0, "beam": 1, "zbuild": 2, "herk": 3}


class MatvisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("user", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("interp", ctypes.c_int), ("max_batch", ctypes.c_int), ("herk_flush_kblocks", ctypes.c_int),
                ("herk_split", ctypes.c_int), ("allocator", _Allocator), ("herk_tile_n", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("overlap_batches", ctypes.c_int), ("fuse_zbuild", ctypes.c_int)]


class _MlpConfig(ctypes.Structure):
    _fields_ = [("n_freq", ctypes.c_int), ("emb_dim", ctypes.c_int), ("width", ctypes.c_int), ("depth", ctypes.c_int),
                ("sigma_az", ctypes.c_float), ("sigma_za", ctypes.c_float), ("sigma_nu", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("tile_n", ctypes.c_int), ("split", ctypes.c_int), ("flush_kblocks", ctypes.c_int),
                ("candidates", ctypes.c_int), ("herk_ms", ctypes.c_double), ("fused", ctypes.c_int)]


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2312_09763_gb300._build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.mv_default_options.argtypes = [ctypes.POINTER(_Options)]
    lib.mv_default_options.restype = None
    lib.mv_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(_Options)]
    lib.mv_destroy.argtypes = [vp]
    lib.mv_destroy.restype = None
    lib.mv_last_error.restype = ctypes.c_char_p
    lib.mv_last_error.argtypes = []
    lib.mv_init_sky.argtypes = [vp, i64, vp, vp, vp, vp, dp]
    lib.mv_set_sky_polarisation.argtypes = [vp, i64, vp, vp, vp]
    lib.mv_set_beam_gaussian.argtypes = [vp, dp]
    lib.mv_set_beam_grid.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp, dp, dp, dp, dp]
    lib.mv_set_antennas.argtypes = [vp, i32, vp, vp, dp]
    lib.mv_simulate.argtypes = [vp, i32, vp, i32, vp, i32, vp, i32, vp]
    lib.mv_simulate_pairs.argtypes = [vp, i32, vp, vp, i32, vp, i32, vp]
    lib.mv_check_device_status.argtypes = [vp, vp]
    lib.mv_last_live_counts.argtypes = [vp, i32, vp]
    lib.mv_last_launch_count.argtypes = [vp]
    lib.mv_last_launch_count.restype = i64
    lib.mv_profile_enable.argtypes = [vp, i32]
    lib.mv_profile_read.argtypes = [vp, i32, vp, vp]
    lib.mv_horizon_cull_static.argtypes = [i64, vp, dp, dp, vp, vp, vp, vp, vp]
    lib.mv_horizon_cull_static.restype = i32
    lib.mv_autotune.argtypes = [vp, i32, vp, i32, vp, i32, i32, vp]
    lib.mv_autotune.restype = i32
    lib.mv_default_mlp_config.argtypes = [ctypes.POINTER(_MlpConfig)]
    lib.mv_default_mlp_config.restype = None
    lib.mv_surrogate_create.argtypes = [vp, ctypes.POINTER(_MlpConfig)]
    lib.mv_surrogate_train.argtypes = [vp, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_uint64, vp, vp]
    lib.mv_surrogate_params.argtypes = [vp, vp, vp, vp, vp]
    lib.mv_surrogate_set_params.argtypes = [vp, vp]
    lib.mv_surrogate_eval.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.mv_surrogate_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.mv_surrogate_save.argtypes = [vp, ctypes.c_char_p]
    lib.mv_surrogate_load.argtypes = [vp, ctypes.c_char_p]
    lib.mv_set_beam_surrogate.argtypes = [vp, i32]
    lib.mv_beam_model_bytes.argtypes = [vp, vp, vp]
    lib.mv_redundancy_plan.argtypes = [i32, vp, vp, dp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.mv_redundancy_plan.restype = i32
    lib.mv_perturb_sky.argtypes = [i64, vp, vp, dp, dp, vp, vp]
    lib.mv_perturb_sky.restype = i32
    lib.mv_set_redundancy.argtypes = [vp, dp, vp]
    lib.mv_set_redundancy.restype = i32
    lib.mv_simulate_unique.argtypes = [vp, i32, vp, i32, vp, i32, vp, i32, vp]
    lib.mv_simulate_unique.restype = i32
    lib.mv_selftest_wait_timeout.argtypes = [vp, dp]
    lib.mv_selftest_wait_timeout.restype = i32
    for name in ("mv_surrogate_create", "mv_surrogate_train", "mv_surrogate_params", "mv_surrogate_set_params",
                 "mv_surrogate_eval", "mv_surrogate_grad", "mv_surrogate_save", "mv_surrogate_load",
                 "mv_set_beam_surrogate"):
        getattr(lib, name).restype = i32
    for name in ("mv_create", "mv_init_sky", "mv_set_beam_gaussian", "mv_set_beam_grid", "mv_set_antennas",
                 "mv_simulate", "mv_simulate_pairs", "mv_check_device_status", "mv_last_live_counts",
                 "mv_profile_enable", "mv_profile_read"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def redundancy_plan(enu, beam_idx=None, tol_m: float = 1e-3, n_feed: int = 1, tile_n: int = 256) -> dict:
    """Redundant-baseline groups of an array and the cover of their
    representatives (mv_redundancy_plan; host only, no GPU needed)."""
    lib = load_library()
    enu = _f64(enu).reshape(-1, 3)
    n = enu.shape[0]
    nbl = n * (n + 1) // 2
    bi = None if beam_idx is None else np.ascontiguousarray(np.asarray(beam_idx, dtype=np.int32))
    nu, kind, nb = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    ra, rb, go = (np.zeros(nbl, np.int32) for _ in range(3))
    co = np.zeros(nbl, np.int8)
    perm = np.zeros(n, np.int32)
    blocks = np.zeros(16, np.int32)
    tiles = np.zeros(2, np.int64)
    st = lib.mv_redundancy_plan(n, _p(enu), _p(bi), float(tol_m), n_feed, tile_n, ctypes.byref(nu), _p(ra), _p(rb),
                                _p(go), _p(co), _p(perm), ctypes.byref(kind), ctypes.byref(nb), _p(blocks), _p(tiles))
    if st != 0:
        raise MatvisError(st, lib.mv_last_error().decode())
    k = nu.value
    return {"n_unique": k, "rep_a": ra[:k].copy(), "rep_b": rb[:k].copy(), "group_of": go, "conj_of": co,
            "perm": perm, "kind": kind.value, "blocks": blocks[:4 * nb.value].reshape(-1, 4).copy(),
            "tiles": int(tiles[0]), "tiles_full": int(tiles[1])}


def perturb_sky(alt, az, lst_ref: float, latitude: float):
    """Perturbed (RA', Dec') of Algorithm 1 from apparent (alt, az) at a
    reference LST (mv_perturb_sky; host only, no GPU needed)."""
    lib = load_library()
    alt, az = _f64(alt).ravel(), _f64(az).ravel()
    if alt.size != az.size:
        raise ValueError("alt and az differ in size")
    ra, dec = np.empty(alt.size), np.empty(alt.size)
    st = lib.mv_perturb_sky(alt.size, _p(alt), _p(az), float(lst_ref), float(latitude), _p(ra), _p(dec))
    if st != 0:
        raise MatvisError(st, lib.mv_last_error().decode())
    return ra, dec


class Simulator:
    """One simulator context on one CUDA device (see include/matvis.h)."""

    def __init__(self, device: int = 0, interp: str = "cubic", max_batch: int = 0, herk_flush_kblocks: int = 0,
                 herk_split: int = 0, herk_tile_n: int = 0, use_graph: bool = True, overlap_batches: bool = False,
                 fuse_zbuild: bool = True, torch_allocator: bool = True):
        import torch  # device memory and streams
        self._torch = torch
        self._lib = load_library()
        self.device = device
        opt = _Options()
        self._lib.mv_default_options(ctypes.byref(opt))
        opt.interp = INTERP[interp]
        opt.max_batch = max_batch
        opt.herk_flush_kblocks = herk_flush_kblocks
        opt.herk_split = herk_split
        opt.herk_tile_n = herk_tile_n
        opt.use_graph = 1 if use_graph else 0
        opt.overlap_batches = 1 if overlap_batches else 0
        opt.fuse_zbuild = 1 if fuse_zbuild else 0
        self._cb = None
        if torch_allocator:
            def _alloc(nbytes, dev, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), int(dev), stream or 0)
                except Exception:
                    return None

            def _free(ptr, nbytes, dev, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_ALLOC(_alloc), _FREE(_free))
            opt.allocator.alloc, opt.allocator.free = self._cb
        torch.cuda.init()
        h = ctypes.c_void_p()
        self._check(self._lib.mv_create(ctypes.byref(h), device, ctypes.byref(opt)))
        self._h = h
        self.n_ant = 0
        self.n_feed = 1

    def _check(self, status: int):
        if status != MV_OK:
            raise MatvisError(status, self._lib.mv_last_error().decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- set-up
    def init_sky(self, ra, dec, flux_ref, spec_idx=None, nu_ref: float = 150e6):
        ra, dec, fl = _f64(ra), _f64(dec), _f64(flux_ref)
        si = None if spec_idx is None else _f64(spec_idx)
        self._check(self._lib.mv_init_sky(self._h, ra.size, _p(ra), _p(dec), _p(fl), _p(si), float(nu_ref)))

    def set_sky_polarisation(self, stokes_quv=None):
        """Stokes Q, U, V ([3][n_src], Jy at nu_ref) of the current sky; None = unpolarised."""
        if stokes_quv is None:
            self._check(self._lib.mv_set_sky_polarisation(self._h, 0, None, None, None))
            return
        q = _f64(stokes_quv).reshape(3, -1)
        self._check(self._lib.mv_set_sky_polarisation(self._h, q.shape[1], _p(q[0]), _p(q[1]), _p(q[2])))

    def set_beam_gaussian(self, fwhm: float):
        self._check(self._lib.mv_set_beam_gaussian(self._h, float(fwhm)))
        self.n_feed = 1

    def set_beam_grid(self, values, nu0: float, dnu: float, dza: float, daz: float):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.complex64))
        if v.ndim != 6:
            raise ValueError("values must be [beam][feed][ax][nu][za][az]")
        nb, nf, na, nn, nz, naz = v.shape
        self._check(self._lib.mv_set_beam_grid(self._h, nb, nf, na, nn, nz, naz, _p(v), float(nu0), float(dnu),
                                               float(dza), float(daz)))
        self.n_feed = nf
        self.n_ax = na

    def set_beam(self, beam: tuple):
        """beam = ("gaussian", fwhm) or ("grid", values, nu0, dnu, dza, daz[, interp])."""
        if beam[0] == "gaussian":
            self.set_beam_gaussian(beam[1])
        elif beam[0] == "grid":
            self.set_beam_grid(*beam[1:6])
        else:
            raise ValueError(beam[0])

    def set_antennas(self, enu, beam_idx=None, lat: float = 0.0):
        enu = _f64(enu).reshape(-1, 3)
        bi = None if beam_idx is None else np.ascontiguousarray(beam_idx, dtype=np.int32)
        self._check(self._lib.mv_set_antennas(self._h, enu.shape[0], _p(enu), _p(bi), float(lat)))
        self.n_ant = enu.shape[0]

    # ------------------------------------------------------------ simulate
    def _out(self, shape, out, host):
        torch = self._torch
        if host:
            if out is None:
                out = np.empty(shape, dtype=np.complex64)
            if isinstance(out, np.ndarray):
                assert out.dtype == np.complex64 and out.flags.c_contiguous and out.shape == tuple(shape)
                return out, out.ctypes.data_as(ctypes.c_void_p), 0
            # a (pinned) torch CPU tensor
            assert (not out.is_cuda) and out.dtype == torch.complex64 and out.is_contiguous()
            return out, ctypes.c_void_p(out.data_ptr()), 0
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous()
        return out, ctypes.c_void_p(out.data_ptr()), 1

    def _stream(self, stream):
        torch = self._torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        # torch's default stream is the legacy NULL stream; name it explicitly
        # (cudaStreamLegacy) since NULL means "the context's own stream" here
        return ctypes.c_void_p(stream.cuda_stream or _CUDA_STREAM_LEGACY)

    def simulate(self, lsts: Sequence[float], freqs: Sequence[float], precision: str = "fp16x3", out=None,
                 host: bool = False, stream=None):
        """V[t, f] for every LST and frequency: complex64 [n_t, n_nu, N, N]."""
        lst, nu = _f64(lsts).ravel(), _f64(freqs).ravel()
        N = self.n_feed * self.n_ant
        arr, ptr, on_dev = self._out((lst.size, nu.size, N, N), out, host)
        self._check(self._lib.mv_simulate(self._h, lst.size, _p(lst), nu.size, _p(nu), PRECISION[precision], ptr,
                                          on_dev, None if host else self._stream(stream)))
        return arr

    def simulate_pairs(self, lsts, freqs, precision: str = "fp16x3", out=None, host: bool = False, stream=None):
        """V for explicit (lst, nu) pairs: complex64 [n_pairs, N, N]."""
        lst, nu = _f64(lsts).ravel(), _f64(freqs).ravel()
        if lst.size != nu.size:
            raise ValueError("lsts and freqs must have the same length")
        N = self.n_feed * self.n_ant
        arr, ptr, on_dev = self._out((lst.size, N, N), out, host)
        self._check(self._lib.mv_simulate_pairs(self._h, lst.size, _p(lst), _p(nu), PRECISION[precision], ptr,
                                                on_dev, None if host else self._stream(stream)))
        return arr

    def set_redundancy(self, tol_m: float = 1e-3) -> int:
        """Plan the redundant-group output for the current antennas and beam
        (mv_set_redundancy); returns the number of groups.  tol_m <= 0: off."""
        n = ctypes.c_int64(0)
        self._check(self._lib.mv_set_redundancy(self._h, float(tol_m), ctypes.byref(n)))
        self.n_unique = int(n.value)
        return self.n_unique

    def simulate_unique(self, lsts, freqs, precision: str = "fp16x3", out=None, host: bool = False, stream=None):
        """One value per redundant group: complex64 [n_t, n_nu, n_unique, n_feed, n_feed]."""
        lst, nu = _f64(lsts).ravel(), _f64(freqs).ravel()
        shape = (lst.size, nu.size, self.n_unique, self.n_feed, self.n_feed)
        arr, ptr, on_dev = self._out(shape, out, host)
        self._check(self._lib.mv_simulate_unique(self._h, lst.size, _p(lst), nu.size, _p(nu), PRECISION[precision],
                                                 ptr, on_dev, None if host else self._stream(stream)))
        return arr

    def selftest_wait_timeout(self, limit_s: float = 0.2) -> str:
        """Run the failure-path self-test (mv_selftest_wait_timeout); returns the
        status name it reports (MV_ERR_DEVICE_TIMEOUT when the bounded wait
        gave up as designed)."""
        return _STATUS.get(self._lib.mv_selftest_wait_timeout(self._h, float(limit_s)), "?")

    def check_device_status(self, stream=None):
        self._check(self._lib.mv_check_device_status(self._h, None if stream is None else self._stream(stream)))

    def last_live_counts(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.int64)
        self._check(self._lib.mv_last_live_counts(self._h, n, _p(out)))
        return out

    def last_launch_count(self) -> int:
        return int(self._lib.mv_last_launch_count(self._h))

    def autotune(self, lsts, freqs, precision: str = "fp16x3", pairs: bool = False) -> dict:
        """Time the tensor-core HERK configurations on the first batch of this
        call shape and keep the fastest (see mv_autotune)."""
        lst, nu = _f64(lsts).ravel(), _f64(freqs).ravel()
        t = _Tuning()
        self._check(self._lib.mv_autotune(self._h, lst.size, _p(lst), nu.size, _p(nu), PRECISION[precision],
                                          1 if pairs else 0, ctypes.byref(t)))
        return {"tile_n": t.tile_n, "split": t.split, "flush_kblocks": t.flush_kblocks,
                "candidates": t.candidates, "herk_ms": t.herk_ms, "fused": bool(t.fused)}

    # --------------------------------------------------------- learned beam
    def surrogate_create(self, n_freq=64, emb_dim=16, width=256, depth=4, sigma_az=2.0, sigma_za=3.0, sigma_nu=1.0,
                         seed=20231213):
        """Fourier-feature MLP standing in for the current gridded beams."""
        c = _MlpConfig(n_freq, emb_dim, width, depth, sigma_az, sigma_za, sigma_nu, seed)
        self._check(self._lib.mv_surrogate_create(self._h, ctypes.byref(c)))
        self._mlp = dict(n_freq=n_freq, emb_dim=emb_dim, width=width, depth=depth)

    def surrogate_train(self, steps: int, batch: int, lr0: float = 1e-3, lr1: float = 1e-5, seed: int = 1):
        """Adam on samples labelled by the gridded beams; returns (first, last) loss."""
        l0, l1 = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.mv_surrogate_train(self._h, steps, batch, lr0, lr1, seed, ctypes.byref(l0),
                                                 ctypes.byref(l1)))
        return l0.value, l1.value

    def surrogate_params(self):
        """(FP32 parameter vector, Fourier matrix [F][3], layout offsets)."""
        n = ctypes.c_int64()
        self._check(self._lib.mv_surrogate_params(self._h, ctypes.byref(n), None, None, None))
        p = np.empty(n.value, dtype=np.float32)
        B = np.empty((self._mlp["n_freq"], 3), dtype=np.float32)
        lay = np.empty(2 * (self._mlp["depth"] + 1) + 2, dtype=np.int64)
        self._check(self._lib.mv_surrogate_params(self._h, ctypes.byref(n), _p(p), _p(B), _p(lay)))
        return p, B, lay

    def surrogate_set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.mv_surrogate_set_params(self._h, _p(p)))

    def surrogate_eval(self, beam, az, za, nu):
        beam = np.ascontiguousarray(beam, dtype=np.int32)
        az, za, nu = _f64(az), _f64(za), _f64(nu)
        out = np.empty((beam.size, 2 * self.n_feed * self._n_ax()), dtype=np.float32)
        self._check(self._lib.mv_surrogate_eval(self._h, beam.size, _p(beam), _p(az), _p(za), _p(nu), _p(out)))
        return out

    def surrogate_grad(self, beam, az, za, nu, target):
        """(gradient of every parameter, loss) for given samples; no update."""
        beam = np.ascontiguousarray(beam, dtype=np.int32)
        az, za, nu = _f64(az), _f64(za), _f64(nu)
        t = np.ascontiguousarray(target, dtype=np.float32)
        n = ctypes.c_int64()
        self._check(self._lib.mv_surrogate_params(self._h, ctypes.byref(n), None, None, None))
        g = np.empty(n.value, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.mv_surrogate_grad(self._h, beam.size, _p(beam), _p(az), _p(za), _p(nu), _p(t), _p(g),
                                                ctypes.byref(loss)))
        return g, loss.value

    def surrogate_save(self, path: str):
        self._check(self._lib.mv_surrogate_save(self._h, str(path).encode()))

    def surrogate_load(self, path: str, **cfg):
        self._check(self._lib.mv_surrogate_load(self._h, str(path).encode()))
        if cfg:
            self._mlp = dict(cfg)

    def set_beam_surrogate(self, enable: bool = True):
        self._check(self._lib.mv_set_beam_surrogate(self._h, 1 if enable else 0))

    def beam_model_bytes(self):
        """(device bytes of the gridded beams as held, device bytes the surrogate's evaluation reads)."""
        g, m = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.mv_beam_model_bytes(self._h, ctypes.byref(g), ctypes.byref(m)))
        return g.value, m.value

    def _n_ax(self) -> int:
        return getattr(self, "n_ax", 1)

    def profile_enable(self, enable: bool = True):
        """Time every kernel launch with CUDA events (clears the counters)."""
        self._check(self._lib.mv_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kind: (launches, total_ms)} for cull, beam, zbuild, herk."""
        out = {}
        for name, k in KERNEL_KINDS.items():
            n, ms = ctypes.c_int64(), ctypes.c_double()
            self._check(self._lib.mv_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (int(n.value), float(ms.value))
        return out
