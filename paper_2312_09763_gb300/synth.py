"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random inputs only: antenna layouts, source catalogues,
beam grids, LST and frequency lists.  It holds none of the simulator's
arithmetic, imports nothing else from this package, and feeds the same arrays
to the CUDA path and to the FP64 oracle.

Every quantity draws from its own stream, keyed by (20231209 + a per-workload
offset, quantity name), so that changing one quantity never shifts another.

The paper's own inputs (a GLEAM-like catalogue, the GSM, the CST HERA beam;
Sec. 5.1) are not available; these stand in for them with the counts, flux
distributions and beam widths of the workloads below.

Workloads (all angles in radians, frequencies in Hz, lengths in metres):

* tiny: 10 antennas uniform in a 50 m square (Up = 0); 1000 sources uniform on
   the sphere, dN/dS ~ S^-1.6 on [0.1, 10] Jy, flat spectra; 1 channel at
   150 MHz; 4 LSTs spanning 10 min; latitude -30.7 deg; analytic Gaussian
   E-field beam, FWHM 10 deg.
* HERA-like: 350 antennas, the triangular-lattice points (14.6 m spacing)
   nearest the origin; 1e5 sources uniform on the sphere, dN/dS ~ S^-1.6 on
   [0.01, 100] Jy, spectral index ~ N(-0.8, 0.2) about 150 MHz; 64 channels
   centred in 100-200 MHz; 60 LSTs one minute apart; scalar gridded beam on a
   1 deg x 1 deg az/za grid and a 1 MHz frequency grid (98-202 MHz), a
   Gaussian with FWHM 10 deg x (150 MHz / nu) times (1 + 0.05 r), r a seeded
   smooth ripple with |r| <= 1.
"""
from __future__ import annotations

import zlib
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 20231209
DEG = np.pi / 180.0
SIDEREAL_MINUTE = 2.0 * np.pi / 1440.0  # radians of LST per minute of sidereal time
HERA_LAT = -30.7 * DEG


def rng(workload: int, quantity: str) -> np.random.Generator:
    """Independent generator for one quantity of one workload."""
    key = zlib.crc32(quantity.encode("utf-8"))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE + workload, key])))


# ------------------------------------------------------------------ arrays

def square_array(n: int, side: float, g: np.random.Generator) -> np.ndarray:
    """n antennas uniform in a side x side square about the origin, Up = 0."""
    enu = np.zeros((n, 3))
    enu[:, :2] = g.uniform(-side / 2, side / 2, size=(n, 2))
    return enu


def hex_array(n: int, spacing: float) -> np.ndarray:
    """The n points of a triangular lattice nearest the origin (ties broken by
    angle), Up = 0.  A HERA-like compact, highly redundant layout."""
    r = int(np.ceil(np.sqrt(n))) + 2
    i, j = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    e = spacing * (i + 0.5 * j)
    no = spacing * (np.sqrt(3.0) / 2.0) * j
    e, no = e.ravel(), no.ravel()
    rad = np.round(np.hypot(e, no) / spacing, 9)
    ang = np.round(np.mod(np.arctan2(no, e), 2 * np.pi), 9)
    order = np.lexsort((ang, rad))[:n]
    enu = np.zeros((n, 3))
    enu[:, 0], enu[:, 1] = e[order], no[order]
    return enu


# ------------------------------------------------------------------- skies

def uniform_sphere(n: int, g: np.random.Generator):
    """(ra, dec) uniform on the sphere."""
    ra = g.uniform(0.0, 2.0 * np.pi, size=n)
    dec = np.arcsin(g.uniform(-1.0, 1.0, size=n))
    return ra, dec


def vmf_cluster(n: int, kappa: float, ra0: float, dec0: float, g: np.random.Generator):
    """(ra, dec) drawn from a von Mises-Fisher distribution on the sphere about
    (ra0, dec0) with concentration kappa (Wood 1994: the cosine of the angle
    to the mean direction by inverse CDF, the azimuth about it uniform)."""
    mu = np.array([np.cos(ra0) * np.cos(dec0), np.sin(ra0) * np.cos(dec0), np.sin(dec0)])
    u = g.uniform(0.0, 1.0, n)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    phi = g.uniform(0.0, 2.0 * np.pi, n)
    a = np.cross(mu, [0.0, 0.0, 1.0])
    a /= np.linalg.norm(a)
    b = np.cross(mu, a)
    s = np.sqrt(np.maximum(0.0, 1.0 - w * w))
    v = w[:, None] * mu + s[:, None] * (np.cos(phi)[:, None] * a + np.sin(phi)[:, None] * b)
    return np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * np.pi), np.arcsin(np.clip(v[:, 2], -1.0, 1.0))


def powerlaw_flux(n: int, smin: float, smax: float, gamma: float, g: np.random.Generator) -> np.ndarray:
    """Fluxes with dN/dS ~ S^-gamma on [smin, smax] (inverse CDF)."""
    a, b = smin ** (1.0 - gamma), smax ** (1.0 - gamma)
    u = g.uniform(0.0, 1.0, size=n)
    return (a + u * (b - a)) ** (1.0 / (1.0 - gamma))


# ------------------------------------------------------------------- beams

def ripple_field(az, za, nu_norm, g: np.random.Generator, n_terms: int = 8):
    """Seeded smooth ripple r(az, za, nu) with |r| <= 1.

    Terms are c_m sin(za)^k_m cos(k_m az + phi_m) cos(l_m za) cos(w_m nu + psi_m)
    with sum |c_m| = 1.  The sin(za)^k factor makes each azimuthal harmonic
    regular at the zenith pole."""
    k = g.integers(0, 4, size=n_terms)
    l = g.uniform(0.5, 3.0, size=n_terms)
    w = g.uniform(0.5, 4.0, size=n_terms)
    phi = g.uniform(0, 2 * np.pi, size=n_terms)
    psi = g.uniform(0, 2 * np.pi, size=n_terms)
    c = g.uniform(-1.0, 1.0, size=n_terms)
    c = c / np.sum(np.abs(c))
    r = np.zeros(np.broadcast(az, za, nu_norm).shape)
    for m in range(n_terms):
        r = r + c[m] * np.sin(za) ** k[m] * np.cos(k[m] * az + phi[m]) * np.cos(l[m] * za) \
            * np.cos(w[m] * nu_norm + psi[m])
    return r


def gaussian_ripple_grid(nu_grid: np.ndarray, n_za: int, n_az: int, fwhm_ref: float,
                         nu_ref: float, ripple: float, g: np.random.Generator) -> np.ndarray:
    """Scalar beam grid, complex64 [1][1][1][nu][za][az]: a Gaussian with
    FWHM(nu) = fwhm_ref * nu_ref / nu times (1 + ripple * r)."""
    za = np.arange(n_za) * (np.pi / 2 / (n_za - 1))
    az = np.arange(n_az) * (2 * np.pi / n_az)
    nun = (nu_grid - nu_ref) / nu_ref
    NU, ZA, AZ = np.meshgrid(nun, za, az, indexing="ij")
    fwhm = fwhm_ref * nu_ref / nu_grid
    env = np.exp(-4.0 * np.log(2.0) * ZA ** 2 / (fwhm[:, None, None] ** 2))
    vals = env * (1.0 + ripple * ripple_field(AZ, ZA, NU, g))
    return vals.astype(np.complex64).reshape(1, 1, 1, len(nu_grid), n_za, n_az)


# ---------------------------------------------------------------- workloads

@dataclass
class Workload:
    """Inputs of one workload; beam is ("gaussian", fwhm) or
    ("grid", values c64 [beam][feed][ax][nu][za][az], nu0, dnu, dza, daz, interp)."""
    name: str
    ra: np.ndarray
    dec: np.ndarray
    flux_ref: np.ndarray
    spec_idx: Optional[np.ndarray]
    nu_ref: float
    enu: np.ndarray
    lat: float
    beam: tuple
    lsts: np.ndarray
    freqs: np.ndarray
    beam_idx: Optional[np.ndarray] = None
    notes: dict = field(default_factory=dict)
    stokes_quv: Optional[np.ndarray] = None   # [3][n_src] Q, U, V (Jy at nu_ref) of a polarised sky

    @property
    def n_ant(self) -> int:
        return self.enu.shape[0]

    @property
    def n_src(self) -> int:
        return self.ra.size


def tiny(n_ant: int = 10, n_src: int = 1000, n_times: int = 4) -> Workload:
    """The tiny workload (module docstring)."""
    enu = square_array(n_ant, 50.0, rng(0, "antennas"))
    ra, dec = uniform_sphere(n_src, rng(0, "positions"))
    flux = powerlaw_flux(n_src, 0.1, 10.0, 1.6, rng(0, "flux"))
    lsts = np.arange(n_times) * (10.0 * SIDEREAL_MINUTE / max(n_times - 1, 1))
    return Workload("tiny: 10 ant x 1000 src x 1 ch x 4 t, gaussian beam",
                    ra, dec, flux, None, 150e6, enu, HERA_LAT,
                    ("gaussian", 10.0 * DEG), lsts, np.array([150e6]))


def hera_like(n_ant: int = 350, n_src: int = 100_000, n_chan: int = 64, n_times: int = 60,
              n_za: int = 91, n_az: int = 360) -> Workload:
    """The HERA-like workload (module docstring); smaller sizes give its test cases."""
    enu = hex_array(n_ant, 14.6)
    ra, dec = uniform_sphere(n_src, rng(1, "positions"))
    flux = powerlaw_flux(n_src, 0.01, 100.0, 1.6, rng(1, "flux"))
    alpha = rng(1, "spectral_index").normal(-0.8, 0.2, size=n_src)
    freqs = 100e6 + (np.arange(n_chan) + 0.5) * (100e6 / n_chan)
    lsts = np.arange(n_times) * SIDEREAL_MINUTE
    nu_grid = 98e6 + np.arange(105) * 1e6
    grid = gaussian_ripple_grid(nu_grid, n_za, n_az, 10.0 * DEG, 150e6, 0.05, rng(1, "beam_ripple"))
    beam = ("grid", grid, 98e6, 1e6, (np.pi / 2) / (n_za - 1), 2 * np.pi / n_az, "cubic")
    return Workload(f"hera_like: {n_ant} ant x {n_src} src x {n_chan} ch x {n_times} t, bicubic grid beam",
                    ra, dec, flux, alpha, 150e6, enu, HERA_LAT, beam, lsts, freqs)


def batched_uneven(n_pairs: int = 256, n_ant: int = 350, n_src: int = 100_000, n_za: int = 91,
                   n_az: int = 360) -> Workload:
    """Batched uneven instances: n_pairs (LST, frequency) pairs, LST ~ U[0, 24 h) and
    nu ~ U[50, 250] MHz, for the HERA-like array; the sky is 40 % uniform and
    60 % von Mises-Fisher clustered (kappa = 20) about RA 6 h, Dec = latitude,
    so the horizon cut leaves about 20k-80k live sources depending on LST;
    fluxes and spectra as the HERA-like workload; its beam on 48-252 MHz.
    `lsts` and `freqs` hold the pairs (equal length)."""
    enu = hex_array(n_ant, 14.6)
    n_uni = int(round(0.4 * n_src))
    ra1, dec1 = uniform_sphere(n_uni, rng(3, "positions_uniform"))
    ra2, dec2 = vmf_cluster(n_src - n_uni, 20.0, np.pi / 2, HERA_LAT, rng(3, "positions_cluster"))
    ra, dec = np.concatenate([ra1, ra2]), np.concatenate([dec1, dec2])
    flux = powerlaw_flux(n_src, 0.01, 100.0, 1.6, rng(3, "flux"))
    alpha = rng(3, "spectral_index").normal(-0.8, 0.2, size=n_src)
    gp = rng(3, "pairs")
    lsts = gp.uniform(0.0, 2 * np.pi, n_pairs)
    freqs = gp.uniform(50e6, 250e6, n_pairs)
    nu_grid = 48e6 + np.arange(205) * 1e6
    grid = gaussian_ripple_grid(nu_grid, n_za, n_az, 10.0 * DEG, 150e6, 0.05, rng(3, "beam_ripple"))
    beam = ("grid", grid, 48e6, 1e6, (np.pi / 2) / (n_za - 1), 2 * np.pi / n_az, "cubic")
    return Workload(f"batched_uneven: {n_pairs} (LST, nu) pairs, {n_ant} ant x {n_src} src (40% uniform + "
                    "60% clustered), bicubic grid beam 48-252 MHz",
                    ra, dec, flux, alpha, 150e6, enu, HERA_LAT, beam, lsts, freqs)


def dipole_feed_offset_grids(n_ant: int, nu_grid: np.ndarray, n_za: int, n_az: int, g: np.random.Generator,
                             offset_m: float = 0.02, fwhm_ref: float = 30.0 * DEG, nu_ref: float = 150e6) -> np.ndarray:
    """Per-antenna Jones beams, complex64 [n_ant][2][2][nu][za][az]: a short
    dipole pair (X along East, Y along North) projected on the (theta, phi)
    basis, times a Gaussian envelope with FWHM fwhm_ref nu_ref / nu, times the
    phase exp(-2 pi i (nu / c) delta_a . s_hat) of a seeded feed displacement
    delta_a ~ U[-offset_m, offset_m] per axis."""
    za = np.arange(n_za) * (np.pi / 2 / (n_za - 1))
    az = np.arange(n_az) * (2 * np.pi / n_az)
    NU, ZA, AZ = np.meshgrid(nu_grid, za, az, indexing="ij")
    env = np.exp(-4.0 * np.log(2.0) * ZA ** 2 / (fwhm_ref * nu_ref / NU) ** 2)
    s = np.stack([np.sin(ZA) * np.sin(AZ), np.sin(ZA) * np.cos(AZ), np.cos(ZA)], -1)
    base = np.zeros((2, 2) + NU.shape)
    base[0, 0] = np.cos(ZA) * np.sin(AZ)
    base[0, 1] = np.cos(AZ)
    base[1, 0] = np.cos(ZA) * np.cos(AZ)
    base[1, 1] = -np.sin(AZ)
    delta = g.uniform(-offset_m, offset_m, size=(n_ant, 3))
    out = np.empty((n_ant, 2, 2) + NU.shape, dtype=np.complex64)
    for a in range(n_ant):
        ph = np.exp(-2j * np.pi * (NU / 299792458.0) * (s @ delta[a]))
        out[a] = (base * (env * ph)[None, None]).astype(np.complex64)
    return out


def learned_beam(n_ant: int = 350, n_src: int = 100_000, n_chan: int = 64, n_times: int = 60, n_za: int = 91,
                 n_az: int = 360, dnu: float = 1e6, nu_lo: float = 98e6, nu_hi: float = 202e6) -> Workload:
    """Learned-beam workload: the HERA-like array and sky with one beam per
    antenna (dipole_feed_offset_grids on a 1 deg x 1 deg x 1 MHz grid over
    98-202 MHz, or [nu_lo, nu_hi] for samples of it), the setting where a
    learned surrogate replaces n_ant grids."""
    w = hera_like(n_ant=n_ant, n_src=n_src, n_chan=n_chan, n_times=n_times, n_za=31, n_az=60)
    n_nu = int(round((nu_hi - nu_lo) / dnu)) + 1
    nu_grid = nu_lo + np.arange(n_nu) * dnu
    grids = dipole_feed_offset_grids(n_ant, nu_grid, n_za, n_az, rng(4, "feed_offsets"))
    w.beam = ("grid", grids, nu_lo, dnu, (np.pi / 2) / (n_za - 1), 2 * np.pi / n_az, "cubic")
    w.beam_idx = np.arange(n_ant, dtype=np.int32)
    w.name = (f"learned_beam: {n_ant} ant (one Jones beam each) x {n_src} src x {n_chan} ch x {n_times} t, "
              f"Fourier-feature MLP beam")
    return w


# ----------------------------------------------------------- diffuse sky

def healpix_ring_pix2ang(nside: int):
    """(theta, phi) of every HEALPix pixel centre in RING order (Gorski et al.
    2005, ApJ 622, 759: polar caps, equatorial belt, south cap)."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    p = np.arange(npix, dtype=np.int64)
    z = np.empty(npix)
    phi = np.empty(npix)
    north = p < ncap
    south = p >= npix - ncap
    belt = ~(north | south)
    # north cap: ring i has 4 i pixels
    pn = p[north]
    i = np.floor(np.sqrt((pn + 1) / 2.0 - np.sqrt(np.floor((pn + 1) / 2.0)))).astype(np.int64) + 1
    j = pn + 1 - 2 * i * (i - 1)
    z[north] = 1.0 - i * i / (3.0 * nside * nside)
    phi[north] = np.pi / (2.0 * i) * (j - 0.5)
    # equatorial belt: rings nside .. 3 nside, 4 nside pixels each
    pe = p[belt] - ncap
    i = pe // (4 * nside) + nside
    j = pe % (4 * nside) + 1
    s = (i - nside + 1) % 2
    z[belt] = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
    phi[belt] = np.pi / (2.0 * nside) * (j - s / 2.0)
    # south cap (mirror of the north cap)
    ps = npix - p[south]
    i = np.floor(np.sqrt(ps / 2.0 - np.sqrt(np.floor(ps / 2.0)))).astype(np.int64) + 1
    j = 4 * i + 1 - (ps - 2 * i * (i - 1))
    z[south] = -1.0 + i * i / (3.0 * nside * nside)
    phi[south] = np.pi / (2.0 * i) * (j - 0.5)
    return np.arccos(np.clip(z, -1, 1)), phi


def gaussian_random_field(theta: np.ndarray, phi: np.ndarray, lmax: int, cl: np.ndarray,
                          g: np.random.Generator) -> np.ndarray:
    """Real Gaussian random field sum_lm a_lm Y_lm at the given points, with
    a_lm ~ N(0, C_l) (complex for m > 0), evaluated ring by ring: the
    normalised associated Legendre functions come from the standard three-term
    recurrence in l at fixed m, and each ring's azimuthal sum is one matrix
    product over m."""
    a = np.zeros((lmax + 1, lmax + 1), dtype=np.complex128)
    for l in range(lmax + 1):
        sd = np.sqrt(cl[l])
        a[l, 0] = sd * g.normal()
        if l > 0:
            a[l, 1:l + 1] = sd * (g.normal(size=l) + 1j * g.normal(size=l)) / np.sqrt(2.0)
    zs, inv = np.unique(np.round(np.cos(theta), 12), return_inverse=True)
    st = np.sqrt(np.maximum(0.0, 1.0 - zs * zs))
    # fm[r, m] = sum_l a_lm lam_lm(z_r), lam_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m,
    # the recursion in l vectorised over the rings
    fm = np.zeros((zs.size, lmax + 1), dtype=np.complex128)
    pmm = np.full(zs.size, 1.0 / np.sqrt(4 * np.pi))
    for m in range(lmax + 1):
        if m > 0:
            pmm = -np.sqrt((2 * m + 1) / (2.0 * m)) * st * pmm
        l2, l1 = None, pmm
        fm[:, m] += a[m, m] * pmm
        if m + 1 <= lmax:
            l2, l1 = pmm, zs * np.sqrt(2 * m + 3) * pmm
            fm[:, m] += a[m + 1, m] * l1
        for l in range(m + 2, lmax + 1):
            al = np.sqrt((4.0 * l * l - 1) / (l * l - m * m))
            bl = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1) ** 2 - 1))
            l2, l1 = l1, al * (zs * l1 - bl * l2)
            fm[:, m] += a[l, m] * l1
    out = np.empty(theta.size)
    for r in range(zs.size):
        sel = np.nonzero(inv == r)[0]
        e = np.exp(1j * np.outer(np.arange(1, lmax + 1), phi[sel]))
        out[sel] = fm[r, 0].real + 2.0 * np.real(fm[r, 1:, None] * e).sum(axis=0)
    return out


def polarised_diffuse(n_ant: int = 350, nside: int = 128, n_chan: int = 32, n_times: int = 120,
                      n_za: int = 91, n_az: int = 360, lmax: int = None, full_stokes: bool = False) -> Workload:
    """Polarised diffuse workload: the HERA-like array, a diffuse sky of 12 nside^2 HEALPix
    pixel centres whose intensities are a log-normal Gaussian random field
    (C_l ~ l^-2.5 for l >= 1, C_0 = 0, field normalised to unit variance)
    turned into fluxes (intensity x pixel area, about 1e3 Jy in total, spectral
    index -2.5), 32 channels centred in 140-160 MHz, 120 LSTs 30 s apart, and
    a 2 feed x 2 axis dipole-like Jones beam on a 1 deg x 1 deg x 1 MHz grid
    (138-162 MHz) with a 5 % ripple and a smooth phase of at most 0.1 rad.

    full_stokes adds linear polarisation of fraction 0.2 with an angle
    chi = pi Phi(h) from a second random field h (same spectrum, Phi the
    normal CDF), Q = 0.2 I cos 2chi, U = 0.2 I sin 2chi, and circular
    polarisation V = 0.01 I g' from a third field g' clipped to [-1, 1]."""
    lmax = 3 * nside - 1 if lmax is None else lmax
    theta, phi = healpix_ring_pix2ang(nside)
    ell = np.arange(lmax + 1, dtype=float)
    cl = np.where(ell >= 1, np.maximum(ell, 1.0) ** -2.5, 0.0)
    f = gaussian_random_field(theta, phi, lmax, cl, rng(2, "grf"))
    f = (f - f.mean()) / f.std()
    inten = np.exp(f - 0.5)
    npix = theta.size
    flux = inten * (4 * np.pi / npix)
    flux *= 1e3 / flux.sum()
    ra, dec = phi, np.pi / 2 - theta
    enu = hex_array(n_ant, 14.6)
    freqs = 140e6 + (np.arange(n_chan) + 0.5) * (20e6 / n_chan)
    lsts = np.arange(n_times) * (0.5 * SIDEREAL_MINUTE)
    nu_grid = 138e6 + np.arange(25) * 1e6
    gb = rng(2, "beam")
    za = np.arange(n_za) * (np.pi / 2 / (n_za - 1))
    az = np.arange(n_az) * (2 * np.pi / n_az)
    NU, ZA, AZ = np.meshgrid(nu_grid, za, az, indexing="ij")
    env = np.exp(-4 * np.log(2) * ZA ** 2 / (30 * DEG * 150e6 / NU) ** 2)
    rip = 1.0 + 0.05 * ripple_field(AZ, ZA, (NU - 150e6) / 150e6, gb)
    pha = 0.1 * ripple_field(AZ, ZA, (NU - 150e6) / 150e6, gb)
    J = np.zeros((1, 2, 2) + NU.shape, dtype=np.complex128)
    J[0, 0, 0] = np.cos(ZA) * np.sin(AZ)
    J[0, 0, 1] = np.cos(AZ)
    J[0, 1, 0] = np.cos(ZA) * np.cos(AZ)
    J[0, 1, 1] = -np.sin(AZ)
    J = (J * (env * rip * np.exp(1j * pha))[None, None, None]).astype(np.complex64)
    beam = ("grid", J, 138e6, 1e6, (np.pi / 2) / (n_za - 1), 2 * np.pi / n_az, "cubic")
    w = Workload(f"polarised_diffuse: {n_ant} ant x {npix} HEALPix pixels (nside {nside}) x {n_chan} ch x "
                 f"{n_times} t, 2x2 Jones beam", ra, dec, flux, np.full(npix, -2.5), 150e6, enu, HERA_LAT,
                 beam, lsts, freqs)
    if full_stokes:
        from scipy.special import ndtr
        h = gaussian_random_field(theta, phi, lmax, cl, rng(2, "pol_angle"))
        chi = np.pi * ndtr((h - h.mean()) / h.std())
        gv = gaussian_random_field(theta, phi, lmax, cl, rng(2, "circular"))
        gv = np.clip((gv - gv.mean()) / gv.std(), -1, 1)
        w.stokes_quv = np.stack([0.2 * flux * np.cos(2 * chi), 0.2 * flux * np.sin(2 * chi), 0.01 * flux * gv])
        w.name = w.name.replace("2x2 Jones beam", "2x2 Jones beam, full Stokes")
    return w
