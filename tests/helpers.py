"""Shared test plumbing: the same seeded workload feeds the CUDA path and the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2312_09763_gb300 import synth


def oracle_problem(w: synth.Workload, beam=None) -> oracle.Problem:
    beam = beam or w.beam
    if beam[0] == "grid":
        vals, nu0, dnu, dza, daz, interp = beam[1:7]
        beam = ("grid", np.asarray(vals).astype(np.complex128), nu0, dnu, dza, daz, interp)
    return oracle.Problem(ra=w.ra, dec=w.dec, flux_ref=w.flux_ref, enu=w.enu, lat=w.lat, beam=beam,
                          spec_idx=w.spec_idx, nu_ref=w.nu_ref, beam_idx=w.beam_idx)


def simulator(w: synth.Workload, interp: str = "cubic", **kw):
    from paper_2312_09763_gb300 import Simulator
    sim = Simulator(0, interp=interp, **kw)
    sim.init_sky(w.ra, w.dec, w.flux_ref, w.spec_idx, w.nu_ref)
    sim.set_beam(w.beam)
    sim.set_antennas(w.enu, w.beam_idx, w.lat)
    return sim


def rel_err(v, vo) -> float:
    """max |V - V_oracle| / max |V_oracle| (the accuracy metric)."""
    v = np.asarray(v, dtype=np.complex128)
    vo = np.asarray(vo, dtype=np.complex128)
    return float(np.abs(v - vo).max() / np.abs(vo).max())


def sample_pairs(n_ant: int, n_cross: int, seed: int = 0):
    """All autocorrelations plus n_cross random cross baselines (a > b)."""
    g = np.random.default_rng(seed)
    a = g.integers(1, n_ant, n_cross)
    b = (g.random(n_cross) * a).astype(np.int64)
    aa = np.concatenate([np.arange(n_ant), a])
    bb = np.concatenate([np.arange(n_ant), b])
    return aa.astype(np.int32), bb.astype(np.int32)


def dipole_jones_grid(nu_grid, n_za, n_az, fwhm_ref, nu_ref, g: np.random.Generator):
    """Dipole-like 2 feed x 2 axis Jones grid (test input): X feed along East,
    Y along North, projected on (theta, phi), times a Gaussian envelope and a
    small seeded ripple and phase."""
    za = np.arange(n_za) * (np.pi / 2 / (n_za - 1))
    az = np.arange(n_az) * (2 * np.pi / n_az)
    NU, ZA, AZ = np.meshgrid(nu_grid, za, az, indexing="ij")
    fwhm = fwhm_ref * nu_ref / NU
    env = np.exp(-4 * np.log(2) * ZA ** 2 / fwhm ** 2)
    ph = 0.1 * np.sin(ZA) * np.cos(AZ + g.uniform(0, 2 * np.pi))
    J = np.zeros((1, 2, 2) + NU.shape, dtype=np.complex128)
    J[0, 0, 0] = np.cos(ZA) * np.sin(AZ)
    J[0, 0, 1] = np.cos(AZ)
    J[0, 1, 0] = np.cos(ZA) * np.cos(AZ)
    J[0, 1, 1] = -np.sin(AZ)
    J = J * env * np.exp(1j * ph) * (1 + 0.05 * np.cos(3 * ZA + 0.2 * (NU / nu_ref)))
    return J.astype(np.complex64)
