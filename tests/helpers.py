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
                          spec_idx=w.spec_idx, nu_ref=w.nu_ref, beam_idx=w.beam_idx, stokes_quv=w.stokes_quv)


def simulator(w: synth.Workload, interp: str = "cubic", **kw):
    from paper_2312_09763_gb300 import Simulator
    sim = Simulator(0, interp=interp, **kw)
    sim.init_sky(w.ra, w.dec, w.flux_ref, w.spec_idx, w.nu_ref)
    sim.set_beam(w.beam)
    sim.set_antennas(w.enu, w.beam_idx, w.lat)
    if w.stokes_quv is not None:
        sim.set_sky_polarisation(w.stokes_quv)
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


def oracle_net(sim, nu0: float, dnu: float, n_nu: int):
    """The FP64 oracle MLP holding the GPU surrogate's current parameters."""
    from oracle import mlp
    p, B, lay = sim.surrogate_params()
    cfg = sim._mlp
    F, E, H, D = cfg["n_freq"], cfg["emb_dim"], cfg["width"], cfg["depth"]
    d0, d0p, off_emb = 2 * F + E, int(lay[-1]), int(lay[-2])
    n_out = 2 * sim.n_feed * sim._n_ax()
    W, b = [], []
    for l in range(D + 1):
        ow, ob = int(lay[2 * l]), int(lay[2 * l + 1])
        kin, nout = (d0p if l == 0 else H), (8 if l == D else H)
        Wl = p[ow:ow + nout * kin].reshape(nout, kin).astype(np.float64)
        bl = p[ob:ob + nout].astype(np.float64)
        if l == 0:
            Wl = Wl[:, :d0]
        if l == D:
            Wl, bl = Wl[:n_out], bl[:n_out]
        W.append(Wl)
        b.append(bl)
    n_beam = (p.size - off_emb) // E
    emb = p[off_emb:off_emb + n_beam * E].reshape(n_beam, E).astype(np.float64)
    lo, hi = nu0, nu0 + (n_nu - 1) * dnu
    return mlp.MLP(B=B.astype(np.float64), emb=emb, W=W, b=b, nu_mid=0.5 * (lo + hi), nu_half=0.5 * (hi - lo))


def flat_grads(sim, g: dict) -> np.ndarray:
    """Oracle gradients laid out like the GPU parameter vector (padding zero)."""
    p, B, lay = sim.surrogate_params()
    cfg = sim._mlp
    F, E, H, D = cfg["n_freq"], cfg["emb_dim"], cfg["width"], cfg["depth"]
    d0, d0p, off_emb = 2 * F + E, int(lay[-1]), int(lay[-2])
    out = np.zeros(p.size)
    for l in range(D + 1):
        ow, ob = int(lay[2 * l]), int(lay[2 * l + 1])
        kin, nout = (d0p if l == 0 else H), (8 if l == D else H)
        Wg = np.zeros((nout, kin))
        gw = g[f"W{l}"]
        Wg[:gw.shape[0], :gw.shape[1]] = gw
        out[ow:ow + nout * kin] = Wg.ravel()
        out[ob:ob + g[f"b{l}"].size] = g[f"b{l}"]
    out[off_emb:off_emb + g["emb"].size] = g["emb"].ravel()
    return out
