"""Algorithm 1 (Sec. 2.3) end to end on the GPU (needs a GB300).

Apparent source directions are modelled as the catalogue seen through a fixed
small frame rotation Q (a stand-in for the astrometric corrections astropy
would supply).  A run of four LSTs is cut into two chunks; each chunk takes
the apparent (alt, az) at its own reference LST, perturbs the catalogue with
mv_perturb_sky and simulates its LSTs.  For a fixed frame rotation the
perturbed catalogue is exact at every LST, so V must match the oracle's
simulation of the rotated catalogue within 1e-5, while the unperturbed
catalogue is visibly wrong.
"""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_err, simulator
from paper_2312_09763_gb300 import perturb_sky, synth

pytestmark = pytest.mark.gpu
DEG = np.pi / 180


def frame_rotation(theta, axis):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(theta) * K + (1 - np.cos(theta)) * K @ K


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_chunked_perturbed_catalogue_matches_apparent_sky(prec):
    w = synth.hera_like(n_ant=60, n_src=20_000, n_chan=2, n_times=4, n_za=46, n_az=120)
    w.lsts = np.array([1.00, 1.05, 2.40, 2.46])
    Q = frame_rotation(0.4 * DEG, [0.3, -0.5, 0.8])
    Xq = oracle.xeq(w.ra, w.dec) @ Q.T
    # the "true" sky: the rotated catalogue's own RA/Dec
    true = synth.hera_like(n_ant=60, n_src=20_000, n_chan=2, n_times=4, n_za=46, n_az=120)
    true.ra = np.mod(np.arctan2(Xq[:, 1], Xq[:, 0]), 2 * np.pi)
    true.dec = np.arctan2(Xq[:, 2], np.hypot(Xq[:, 0], Xq[:, 1]))
    P_true = oracle_problem(true)
    sim = simulator(w)
    for chunk in (slice(0, 2), slice(2, 4)):
        lsts = w.lsts[chunk]
        lst_ref = float(lsts.mean())
        az, za = oracle.azza(oracle.to_topo(oracle.rotation(lst_ref, w.lat), Xq))
        ra, dec = perturb_sky(np.pi / 2 - za, az, lst_ref, w.lat)
        sim.init_sky(w.ra, w.dec, w.flux_ref, w.spec_idx, w.nu_ref)
        V0 = sim.simulate(lsts, w.freqs, prec).cpu().numpy()
        sim.init_sky(ra, dec, w.flux_ref, w.spec_idx, w.nu_ref)
        V = sim.simulate(lsts, w.freqs, prec).cpu().numpy()
        for it, lst in enumerate(lsts):
            for ic, nu in enumerate(w.freqs):
                Vo = oracle.vis(P_true, lst, nu)
                assert rel_err(V[it, ic], Vo) <= 1e-5, (lst, nu)
                assert rel_err(V0[it, ic], Vo) > 1e-3
