"""Polarised diffuse sky (HEALPix pixel centres, log-normal random field,
2 feed x 2 axis Jones beam) vs the FP64 oracle (needs a GB300).

Small case: 40 antennas x nside 16 (3,072 pixels), every visibility of two
LSTs x two channels.  Full size: 350 antennas x nside 128 (196,608 pixels),
two LSTs x two channels, every autocorrelation and 300 random baselines, all
four feed products each.  Tolerances as for the point-source sky (1e-5;
BF16x3 2e-5); live counts bit-exact.  The same with full Stokes (Q, U, V;
Z = A F M with C = M M^dagger, eq. "fullz") against the oracle's direct sum
over the coherency.
"""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_err, sample_pairs, simulator
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "fp16x3": 1e-5}


@pytest.mark.parametrize("full_stokes", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_small_diffuse_full_parity(prec, full_stokes):
    w = synth.polarised_diffuse(n_ant=40, nside=16, n_chan=2, n_times=2, n_za=31, n_az=72, lmax=40,
                                full_stokes=full_stokes)
    w.lsts = np.array([0.4, 3.9])
    sim = simulator(w)
    V = sim.simulate(w.lsts, w.freqs, prec).cpu().numpy()
    assert V.shape == (2, 2, 80, 80)
    P = oracle_problem(w)
    for it, lst in enumerate(w.lsts):
        for ic, nu in enumerate(w.freqs):
            assert rel_err(V[it, ic], oracle.vis(P, lst, nu)) <= TOL[prec], (it, ic)
    live = sim.last_live_counts(4).reshape(2, 2)   # [time][channel]
    assert list(live[:, 0]) == list(live[:, 1]) == [oracle.count_live(P, t) for t in w.lsts]


@pytest.fixture(scope="module")
def diffuse():
    w = synth.polarised_diffuse(full_stokes=True)
    stokes = w.stokes_quv
    w.stokes_quv = None
    return w, stokes


@pytest.mark.parametrize("prec,full_stokes", [("fp32", False), ("fp16x3", False),
                                              ("fp32", True), ("fp16x3", True)])
def test_full_size_diffuse_sampled(diffuse, prec, full_stokes):
    w, stokes = diffuse
    w.stokes_quv = stokes if full_stokes else None
    P = oracle_problem(w)
    lsts, freqs = w.lsts[[0, 119]], w.freqs[[0, 31]]
    sim = simulator(w)
    V = sim.simulate(lsts, freqs, prec).cpu().numpy()
    N = w.n_ant
    assert V.shape == (2, 2, 2 * N, 2 * N)
    live = sim.last_live_counts(4).reshape(2, 2)
    assert list(live[:, 1]) == [oracle.count_live(P, t) for t in lsts]
    pa, pb = sample_pairs(N, 300, seed=3)
    for it, lst in enumerate(lsts):
        for ic, nu in enumerate(freqs):
            vo = oracle.vis(P, lst, nu, pairs=(pa, pb))           # (pairs, feed, feed)
            v = V[it, ic].reshape(N, 2, N, 2)[pa, :, pb, :]
            assert rel_err(v, vo) <= TOL[prec], (it, ic)
            vm = V[it, ic].reshape(N, 2, N, 2)[pb, :, pa, :]
            assert np.array_equal(vm, np.conj(np.swapaxes(v, 1, 2)))


def test_polarisation_argument_checks():
    w = synth.polarised_diffuse(n_ant=10, nside=4, n_chan=1, n_times=1, n_za=31, n_az=72, lmax=8)
    sim = simulator(w)
    from paper_2312_09763_gb300.binding import MatvisError
    over = np.zeros((3, w.n_src))
    over[0] = 1.01 * w.flux_ref
    with pytest.raises(MatvisError, match="MV_ERR_ARG"):
        sim.set_sky_polarisation(over)
    sim.set_sky_polarisation(np.zeros((3, w.n_src)))
    sim.set_beam_gaussian(0.3)  # single-axis beam
    with pytest.raises(MatvisError, match="two-axis"):
        sim.simulate(w.lsts, w.freqs, "fp32")
    sim.set_sky_polarisation(None)
    sim.simulate(w.lsts, w.freqs, "fp32")
