"""Large and extreme shapes against the FP64 oracle (needs a GB300): four
million sources on a small array (long source axis, 64-bit offsets), a
256-channel batch (the largest batch, sixteen Z groups in one launch) and
1000 antennas (2000 real rows, 136 tiles of the lower triangle).  FP16x3 and
FP32, tolerance 1e-5.  And the failure path: a bounded device-side wait that
runs out reports MV_ERR_DEVICE_TIMEOUT without a fault or a hang."""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_err, sample_pairs, simulator
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_four_million_sources(prec):
    w = synth.hera_like(n_ant=24, n_src=4_000_000, n_chan=2, n_times=1, n_za=46, n_az=120)
    w.freqs = np.array([120.5e6, 180.25e6])
    sim = simulator(w)
    V = sim.simulate(w.lsts, w.freqs, prec).cpu().numpy()
    P = oracle_problem(w)
    assert sim.last_live_counts(2)[0] == oracle.count_live(P, w.lsts[0])
    for ic, nu in enumerate(w.freqs):
        assert rel_err(V[0, ic], oracle.vis(P, w.lsts[0], nu)) <= 1e-5, ic


def test_largest_batch_of_channels():
    w = synth.hera_like(n_ant=20, n_src=3000, n_chan=256, n_times=1, n_za=46, n_az=120)
    sim = simulator(w, max_batch=256)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    assert V.shape == (1, 256, 20, 20)
    P = oracle_problem(w)
    for ic in (0, 15, 16, 127, 200, 255):
        assert rel_err(V[0, ic], oracle.vis(P, w.lsts[0], w.freqs[ic])) <= 1e-5, ic


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_thousand_antennas(prec):
    w = synth.hera_like(n_ant=1000, n_src=2000, n_chan=1, n_times=2, n_za=46, n_az=120)
    sim = simulator(w)
    V = sim.simulate(w.lsts, w.freqs, prec).cpu().numpy()
    assert V.shape == (2, 1, 1000, 1000)
    P = oracle_problem(w)
    pa, pb = sample_pairs(1000, 3000, seed=4)
    for it in range(2):
        vo = oracle.vis(P, w.lsts[it], w.freqs[0], pairs=(pa, pb))[:, 0, 0]
        assert rel_err(V[it, 0][pa, pb], vo) <= 1e-5, it


def test_bounded_wait_gives_up_and_the_context_survives():
    # a barrier nothing completes: the kernel's bounded wait gives up after
    # the limit, the host reads the timeout, and the context keeps working
    import time
    w = synth.hera_like(n_ant=40, n_src=3000, n_chan=2, n_times=1, n_za=46, n_az=120)
    sim = simulator(w)
    t0 = time.perf_counter()
    assert sim.selftest_wait_timeout(0.2) == "MV_ERR_DEVICE_TIMEOUT"
    assert 0.19 < time.perf_counter() - t0 < 5.0
    sim.check_device_status()  # the status word was cleared
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    P = oracle_problem(w)
    assert rel_err(V[0, 1], oracle.vis(P, w.lsts[0], w.freqs[1])) <= 1e-5
