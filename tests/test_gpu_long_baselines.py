"""Long baselines and far-off array centres against the FP64 oracle (needs a GB300).

The phase (nu/c) x_a . s_hat reaches thousands of turns on kilometre
baselines and at antenna positions kilometres from the array's origin.  The
Z build forms it in 64-bit fixed point (32 x 32 -> 64-bit products that wrap
modulo one turn), so these cases exercise exactly the wrap that short
baselines never reach.  Tolerance: max|V - V_oracle| / max|V_oracle| <= 1e-5
for both modes.
"""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_err, sample_pairs, simulator
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
PRECS = ["fp32", "fp16x3"]


@pytest.fixture(scope="module")
def hera_sample():
    # the 350-antenna array and the 1e5-source sky, 2 LSTs x 2 channels at
    # both ends of the band
    w = synth.hera_like()
    w.lsts, w.freqs = w.lsts[[0, 59]], w.freqs[[0, 63]]
    return w


@pytest.mark.parametrize("prec", PRECS)
def test_array_translated_ten_kilometres(hera_sample, prec):
    w = hera_sample
    base = simulator(w).simulate(w.lsts, w.freqs, prec).cpu().numpy()
    w2 = synth.hera_like()
    w2.lsts, w2.freqs = w.lsts, w.freqs
    w2.enu = w.enu + np.array([10_000.0, -7_000.0, 3.0])
    V = simulator(w2).simulate(w2.lsts, w2.freqs, prec).cpu().numpy()
    P = oracle_problem(w2)
    pa, pb = sample_pairs(w2.n_ant, 300, seed=13)
    for it, lst in enumerate(w2.lsts):
        for ic, nu in enumerate(w2.freqs):
            vo = oracle.vis(P, lst, nu, pairs=(pa, pb))[:, 0, 0]
            assert rel_err(V[it, ic][pa, pb], vo) <= TOL, (it, ic)
            # V depends on baselines only: the untranslated array's V
            assert rel_err(V[it, ic], base[it, ic]) <= TOL, (it, ic)


@pytest.mark.parametrize("prec", PRECS)
def test_three_kilometre_random_array(prec):
    # 96 antennas uniform in a 3 km square with +-5 m of Up: baselines up to
    # ~4 km, phases up to ~2e3 turns at 200 MHz
    w = synth.hera_like(n_ant=96, n_src=30_000, n_chan=3, n_times=2, n_za=46, n_az=120)
    g = np.random.default_rng(21)
    w.enu = np.zeros((96, 3))
    w.enu[:, :2] = g.uniform(-1500, 1500, (96, 2))
    w.enu[:, 2] = g.uniform(-5, 5, 96)
    w.freqs = np.array([120.3e6, 160.7e6, 199.1e6])
    V = simulator(w).simulate(w.lsts, w.freqs, prec).cpu().numpy()
    P = oracle_problem(w)
    for it, lst in enumerate(w.lsts):
        for ic, nu in enumerate(w.freqs):
            assert rel_err(V[it, ic], oracle.vis(P, lst, nu)) <= TOL, (it, ic)
