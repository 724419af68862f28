"""Parity at the full sizes, in the launch configuration the benchmark times
(needs a GB300): the whole 350-antenna x 1e5-source x 64-channel x 60-LST
workload in one mv_simulate call after mv_autotune (persistent HERK with the
fused Z build, CUDA graph, autotuned tile/split/flush), FP16x3, checked on
sampled outputs the oracle computes one by one: every autocorrelation and 150
random baselines of six instances (first and last channel and LST, two more).
The same for the polarised diffuse sky (120 LSTs x 32 channels, 2 x 2 Jones,
full Stokes), four instances.  Tolerance 1e-5 (max over the sampled outputs
of one instance, relative to their maximum); live counts bit-exact.  And the
learned-beam sample of the benchmark (350 per-antenna beams as the 4 x 256
network, 1e5 sources, one LST x 8 channels) against the oracle holding the
same network, on the baselines among 12 antennas of two channels, within 3e-2
(BF16 operands and activations).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import oracle_net, oracle_problem, rel_err, sample_pairs, simulator
from oracle import mlp
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu


def check(sim, w, P, V, picks, n_pairs, nf, seed):
    N = w.n_ant
    live = sim.last_live_counts(len(w.lsts) * len(w.freqs)).reshape(len(w.lsts), len(w.freqs))
    pa, pb = sample_pairs(N, n_pairs, seed=seed)
    ia = torch.as_tensor(pa, device=V.device, dtype=torch.long)
    ib = torch.as_tensor(pb, device=V.device, dtype=torch.long)
    for it, ic in picks:
        assert live[it, ic] == oracle.count_live(P, w.lsts[it])
        Vi = V[it, ic].reshape(N, nf, N, nf)
        v = Vi[ia, :, ib, :].cpu().numpy()                 # (pairs, nf, nf)
        vo = oracle.vis(P, w.lsts[it], w.freqs[ic], pairs=(pa, pb))
        assert rel_err(v, vo) <= 1e-5, (it, ic)


def test_hera_workload_as_benchmarked():
    w = synth.hera_like()
    P = oracle_problem(w)
    sim = simulator(w)
    sim.autotune(w.lsts, w.freqs, "fp16x3")
    V = torch.empty((60, 64, 350, 350), dtype=torch.complex64, device="cuda")
    for _ in range(2):  # capture, then replay
        sim.simulate(w.lsts, w.freqs, "fp16x3", out=V)
    torch.cuda.synchronize()
    picks = [(0, 0), (59, 63), (0, 63), (59, 0), (17, 31), (42, 9)]
    check(sim, w, P, V, picks, 150, 1, seed=11)


def test_diffuse_workload_as_benchmarked():
    w = synth.polarised_diffuse(full_stokes=True)
    P = oracle_problem(w)
    sim = simulator(w)
    sim.autotune(w.lsts, w.freqs, "fp16x3")
    V = torch.empty((120, 32, 700, 700), dtype=torch.complex64, device="cuda")
    sim.simulate(w.lsts, w.freqs, "fp16x3", out=V)
    torch.cuda.synchronize()
    check(sim, w, P, V, [(0, 0), (119, 31), (60, 15), (7, 28)], 100, 2, seed=12)


def test_hera_redundant_groups_as_benchmarked():
    # bench.py --unique: one value per redundant group over the whole workload
    # (cover of the representatives, 256-column tiles, CUDA graph); every
    # group of four instances against the oracle at its representative
    from paper_2312_09763_gb300 import redundancy_plan
    w = synth.hera_like()
    P = oracle_problem(w)
    sim = simulator(w)
    n_u = sim.set_redundancy(1e-3)
    plan = redundancy_plan(w.enu, None, 1e-3, 1, 128)
    assert plan["kind"] in (1, 2) and plan["tiles"] < plan["tiles_full"]
    V = torch.empty((60, 64, n_u, 1, 1), dtype=torch.complex64, device="cuda")
    for _ in range(2):  # capture, then replay
        sim.simulate_unique(w.lsts, w.freqs, "fp16x3", out=V)
    torch.cuda.synchronize()
    for it, ic in [(0, 0), (59, 63), (30, 17), (11, 50)]:
        vo = oracle.vis(P, w.lsts[it], w.freqs[ic], pairs=(plan["rep_a"], plan["rep_b"]))
        assert rel_err(V[it, ic].cpu().numpy(), vo) <= 1e-5, (it, ic)


def test_learned_beam_workload_as_benchmarked():
    # one call of the benchmark's learned-beam sample: per instance the first
    # layer's source part (50,013 live sources), its beam part (350 beams) and
    # the fused forward pass over ~68,800 tiles of 8 beams x 32 sources, then
    # the Z build and HERK.  The oracle evaluates the same network (FP64) for
    # the beams of 12 antennas and sums their baselines.
    w = synth.learned_beam(n_chan=8, n_times=1, nu_lo=143e6, nu_hi=157e6)
    w.freqs = 146.5e6 + np.arange(8) * 1e6
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=200, batch=16384, lr0=2e-3, lr1=1e-4, seed=3)
    net = oracle_net(sim, w.beam[2], w.beam[3], w.beam[1].shape[3])
    sim.set_beam_surrogate(True)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3")
    torch.cuda.synchronize()
    ants = np.sort(np.random.default_rng(13).choice(w.n_ant, 12, replace=False))
    # the oracle's problem on those 12 antennas (local beam indices 0..11)
    P = oracle.Problem(ra=w.ra, dec=w.dec, flux_ref=w.flux_ref, enu=w.enu[ants], lat=w.lat, beam=("uniform",),
                       spec_idx=w.spec_idx, nu_ref=w.nu_ref, beam_idx=np.arange(12, dtype=np.int32))
    la, lb = np.tril_indices(12)
    for ic in (0, 7):
        f = float(w.freqs[ic])

        def beam_fn(az, za, nu):
            n = az.size
            out = np.empty((12, 2, 2, n), dtype=np.complex128)
            for k, a in enumerate(ants):
                y = mlp.forward(net, np.full(n, a), az, za, np.full(n, nu))
                out[k] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
            return out
        vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn, pairs=(la, lb))
        Vi = V[0, ic].reshape(w.n_ant, 2, w.n_ant, 2)
        ia = torch.as_tensor(ants[la], device=V.device, dtype=torch.long)
        ib = torch.as_tensor(ants[lb], device=V.device, dtype=torch.long)
        v = Vi[ia, :, ib, :].cpu().numpy()
        assert rel_err(v, vo) <= 3e-2, ic
