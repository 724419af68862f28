"""Parity at the full sizes, in the launch configuration the benchmark times
(needs a GB300): the whole 350-antenna x 1e5-source x 64-channel x 60-LST
workload in one mv_simulate call after mv_autotune (persistent HERK with the
fused Z build, CUDA graph, autotuned tile/split/flush), FP16x3, checked on
sampled outputs the oracle computes one by one: every autocorrelation and 150
random baselines of six instances (first and last channel and LST, two more).
The same for the polarised diffuse sky (120 LSTs x 32 channels, 2 x 2 Jones,
full Stokes), four instances.  Tolerance 1e-5 (max over the sampled outputs
of one instance, relative to their maximum); live counts bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import oracle_problem, rel_err, sample_pairs, simulator
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
