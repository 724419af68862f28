"""The redundant-group output (Appendix A) on the GPU: one value per group of
redundant baselines, computed on the tiles of the planned cover only (needs a
GB300).  The values are checked against the FP64 oracle at the
representatives, and the full-V path is checked against them at every
baseline of every group (equal, or for a reversed baseline the conjugate with
the feeds swapped, V_ab^{pq} = conj(V_rep^{qp}); identical beams).
"""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_err, simulator
from paper_2312_09763_gb300 import MatvisError, redundancy_plan, synth

pytestmark = pytest.mark.gpu


def expand(Vu, plan, n_ant, nf):
    """Full V [.., N, N] from one value per group (lower and upper triangle)."""
    a = np.concatenate([np.full(n_ant - i, i) for i in range(n_ant)])
    b = np.concatenate([np.arange(i, n_ant) for i in range(n_ant)])
    g, cj = plan["group_of"], plan["conj_of"].astype(bool)
    lead = Vu.shape[:-3]
    flat = Vu.reshape((-1,) + Vu.shape[-3:])
    out = np.zeros((flat.shape[0], n_ant, nf, n_ant, nf), np.complex64)
    for i in range(flat.shape[0]):
        vals = flat[i][g]                                     # [n_bl, nf, nf]
        # a reversed baseline: V_ab^{pq} = conj(V_rep^{qp})
        vals = np.where(cj[:, None, None], np.conj(np.swapaxes(vals, -1, -2)), vals)
        out[i, b, :, a, :] = np.conj(np.swapaxes(vals, -1, -2))
        out[i, a, :, b, :] = vals
    return out.reshape(lead + (n_ant * nf, n_ant * nf))


@pytest.mark.parametrize("n_ant,tile_n,split", [(250, 256, 0), (250, 256, 1), (250, 128, 0), (250, 128, 3),
                                                (100, 256, 0)])
def test_hera_like_groups_match_oracle_and_full_v(n_ant, tile_n, split):
    # 250 antennas: a cover of two blocks; 100: one block (kind 2, columns first)
    w = synth.hera_like(n_ant=n_ant, n_src=6000, n_chan=3, n_times=2, n_za=46, n_az=120)
    sim = simulator(w, herk_tile_n=tile_n, herk_split=split)
    n_u = sim.set_redundancy(1e-3)
    plan = redundancy_plan(w.enu, None, 1e-3, 1, 128)
    assert n_u == plan["n_unique"] and plan["kind"] in (1, 2)
    for prec in ("fp16x3",):
        tol = 1e-5
        Vu = sim.simulate_unique(w.lsts, w.freqs, prec).cpu().numpy()
        assert Vu.shape == (2, 3, n_u, 1, 1)
        P = oracle_problem(w)
        for it in range(2):
            for ic in (0, 2):
                vo = oracle.vis(P, w.lsts[it], w.freqs[ic], pairs=(plan["rep_a"], plan["rep_b"]))
                assert rel_err(Vu[it, ic], vo) <= tol, (prec, it, ic)
        # the full V at every baseline: the group's value or its conjugate
        Vf = sim.simulate(w.lsts, w.freqs, prec).cpu().numpy()
        assert rel_err(expand(Vu, plan, w.n_ant, 1), Vf) <= 2 * tol


@pytest.mark.parametrize("redundant,tile_n", [(False, 128), (False, 256), (True, 128)])
def test_fused_schedule_matches_the_separate_one(redundant, tile_n):
    # several batches.  A non-redundant array's cover is the whole triangle:
    # there each HERK launch also builds the next batch's Z planes (fused
    # schedule, no Z-build launch after the first batch); a smaller cover
    # keeps the Z build in its own launches.  One HERK configuration, so the
    # schedules sum in the same order.
    w = synth.hera_like(n_ant=250 if redundant else 120, n_src=6000, n_chan=4, n_times=2, n_za=46, n_az=120)
    if not redundant:
        w.enu = synth.square_array(120, 300.0, np.random.default_rng(5))
    plan = redundancy_plan(w.enu, None, 1e-3, 1, 128)
    assert (plan["kind"] == 0) == (not redundant)
    out, n_launch = {}, {}
    for fuse in (True, False):
        sim = simulator(w, max_batch=2, herk_tile_n=tile_n, herk_split=2, fuse_zbuild=fuse)
        sim.set_redundancy(1e-3)
        out[fuse] = sim.simulate_unique(w.lsts, w.freqs, "fp16x3").cpu().numpy()
        n_launch[fuse] = sim.last_launch_count()
    # 4 batches: the fused schedule saves the Z-build launches of batches 1-3
    assert n_launch[False] - n_launch[True] == (0 if redundant else 3)
    assert np.array_equal(out[True], out[False])
    P = oracle_problem(w)
    for it, ic in ((0, 0), (1, 3)):
        vo = oracle.vis(P, w.lsts[it], w.freqs[ic], pairs=(plan["rep_a"], plan["rep_b"]))
        assert rel_err(out[True][it, ic], vo) <= 1e-5, (it, ic)


def test_two_feeds_and_a_polarised_sky():
    w = synth.polarised_diffuse(n_ant=100, nside=16, n_chan=2, n_times=2, n_za=31, n_az=72, lmax=40,
                                full_stokes=True)
    sim = simulator(w)
    n_u = sim.set_redundancy(1e-3)
    plan = redundancy_plan(w.enu, None, 1e-3, 2, 128)
    assert plan["kind"] in (1, 2)
    Vu = sim.simulate_unique(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    assert Vu.shape == (2, 2, n_u, 2, 2)
    P = oracle_problem(w)
    vo = oracle.vis(P, w.lsts[1], w.freqs[0], pairs=(plan["rep_a"], plan["rep_b"]))
    assert rel_err(Vu[1, 0], vo) <= 1e-5
    Vf = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    assert rel_err(expand(Vu, plan, w.n_ant, 2), Vf) <= 2e-5


def test_non_redundant_array_uses_the_triangle():
    w = synth.tiny(n_ant=10, n_src=1000, n_times=2)
    sim = simulator(w)
    n_u = sim.set_redundancy(1e-3)
    plan = redundancy_plan(w.enu, None, 1e-3, 1, 128)
    assert plan["kind"] == 0 and n_u == 10 * 9 // 2 + 1
    Vu = sim.simulate_unique(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    P = oracle_problem(w)
    for it in range(2):
        vo = oracle.vis(P, w.lsts[it], w.freqs[0], pairs=(plan["rep_a"], plan["rep_b"]))
        assert rel_err(Vu[it, 0], vo) <= 1e-5


def test_unique_output_state_and_arguments():
    w = synth.hera_like(n_ant=30, n_src=2000, n_chan=2, n_times=1, n_za=46, n_az=120)
    sim = simulator(w)
    sim.n_unique = 1  # no plan yet: the call is refused before it writes
    with pytest.raises(MatvisError, match="MV_ERR_STATE"):
        sim.simulate_unique(w.lsts, w.freqs, "fp16x3")
    sim.set_redundancy(1e-3)
    with pytest.raises(MatvisError, match="MV_ERR_ARG"):
        sim.simulate_unique(w.lsts, w.freqs, "fp32")
    # a new array drops the plan
    sim.set_antennas(w.enu, None, w.lat)
    with pytest.raises(MatvisError, match="MV_ERR_STATE"):
        sim.simulate_unique(w.lsts, w.freqs, "fp16x3")


@pytest.mark.parametrize("every,kinds", [(10, (2,)), (25, (1,)), (3, (0,))])
def test_two_beam_types_split_the_groups(every, kinds):
    # every n-th antenna has a second beam: groups need equal beam pairs, so a
    # reversed baseline between different beams joins only the group whose
    # beams are swapped to match; the cover is a block of either orientation,
    # or (with many such antennas) the whole triangle
    w = synth.hera_like(n_ant=250, n_src=5000, n_chan=2, n_times=1, n_za=46, n_az=120)
    grid = w.beam[1]
    g2 = (grid * np.complex64(0.7 - 0.2j)).astype(np.complex64)
    w.beam = ("grid", np.concatenate([grid, g2], axis=0)) + tuple(w.beam[2:])
    w.beam_idx = (np.arange(w.n_ant) % every == 0).astype(np.int32)
    sim = simulator(w)
    n_u = sim.set_redundancy(1e-3)
    plan = redundancy_plan(w.enu, w.beam_idx, 1e-3, 1, 128)
    one = redundancy_plan(w.enu, None, 1e-3, 1, 128)
    assert n_u == plan["n_unique"] > one["n_unique"] and plan["kind"] in kinds
    Vu = sim.simulate_unique(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    P = oracle_problem(w)
    vo = oracle.vis(P, w.lsts[0], w.freqs[1], pairs=(plan["rep_a"], plan["rep_b"]))
    assert rel_err(Vu[0, 1], vo) <= 1e-5
    Vf = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    assert rel_err(expand(Vu, plan, w.n_ant, 1), Vf) <= 2e-5
