"""Redundant-baseline groups and the sub-matrix cover of their representatives
(Appendix A), host logic, no GPU: the groups against a brute-force grouping of
the baseline vectors written here, the cover against the representatives."""
import numpy as np
import pytest

from paper_2312_09763_gb300 import synth

redundancy_plan = pytest.importorskip("paper_2312_09763_gb300").redundancy_plan


def brute_groups(enu, beam, tol):
    """Baselines (a <= b) in row-major order; key = the baseline vector on a
    tol grid with the sign that makes its first nonzero component positive,
    and the beam pair in that orientation."""
    n = enu.shape[0]
    keys, flips = [], []
    for a in range(n):
        for b in range(a, n):
            q = tuple(int(v) for v in np.rint((enu[a] - enu[b]) / tol))
            nz = [v for v in q if v != 0]
            flip = bool(nz) and nz[0] < 0
            ba, bb = int(beam[a]), int(beam[b])
            keys.append((tuple(-v for v in q), bb, ba) if flip else (q, ba, bb))
            flips.append(flip)
    first = {}
    group = np.empty(len(keys), np.int64)
    conj = np.empty(len(keys), np.int8)
    rep_flip = []
    for i, k in enumerate(keys):
        if k not in first:
            first[k] = len(first)
            rep_flip.append(flips[i])
        group[i] = first[k]
        conj[i] = flips[i] != rep_flip[group[i]]
    return len(first), group, conj


def check_plan(enu, beam, tol, n_feed, tile_n):
    p = redundancy_plan(enu, beam, tol, n_feed, tile_n)
    n = enu.shape[0]
    n_u, group, conj = brute_groups(enu, np.zeros(n, int) if beam is None else beam, tol)
    assert p["n_unique"] == n_u
    assert np.array_equal(p["group_of"], group) and np.array_equal(p["conj_of"], conj)
    # representatives: the first member of each group (a <= b, row-major)
    a_of = np.concatenate([np.full(n - a, a) for a in range(n)])
    b_of = np.concatenate([np.arange(a, n) for a in range(n)])
    firsts = np.array([np.flatnonzero(group == g)[0] for g in range(n_u)])
    assert np.array_equal(p["rep_a"], a_of[firsts]) and np.array_equal(p["rep_b"], b_of[firsts])
    # the cover: a permutation, and every representative inside a block in the
    # plan's orientation (kind 0: the lower triangle, i.e. (row b, column a))
    perm = p["perm"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    if p["kind"] == 0:
        assert np.array_equal(perm, np.arange(n))
    else:
        r, c = (p["rep_a"], p["rep_b"]) if p["kind"] == 1 else (p["rep_b"], p["rep_a"])
        pr, pc = perm[r], perm[c]
        inside = np.zeros(n_u, bool)
        for r0, r1, c0, c1 in p["blocks"]:
            inside |= (pr >= r0) & (pr < r1) & (pc >= c0) & (pc < c1)
        assert inside.all()
        # its cost in 128 x tile_n tiles of the real Gram matrix
        cost = sum(-(-2 * n_feed * (r1 - r0) // 128) * -(-2 * n_feed * (c1 - c0) // tile_n)
                   for r0, r1, c0, c1 in p["blocks"])
        assert cost == p["tiles"] < p["tiles_full"]
    return p


@pytest.mark.parametrize("tile_n", [128, 256])
def test_hera_like_array_groups_and_cover(tile_n):
    w = synth.hera_like(n_src=10, n_chan=1, n_times=1)
    p = check_plan(w.enu, None, 1e-3, 1, tile_n)
    # a triangular lattice: a few hundred groups of the 61,425 baselines, and a
    # cover of at most half the tiles of the whole triangle
    assert 300 < p["n_unique"] < 2000 and p["kind"] in (1, 2)
    assert p["tiles"] <= p["tiles_full"] // 2


def test_beams_split_groups_and_feeds_scale_tiles():
    w = synth.hera_like(n_ant=60, n_src=10, n_chan=1, n_times=1)
    beam = (np.arange(60) % 2).astype(np.int32)
    p1 = check_plan(w.enu, None, 1e-3, 1, 256)
    p2 = check_plan(w.enu, beam, 1e-3, 1, 256)
    assert p2["n_unique"] > p1["n_unique"]
    check_plan(w.enu, beam, 1e-3, 2, 128)


def test_non_redundant_array_keeps_the_triangle():
    g = np.random.default_rng(4)
    enu = np.c_[g.uniform(-500, 500, (40, 2)), np.zeros(40)]
    p = check_plan(enu, None, 1e-3, 1, 256)
    # only the autocorrelations coincide (a vector and its reverse are one group)
    assert p["n_unique"] == 40 * 39 // 2 + 1 and p["kind"] == 0


def test_tolerance_merges_near_equal_vectors_and_rejects_bad_input():
    enu = np.array([[0.0, 0, 0], [14.6, 0, 0], [29.2004, 0, 0]])
    assert redundancy_plan(enu, tol_m=1e-2)["n_unique"] == 3    # autos, 14.6 m, 29.2 m
    assert redundancy_plan(enu, tol_m=1e-5)["n_unique"] == 4    # the two 14.6 m baselines differ by 0.4 mm
    from paper_2312_09763_gb300 import MatvisError
    with pytest.raises(MatvisError):
        redundancy_plan(enu, tol_m=0.0)
    with pytest.raises(MatvisError):
        redundancy_plan(np.array([[0.0, np.nan, 0.0]]))
