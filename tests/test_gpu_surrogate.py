"""Learned beam: the GPU Fourier-feature MLP against the FP64 oracle MLP
(same weights), its training against the gridded beam, and simulation with
it (needs a GB300).

Stated bounds (BF16 operands and activations, FP32 accumulation: each layer
rounds its inputs to 8 significant bits, relative 2^-9):
  forward          max |y - y_oracle| <= 3e-2 max |y_oracle|
  gradients        cosine(g, g_oracle) >= 0.995, |g - g_oracle| <= 0.1 |g_oracle|
  visibilities     with the same network, max |V - V_oracle| <= 3e-2 max |V_oracle|
  trained beam     (64 frequencies, 4 x 256, 3000 steps of 8192 samples) on 12
                   per-antenna Jones grids: RMS |A_net - A_grid| <= 0.06 RMS |A_grid|
                   (measured 0.026-0.044) and visibilities within 0.08 of the
                   gridded path's (measured 0.033-0.035)
  gain             on 350 per-antenna Jones grids the network holds >= 500x less
                   device memory than the grids; the gridded path stays within
                   1e-5 of the oracle and the network within 0.08
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from helpers import flat_grads, oracle_net, oracle_problem, rel_err, sample_pairs, simulator
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu
SMALL = dict(n_freq=16, emb_dim=4, width=64, depth=2, sigma_az=2.0, sigma_za=2.0, sigma_nu=1.0)


def workload(n_ant=12, n_src=2000):
    return synth.learned_beam(n_ant=n_ant, n_src=n_src, n_chan=2, n_times=1, n_za=31, n_az=72, dnu=4e6)


def grid_meta(w):
    g = w.beam
    return g[2], g[3], g[1].shape[3]


def points(n, n_beam, seed, w):
    nu0, dnu, n_nu = grid_meta(w)
    r = np.random.default_rng(seed)
    return (r.integers(0, n_beam, n).astype(np.int32), r.uniform(0, 2 * np.pi, n), r.uniform(0, np.pi / 2, n),
            r.uniform(nu0 + dnu, nu0 + (n_nu - 3) * dnu, n))


def test_forward_matches_oracle_network():
    w = workload()
    sim = simulator(w)
    sim.surrogate_create(**SMALL)
    beam, az, za, nu = points(1024, w.n_ant, 1, w)
    y = sim.surrogate_eval(beam, az, za, nu)
    yo = mlp.forward(oracle_net(sim, *grid_meta(w)), beam, az, za, nu)
    assert y.shape == yo.shape == (1024, 8)
    assert np.abs(y - yo).max() <= 3e-2 * np.abs(yo).max()


def test_gradients_match_oracle_network():
    w = workload()
    sim = simulator(w)
    sim.surrogate_create(**SMALL)
    beam, az, za, nu = points(512, w.n_ant, 2, w)
    t = np.random.default_rng(3).normal(size=(512, 8)).astype(np.float32)
    g, loss = sim.surrogate_grad(beam, az, za, nu, t)
    net = oracle_net(sim, *grid_meta(w))
    lo, go = mlp.loss_and_grads(net, beam, az, za, nu, t.astype(np.float64))
    go = flat_grads(sim, go)
    assert abs(loss - lo) <= 1e-2 * lo
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.995, cos
    assert np.linalg.norm(g - go) <= 0.1 * np.linalg.norm(go)


@pytest.mark.parametrize("n, cfg", [
    # the fused training pass (one launch for features, forward, loss and input
    # gradients): the default 4 x 256 network, a batch of 7 full 128-row tiles
    # and a ragged one
    (1000, dict()),
    # a width that is not a multiple of 64: the product-by-product path
    (600, dict(n_freq=16, emb_dim=8, width=80, depth=3)),
    # the fused pass at its edges: one full tile plus 8 rows, width 128, one
    # hidden layer, 24 frequencies (sine and cosine chunks unevenly spread);
    # width 192 and the deepest fused network (5 layers: 6 weight-gradient
    # products in one launch); exactly one tile
    (136, dict(n_freq=24, emb_dim=8, width=128, depth=1)),
    (304, dict(n_freq=32, emb_dim=16, width=192, depth=5)),
    (128, dict()),
])
def test_gradients_match_oracle_network_shapes(n, cfg):
    w = workload()
    sim = simulator(w)
    sim.surrogate_create(**cfg)
    beam, az, za, nu = points(n, w.n_ant, 5, w)
    t = np.random.default_rng(6).normal(size=(n, 8)).astype(np.float32)
    g, loss = sim.surrogate_grad(beam, az, za, nu, t)
    net = oracle_net(sim, *grid_meta(w))
    lo, go = mlp.loss_and_grads(net, beam, az, za, nu, t.astype(np.float64))
    go = flat_grads(sim, go)
    assert abs(loss - lo) <= 1e-2 * lo
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.995, cos
    assert np.linalg.norm(g - go) <= 0.1 * np.linalg.norm(go)


def test_training_fits_the_gridded_beams():
    w = workload()
    sim = simulator(w)
    sim.surrogate_create()
    l0, l1 = sim.surrogate_train(steps=3000, batch=8192, lr0=2e-3, lr1=1e-5, seed=7)
    assert l1 < 0.05 * l0, (l0, l1)
    beam, az, za, nu = points(2000, w.n_ant, 4, w)
    y = sim.surrogate_eval(beam, az, za, nu)
    P = oracle_problem(w)
    # grid values at the same points (oracle interpolation, one call per point frequency)
    A = np.stack([oracle.beam_eval(P, [az[i]], [za[i]], nu[i])[beam[i], :, :, 0].ravel() for i in range(400)])
    Y = y[:400, 0::2] + 1j * y[:400, 1::2]
    assert np.sqrt(np.mean(np.abs(Y - A) ** 2)) <= 0.06 * np.sqrt(np.mean(np.abs(A) ** 2))


def test_simulate_with_the_surrogate_matches_oracle_with_same_network(tmp_path):
    w = workload(n_ant=12, n_src=3000)
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=3000, batch=8192, lr0=2e-3, lr1=1e-5, seed=9)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    for prec in ("fp32", "fp16x3"):
        V = sim.simulate(w.lsts, w.freqs, prec).cpu().numpy()
        P = oracle_problem(w)
        for ic, f in enumerate(w.freqs):
            def beam_fn(az, za, nu):
                n = az.size
                out = np.empty((w.n_ant, 2, 2, n), dtype=np.complex128)
                for b in range(w.n_ant):
                    y = mlp.forward(net, np.full(n, b), az, za, np.full(n, nu))
                    out[b] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
                return out
            Vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn)
            assert rel_err(V[0, ic], Vo) <= 3e-2, (prec, ic)
    # the learned beam against the gridded one (its modelling error), reported as a bound
    sim.set_beam_surrogate(False)
    Vg = sim.simulate(w.lsts, w.freqs, "fp32").cpu().numpy()
    assert rel_err(V, Vg) <= 0.08
    # save / load round trip
    path = tmp_path / "beam.mvmlp"
    y0 = sim.surrogate_eval([0, 5], [0.3, 1.0], [0.2, 0.7], [150e6, 160e6])
    sim.surrogate_save(path)
    sim2 = simulator(w)
    sim2.surrogate_load(path, **sim._mlp)
    assert np.array_equal(sim2.surrogate_eval([0, 5], [0.3, 1.0], [0.2, 0.7], [150e6, 160e6]), y0)


def test_surrogate_with_a_polarised_sky():
    # the tensor-core forward pass applies the coherency square root to the
    # network's Jones terms (eq. "fullz"); same network on both sides
    w = workload(n_ant=12, n_src=3000)
    g = np.random.default_rng(5)
    d = g.normal(size=(3, w.n_src))
    w.stokes_quv = d * (0.5 * g.uniform(0, 1, w.n_src) * w.flux_ref / np.linalg.norm(d, axis=0))
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=300, batch=8192, lr0=2e-3, lr1=1e-5, seed=3)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    P = oracle_problem(w)
    for ic, f in enumerate(w.freqs):
        def beam_fn(az, za, nu):
            n = az.size
            out = np.empty((w.n_ant, 2, 2, n), dtype=np.complex128)
            for b in range(w.n_ant):
                y = mlp.forward(net, np.full(n, b), az, za, np.full(n, nu))
                out[b] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
            return out
        Vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn)
        assert rel_err(V[0, ic], Vo) <= 3e-2, ic
    # and the polarisation matters at this level
    P.stokes_quv = None
    Vu = oracle.vis_with_beam_fn(P, w.lsts[0], w.freqs[0], beam_fn)
    assert rel_err(V[0, 0], Vu) > 0.02


@pytest.mark.parametrize("polarised", [False, True])
def test_surrogate_several_tiles_per_sm(polarised):
    # 48 beams x ~3000 live sources: ~570 tiles of 256 network rows (8 beams x
    # 32 sources), several per persistent CTA, so each CTA carries a tile's
    # gathered source data and the next tile's C rows across the tile boundary
    w = workload(n_ant=48, n_src=6000)
    if polarised:
        g = np.random.default_rng(8)
        d = g.normal(size=(3, w.n_src))
        w.stokes_quv = d * (0.6 * g.uniform(0, 1, w.n_src) * w.flux_ref / np.linalg.norm(d, axis=0))
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=200, batch=8192, lr0=2e-3, lr1=1e-5, seed=4)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    live = int(sim.last_live_counts(len(w.lsts) * len(w.freqs))[0])
    assert w.n_ant * live > 3 * 152 * 256
    P = oracle_problem(w)
    f = w.freqs[1]

    def beam_fn(az, za, nu):
        n = az.size
        out = np.empty((w.n_ant, 2, 2, n), dtype=np.complex128)
        for b in range(w.n_ant):
            y = mlp.forward(net, np.full(n, b), az, za, np.full(n, nu))
            out[b] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
        return out
    Vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn)
    assert rel_err(V[0, 1], Vo) <= 3e-2


@pytest.mark.parametrize("n_ant,cfg", [
    # one hidden layer: the fused pass goes from h_1 = relu(P + C) straight to
    # the output layer; width 128 (two 64-column halves per warp)
    (13, dict(n_freq=16, emb_dim=8, width=128, depth=1)),
    # width 128 with three hidden layers; 13 beams: a partly filled 8-beam group
    (13, dict(n_freq=24, emb_dim=8, width=128, depth=3)),
])
def test_simulate_with_other_network_shapes(n_ant, cfg):
    w = workload(n_ant=n_ant, n_src=3000)
    sim = simulator(w)
    sim.surrogate_create(**cfg)
    sim.surrogate_train(steps=100, batch=4096, lr0=2e-3, lr1=1e-4, seed=2)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    live = int(sim.last_live_counts(len(w.lsts) * len(w.freqs))[0])
    assert live % 32 != 0  # a partly filled 32-source block
    P = oracle_problem(w)
    f = w.freqs[0]

    def beam_fn(az, za, nu):
        n = az.size
        out = np.empty((w.n_ant, 2, 2, n), dtype=np.complex128)
        for b in range(w.n_ant):
            y = mlp.forward(net, np.full(n, b), az, za, np.full(n, nu))
            out[b] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
        return out
    Vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn)
    assert rel_err(V[0, 0], Vo) <= 3e-2


def test_surrogate_edge_cases():
    # the learned beam with no live source (every instance's WA and V zero)
    # and with one live source (a 32-source block holding one valid row)
    w = workload(n_ant=12, n_src=2000)
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=100, batch=4096, lr0=2e-3, lr1=1e-4, seed=8)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    lst, f = float(w.lsts[0]), float(w.freqs[0])
    sim.init_sky([0.0, 2.0], [np.pi / 3, np.pi / 3], [1.0, 3.0], nu_ref=w.nu_ref)  # never rises at HERA
    V = sim.simulate([lst], [f], "fp16x3").cpu().numpy()
    assert sim.last_live_counts(1)[0] == 0
    assert np.all(V == 0)
    ra, dec, flux = np.array([lst + 0.05]), np.array([w.lat + 0.1]), np.array([2.0])
    sim.init_sky(ra, dec, flux, nu_ref=w.nu_ref)
    V = sim.simulate([lst], [f], "fp16x3").cpu().numpy()[0, 0]
    assert sim.last_live_counts(1)[0] == 1
    P = oracle.Problem(ra=ra, dec=dec, flux_ref=flux, enu=w.enu, lat=w.lat, beam=("uniform",), nu_ref=w.nu_ref,
                       beam_idx=w.beam_idx)

    def beam_fn(az, za, nu):
        n = az.size
        out = np.empty((w.n_ant, 2, 2, n), dtype=np.complex128)
        for b in range(w.n_ant):
            y = mlp.forward(net, np.full(n, b), az, za, np.full(n, nu))
            out[b] = (y[:, 0::2] + 1j * y[:, 1::2]).T.reshape(2, 2, n)
        return out
    Vo = oracle.vis_with_beam_fn(P, lst, f, beam_fn)
    assert rel_err(V, Vo) <= 3e-2


def test_surrogate_of_one_unpolarised_beam():
    # every antenna on one single-feed, single-axis gridded beam: the network
    # has one embedding row and 2 outputs (one complex gain), so a tile holds 1
    # beam of its 8 and one WA component per row
    w = synth.hera_like(n_ant=20, n_src=3000, n_chan=2, n_times=1)
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=3000, batch=8192, lr0=2e-3, lr1=1e-5, seed=6)
    net = oracle_net(sim, *grid_meta(w))
    sim.set_beam_surrogate(True)
    V = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    P = oracle_problem(w)

    def beam_fn(az, za, nu):
        y = mlp.forward(net, np.zeros(az.size, dtype=np.int64), az, za, np.full(az.size, nu))
        return (y[:, 0] + 1j * y[:, 1]).reshape(1, 1, 1, az.size)
    for ic, f in enumerate(w.freqs):
        Vo = oracle.vis_with_beam_fn(P, w.lsts[0], f, beam_fn)
        assert rel_err(V[0, ic], Vo) <= 3e-2, ic
    # and the network stands in for the grid
    sim.set_beam_surrogate(False)
    Vg = sim.simulate(w.lsts, w.freqs, "fp16x3").cpu().numpy()
    assert rel_err(V, Vg) <= 0.08  # measured 0.025


def test_what_the_surrogate_gains_over_per_antenna_grids():
    # Sec. 3.1: with a beam per antenna the interpolation step holds and reads
    # one grid per antenna.  On 350 per-antenna Jones beams (1 deg x 1 deg x
    # 1 MHz, 9 frequency nodes) the trained network stands in for all of them:
    # measured here are the device bytes each beam model holds, the time per
    # instance of each path, and each path's visibility error against the FP64
    # oracle (which interpolates the grids).
    import time
    import torch
    w = synth.learned_beam(n_ant=350, n_src=6000, n_chan=2, n_times=1, nu_lo=146e6, nu_hi=154e6)
    w.freqs = np.array([149.5e6, 150.5e6])
    sim = simulator(w)
    sim.surrogate_create()
    sim.surrogate_train(steps=2000, batch=16384, lr0=2e-3, lr1=1e-5, seed=11)
    V = {}
    ms = {}
    for path in ("grid", "surrogate"):
        sim.set_beam_surrogate(path == "surrogate")
        out = sim.simulate(w.lsts, w.freqs, "fp16x3")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            sim.simulate(w.lsts, w.freqs, "fp16x3", out=out)
        torch.cuda.synchronize()
        ms[path] = (time.perf_counter() - t0) / 3 / len(w.freqs) * 1e3
        V[path] = out.cpu().numpy()
    grid_bytes, sur_bytes = sim.beam_model_bytes()
    # memory: the gridded beams (350 x 2 x 2 x 9 x 91 x 360 complex64 plus the
    # per-channel planes, ~1.8 GB) against the network's ~1.5 MB
    assert grid_bytes >= 1.5e9 and sur_bytes <= 3e6
    assert grid_bytes >= 500 * sur_bytes
    # accuracy against the oracle's interpolation of the grids on sampled baselines
    P = oracle_problem(w)
    pa, pb = sample_pairs(w.n_ant, 150, seed=3)
    err = {}
    for ic, nu in enumerate(w.freqs):
        vo = oracle.vis(P, w.lsts[0], nu, pairs=(pa, pb))
        for path in V:
            vv = V[path][0, ic].reshape(w.n_ant, 2, w.n_ant, 2)[pa, :, pb, :]
            err[path] = max(err.get(path, 0.0), rel_err(vv, vo))
    assert err["grid"] <= 1e-5
    assert err["surrogate"] <= 0.08
    print(f"beam model bytes: grid {grid_bytes:.3e}, surrogate {sur_bytes:.3e} ({grid_bytes / sur_bytes:.0f}x); "
          f"ms per instance: grid {ms['grid']:.3f}, surrogate {ms['surrogate']:.3f}; "
          f"max rel err vs oracle: grid {err['grid']:.2e}, surrogate {err['surrogate']:.3f}")
