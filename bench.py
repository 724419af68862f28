"""Throughput benchmark: visibilities per second on the HERA-like workload.

One step = one full simulate call over the workload's 60 LSTs x 64 channels
(3840 (time, frequency) instances of 350 antennas x 1e5 sources: rotation,
horizon cut, beam interpolation, FP64-phase Z build and V = Z Z^H), inputs
already resident on the device.  vis = N_ant (N_ant + 1) / 2 baselines
(autocorrelations included) x channels x times.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp16x3|fp32]
                    [--impl ours|reference] [--workload hera|diffuse|uneven]

--workload diffuse times the polarised HEALPix sky (350 antennas, 196,608
pixels, 32 channels x 120 LSTs, 2 x 2 Jones beam) and --workload uneven the
256 random (LST, nu) pairs through mv_simulate_pairs; the default is the
HERA-like point-source workload above.

Under torchrun each rank simulates the full workload on its own GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) per instance of k_herk_tc<128> on the 350-antenna,
# 1e5-source workload in FP16x3: one ncu capture of 16 instances (2.4452 GB),
# summarised in profiles/k_herk_tc_350ant_1e5src_16ch.txt.
HERK_DRAM_BYTES_PER_INSTANCE = (2.4280e9 + 0.0172e9) / 16
# The same for the HERK launch that also builds the next batch's U planes
# (k_herk_tc<128, 2, 1, 1>) in the configuration the autotuner keeps on the
# 350-antenna workload (128 columns, split 4, flush 16): 2.5270 GB read +
# 2.3306 GB written for 16 + 16 instances (split-K partial tiles included),
# summarised in profiles/k_herk_tc_fused_zbuild_350ant_1e5src_2x16ch.txt.
FUSED_DRAM_BYTES_PER_INSTANCE = (2.5270e9 + 2.3306e9) / 16
# k_mlp_wa on the learned-beam sample (one launch = one instance of 350 beams x
# 50,013 live sources): 53.7 MB read + 500.0 MB written, summarised in
# profiles/k_mlp_wa_learned_350beams_1e5src.txt.
MLP_DRAM_BYTES_PER_LAUNCH = 53.68e6 + 499.97e6
# k_herk_tc<128> over the redundant-group cover of the same workload: 2.3149 GB
# read + 43.3 MB written for 16 instances, summarised in
# profiles/k_herk_tc_redundant_cover_350ant_1e5src_16ch.txt.
UNIQUE_DRAM_BYTES_PER_INSTANCE = (2.3149e9 + 0.0433e9) / 16
METRIC = "vis/s (bl·chan·time) at 350 ant×1e5 src; split-prec TC vs FP32 @1e-5 rel err"
UNIT = "vis/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="fp16x3", choices=["fp16x3", "fp32"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="small workload (profiling captures)")
    ap.add_argument("--small-lsts", type=int, default=1, help="LSTs of the small workload")
    ap.add_argument("--workload", default="hera", choices=["hera", "diffuse", "uneven", "learned"],
                    help="hera: 350 ant x 1e5 src x 64 ch x 60 t (default); diffuse: 350 ant x 196,608 HEALPix "
                         "pixels x 32 ch x 120 t, 2x2 Jones beam; uneven: 256 (LST, nu) pairs, one call; "
                         "learned: one LST x 8 channels of the learned-beam workload (350 per-antenna Jones "
                         "beams replaced by the trained surrogate)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--overlap", action="store_true", help="Z build / HERK overlap (mv_options.overlap_batches)")
    ap.add_argument("--unique", action="store_true",
                    help="one value per redundant baseline group (mv_simulate_unique, Appendix A); value counts "
                         "the baselines the groups represent")
    ap.add_argument("--max-batch", type=int, default=0, help="instances per launch (mv_options.max_batch; 0 = auto)")
    ap.add_argument("--sweep", action="store_true",
                    help="scaling sweep instead of the benchmark line: time per instance over sources 2^10..2^19 "
                         "x antennas 2^3..2^8 (one LST x 16 channels each), one JSON line per point")
    ap.add_argument("--train-steps", type=int, default=611,
                    help="learned workload: Adam steps (default 611 of 16384 samples, i.e. 1e7 samples)")
    ap.add_argument("--train-batch", type=int, default=16384, help="learned workload: samples per Adam step")
    ap.add_argument("--train-peak-batch", type=int, default=65536,
                    help="learned workload: batch of the training-throughput measurement (100 steps, learning rate 1e-12)")
    ap.add_argument("--no-fuse", action="store_true", help="Z build as its own launch (mv_options.fuse_zbuild = 0)")
    ap.add_argument("--herk-config", default=None, metavar="BN,SPLIT,FLUSH",
                    help="fix the tensor-core HERK tile width, split-K and flush interval (skips autotune)")
    ap.add_argument("--fp32-steps", type=int, default=2,
                    help="timed steps of the FP32 CUDA-core arm on the same workload (after one warm-up step; "
                         "0 skips it)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """Barrier and max-over-ranks on the host (gloo); a no-op at world size 1."""

    def __init__(self, world: int):
        self.world = world
        if world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


def workload(args):
    from paper_2312_09763_gb300 import synth
    if args.workload == "diffuse":
        return synth.polarised_diffuse()
    if args.workload == "uneven":
        return synth.batched_uneven()
    if args.workload == "learned" and args.small:
        # profiling captures: 2 channels, grids over 148-152 MHz (~1.1 GB)
        w = synth.learned_beam(n_chan=2, n_times=1, nu_lo=148e6, nu_hi=152e6)
        w.freqs = 149.5e6 + np.arange(2) * 1e6
        w.name = w.name.replace("x 2 ch x 1 t", "x 2 ch (149.5-150.5 MHz) x 1 t")
        return w
    if args.workload == "learned":
        # one LST x 8 channels (146.5-153.5 MHz) of the learned-beam workload;
        # per-antenna grids over 143-157 MHz cover the cubic stencil
        w = synth.learned_beam(n_chan=8, n_times=1, nu_lo=143e6, nu_hi=157e6)
        w.freqs = 146.5e6 + np.arange(8) * 1e6
        w.name = w.name.replace("x 8 ch x 1 t", "x 8 ch (146.5-153.5 MHz) x 1 t")
        return w
    if args.small:  # profiling captures: 16 channels of 1 LST of the full sky (~2.2 GB of Z planes)
        w = synth.hera_like(n_ant=350, n_src=100_000, n_chan=16, n_times=args.small_lsts)
        w.freqs = synth.hera_like().freqs[24:40]
        return w
    return synth.hera_like()


def n_instances(w, pairs: bool) -> int:
    return len(w.lsts) if pairs else len(w.lsts) * len(w.freqs)


def n_vis(w, pairs: bool = False) -> int:
    """Baselines (a >= b) x instances; a Jones beam's 2 x 2 feed products count once."""
    return w.n_ant * (w.n_ant + 1) // 2 * n_instances(w, pairs)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mv_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["bf16_tflops"], d["bf16_tflops_sustained"], d["hbm_gbs"], "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


def cpu_baseline(w, budget_pairs: int = None, keep: dict = None, min_seconds: float = 0.0, max_instances: int = 8):
    """The FP64 oracle as it stands, on the host cores: all baselines a >= b of
    one instance (LST 0, first channel) of the same workload, then of the next
    channels at LST 0 until min_seconds of oracle time have passed (at most
    max_instances).  keep (a dict): receives the oracle's V of the first
    instance's baselines and their (a, b) indices."""
    import oracle
    oracle.build()
    P = oracle.Problem(ra=w.ra, dec=w.dec, flux_ref=w.flux_ref, enu=w.enu, lat=w.lat,
                       beam=(w.beam[0], np.asarray(w.beam[1]).astype(np.complex128)) + tuple(w.beam[2:]),
                       spec_idx=w.spec_idx, nu_ref=w.nu_ref, beam_idx=w.beam_idx, stokes_quv=w.stokes_quv)
    a, b = np.tril_indices(w.n_ant)
    if budget_pairs is not None:
        a, b = a[:budget_pairs], b[:budget_pairs]
    cores = os.cpu_count() or 1
    dt, n_inst = 0.0, 0
    while n_inst < min(max_instances, len(w.freqs)) and (n_inst == 0 or dt < min_seconds):
        t0 = time.perf_counter()
        vo = oracle.vis(P, w.lsts[0], w.freqs[n_inst], pairs=(a, b), threads=cores)
        dt += time.perf_counter() - t0
        if n_inst == 0 and keep is not None:
            keep.update(V=vo, a=a, b=b)
        n_inst += 1
    f_last = w.freqs[n_inst - 1]
    chans = (f"{w.freqs[0] / 1e6:.4f} MHz" if n_inst == 1 else
             f"{n_inst} channels {w.freqs[0] / 1e6:.4f}-{f_last / 1e6:.4f} MHz")
    return {"value": n_inst * a.size / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{a.size} baselines (a >= b) of {n_inst} instance(s) (LST {w.lsts[0]:.4f} rad, {chans}) "
                      f"of the {w.n_ant}-antenna x {w.n_src}-source workload, FP64 direct sum, {dt:.1f} s"}


def max_rel_err(v0, keep: dict, nf: int) -> float:
    """max |V - V_oracle| / max |V_oracle| over the oracle's baselines of the
    first instance; v0 is the GPU's V of that instance, [N nf][N nf]."""
    a, b, vo = keep["a"], keep["b"], keep["V"]
    n = v0.shape[0] // nf
    v = v0.reshape(n, nf, n, nf)[a, :, b, :]
    return float(np.abs(v - vo).max() / np.abs(vo).max())


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same metric and workload."""
    if rank != 0:
        return
    w = workload(args)
    per_step = 2048
    for _ in range(args.warmup):
        cpu_baseline(w, budget_pairs=256)
    vals, t_all = [], 0.0
    for _ in range(args.steps):
        cb = cpu_baseline(w, budget_pairs=per_step)
        vals.append(cb["value"])
        t_all += per_step / cb["value"]
    value = per_step * args.steps / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "sample": f"{per_step} baselines of one instance per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} baselines (a >= b) of one instance per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep(args):
    """Runtime against catalogue size and array size (the shape of the paper's
    scaling tests, Sec. 4.3): HERA-like arrays of 2^3..2^8 antennas and uniform
    skies of 2^10..2^19 sources, one LST x 16 channels, FP16x3 (or --precision),
    CUDA events around warm simulate calls."""
    import torch
    from paper_2312_09763_gb300 import Simulator, synth
    torch.cuda.set_device(0)
    for lg_ant in range(3, 9):
        for lg_src in range(10, 20, 3):
            w = synth.hera_like(n_ant=2 ** lg_ant, n_src=2 ** lg_src, n_chan=16, n_times=1, n_za=46, n_az=120)
            sim = Simulator(0)
            sim.init_sky(w.ra, w.dec, w.flux_ref, w.spec_idx, w.nu_ref)
            sim.set_beam(w.beam)
            sim.set_antennas(w.enu, None, w.lat)
            V = torch.empty((1, 16, w.n_ant, w.n_ant), dtype=torch.complex64, device="cuda")
            for _ in range(3):
                sim.simulate(w.lsts, w.freqs, args.precision, out=V)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 10
            for _ in range(reps):
                sim.simulate(w.lsts, w.freqs, args.precision, out=V)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps / 16
            live = int(sim.last_live_counts(16)[0])
            print(json.dumps({"sweep": True, "n_ant": w.n_ant, "n_src": w.n_src, "live": live,
                              "precision": args.precision, "ms_per_instance": ms,
                              "vis_per_s": w.n_ant * (w.n_ant + 1) / 2 / (ms / 1e3)}), flush=True)
            sim.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweep:
        sweep(args)
        return
    import torch
    from paper_2312_09763_gb300 import Simulator
    d = Dist(world)
    torch.cuda.set_device(local)
    w = workload(args)
    pairs = args.workload == "uneven"
    hk = {}
    if args.herk_config:
        bn, split, flush = (int(x) for x in args.herk_config.split(","))
        hk = dict(herk_tile_n=bn, herk_split=split, herk_flush_kblocks=flush)
        args.no_autotune = True
    sim = Simulator(local, overlap_batches=args.overlap, max_batch=args.max_batch, fuse_zbuild=not args.no_fuse, **hk)
    sim.init_sky(w.ra, w.dec, w.flux_ref, w.spec_idx, w.nu_ref)
    sim.set_beam(w.beam)
    sim.set_antennas(w.enu, w.beam_idx, w.lat)
    n_unique = None
    if args.unique:
        if args.workload in ("uneven", "learned"):
            raise SystemExit("--unique: hera or diffuse workload")
        n_unique = sim.set_redundancy(1e-3)
        args.no_autotune = True  # the cover has its own tile list and configuration
    learned = None
    if args.workload == "learned":
        # no host round trip of the 5.5 GB of per-antenna grids each step, and
        # no CPU baseline over 350 per-antenna beams: device-side numbers only
        args.no_e2e = args.no_cpu_baseline = True
        # the surrogate of the 350 gridded beams: by default 611 Adam steps of 16384 samples (1e7 samples)
        sim.surrogate_create()
        p_init = sim.surrogate_params()[0].copy()
        # untimed: the work buffers and first launches, then back to the initial weights (and a fresh Adam)
        sim.surrogate_train(steps=3, batch=args.train_batch, lr0=1e-6, lr1=1e-6, seed=99)
        sim.surrogate_set_params(p_init)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l0, l1 = sim.surrogate_train(steps=args.train_steps, batch=args.train_batch, lr0=2e-3, lr1=1e-5, seed=1)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        # the gridded path's V on this sample (the surrogate's modelling error) and
        # its time per instance, against the surrogate's below
        tuning = None if args.precision == "fp32" or args.no_autotune else sim.autotune(w.lsts, w.freqs, args.precision)
        args.no_autotune = True
        Vg = sim.simulate(w.lsts, w.freqs, args.precision)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(2):
            sim.simulate(w.lsts, w.freqs, args.precision, out=Vg)
        g1.record()
        torch.cuda.synchronize()
        grid_ms = g0.elapsed_time(g1) / 2
        grid_bytes, sur_bytes = sim.beam_model_bytes()
        # training throughput at a large batch: the same training steps with a
        # vanishing learning rate (the trained network stays as it is); the
        # first call picks the SM split between the training launches and the
        # sampler
        pb = args.train_peak_batch
        sim.surrogate_train(steps=12, batch=pb, lr0=1e-12, lr1=0.0, seed=5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.surrogate_train(steps=100, batch=pb, lr0=1e-12, lr1=0.0, seed=6)
        torch.cuda.synchronize()
        t_peak = time.perf_counter() - t0
        sim.set_beam_surrogate(True)
        n_samp = args.train_steps * args.train_batch
        learned = {"train_samples": n_samp, "train_batch": args.train_batch, "train_s": t_train,
                   "train_samples_per_s": n_samp / t_train, "loss_first": l0, "loss_last": l1,
                   "train_peak_batch": pb, "train_peak_samples_per_s": 100 * pb / t_peak,
                   "grid_ms_per_instance": grid_ms / n_instances(w, pairs),
                   "grid_beam_bytes": grid_bytes, "surrogate_beam_bytes": sur_bytes}
    N = w.n_ant
    nf, nax = sim.n_feed, sim._n_ax()
    shape = (len(w.lsts), N * nf, N * nf) if pairs else (len(w.lsts), len(w.freqs), N * nf, N * nf)
    if n_unique is not None:
        shape = (len(w.lsts), len(w.freqs), n_unique, nf, nf)
    V = torch.empty(shape, dtype=torch.complex64, device=f"cuda:{local}")
    run = sim.simulate_pairs if pairs else (sim.simulate_unique if n_unique is not None else sim.simulate)
    stream = torch.cuda.current_stream()
    if learned is None:
        tuning = None
    if args.precision != "fp32" and not args.no_autotune:
        tuning = sim.autotune(w.lsts, w.freqs, args.precision, pairs=pairs)
    for _ in range(args.warmup):
        run(w.lsts, w.freqs, args.precision, out=V)
    torch.cuda.synchronize()
    live = sim.last_live_counts(n_instances(w, pairs))
    sim.profile_enable(True)
    clocks = Clocks(local)
    clocks.start()
    d.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        run(w.lsts, w.freqs, args.precision, out=V)
        launches += sim.last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = sim.profile_read()
    sim.profile_enable(False)
    sim.check_device_status()
    ms_max = d.max(ms)
    vis_step = n_vis(w, pairs)
    value = world * vis_step * args.steps / (ms_max / 1e3)

    # roofline of the dominant kernel (the HERK)
    burst, sustained, hbm, src = peaks()
    n_h, ms_h = prof["herk"]
    rows = 2 * N * nf
    K = live.astype(np.float64) * nax
    if args.precision == "fp32":
        roof = None
    else:
        # algorithmic flops of one step: three real products over the lower
        # triangle of the 2N x 2N real Gram matrix, for every instance
        flops_step = float(np.sum(3 * 2.0 * rows * (rows + 1) / 2 * K))
        achieved = flops_step * args.steps / (ms_h / 1e3) / 1e12
        # with the fused Z build (the schedule the autotuner timed faster, or
        # the default for a forced 128-column tile) the timed HERK launches
        # also write the next batch's U planes
        fused = not args.no_fuse and args.precision != "fp32" and nf == nax and \
            (bool(tuning.get("fused")) if tuning is not None else hk.get("herk_tile_n") == 128)
        traffic = None
        if args.workload == "hera" and not args.small and args.precision == "fp16x3" and tuning \
                and tuning.get("tile_n") == 128:
            per = FUSED_DRAM_BYTES_PER_INSTANCE if fused else HERK_DRAM_BYTES_PER_INSTANCE
            traffic = per * n_instances(w, pairs) / max(n_h / args.steps, 1)
        roof = {"bound": "tensor", "achieved": achieved, "peak": sustained, "unit": "TFLOP/s",
                "frac": achieved / sustained, "traffic": traffic, "traffic_unit": "B per launch",
                "kernel": "k_herk_tc" + (" (fused with the next batch's Z build)" if fused else ""),
                "launches": n_h, "avg_launch_ms": ms_h / max(n_h, 1),
                "peak_source": f"{src} bf16 sustained (kernel timed inside a long step)"}
        if fused:
            # its second bound: the U planes written (next batch) and read (this
            # batch) once each, hi + lo halves
            kpad = np.ceil(K / 256.0) * 256
            z_bytes = float(np.sum(rows * kpad * 4.0))
            roof["hbm_bytes_per_step"] = 2 * z_bytes
            roof["hbm_achieved_gbs"] = 2 * z_bytes * args.steps / (ms_h / 1e3) / 1e9
            roof["hbm_frac"] = roof["hbm_achieved_gbs"] / hbm
            roof["hbm_peak_gbs"] = hbm
    # the first instance's V, kept for its error against the oracle
    v_first = V[(0, 0) if not pairs else (0,)].cpu().numpy() if n_unique is None and learned is None else None
    fp32_arm = None
    if args.fp32_steps > 0 and args.precision != "fp32" and n_unique is None and learned is None:
        # the plain FP32 CUDA-core path on the same workload and buffers: the
        # split-precision tensor-core path's speed-up at the same 1e-5 target
        run(w.lsts, w.freqs, "fp32", out=V)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp32_steps):
            run(w.lsts, w.freqs, "fp32", out=V)
        f1.record(stream)
        torch.cuda.synchronize()
        ms32 = d.max(f0.elapsed_time(f1))
        v32 = world * vis_step * args.fp32_steps / (ms32 / 1e3)
        fp32_arm = {"value": v32, "unit": UNIT, "ms_per_step": ms32 / args.fp32_steps, "steps": args.fp32_steps,
                    "warmup": 1, "speedup_vs_fp32": value / v32,
                    "v_first": V[(0, 0) if not pairs else (0,)].cpu().numpy()}
    unique_info = None
    if n_unique is not None and roof is not None:
        # the redundant-group output: the HERK computes the cover's blocks only;
        # algorithmic work = the sub-matrix area (real rows) of Appendix A
        from paper_2312_09763_gb300 import redundancy_plan
        plan = redundancy_plan(w.enu, w.beam_idx, 1e-3, nf, 128)
        if plan["kind"] == 0:
            area = rows * (rows + 1) / 2
        else:
            area = float(sum(4 * nf * nf * (r1 - r0) * (c1 - c0) for r0, r1, c0, c1 in plan["blocks"]))
        flops_u = float(np.sum(3 * 2.0 * area * K))
        tflops = flops_u * args.steps / (ms_h / 1e3) / 1e12
        # the cover's few tiles per instance read each U plane from HBM about
        # once: that read (hi + lo halves) is the bound that binds here
        kpad = np.ceil(K / 256.0) * 256
        u_bytes = float(np.sum(rows * kpad * 4.0))
        n_launch = max(n_h / args.steps, 1)
        gbs = u_bytes * args.steps / (ms_h / 1e3) / 1e9
        traffic = None
        if args.workload == "hera" and not args.small and args.precision == "fp16x3":
            traffic = UNIQUE_DRAM_BYTES_PER_INSTANCE * n_instances(w, pairs) / n_launch
        roof.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "traffic": traffic, "kernel": "k_herk_tc over the redundant-group cover",
                     "peak_source": f"{src} HBM copy rate",
                     "algorithmic_bytes_per_launch": u_bytes / n_launch,
                     "tensor_achieved_tflops": tflops, "tensor_frac": tflops / sustained})
        for k in ("hbm_bytes_per_step", "hbm_achieved_gbs", "hbm_frac", "hbm_peak_gbs"):
            roof.pop(k, None)
        unique_info = {"n_unique": n_unique, "cover_kind": plan["kind"], "cover_blocks": plan["blocks"].tolist(),
                       "cover_tiles": plan["tiles"], "triangle_tiles": plan["tiles_full"],
                       "unique_vis_per_s": world * n_unique * nf * nf * n_instances(w, pairs) * args.steps
                       / (ms_max / 1e3)}
    if learned is not None:
        # the surrogate's forward pass dominates: one row of the network per
        # (antenna beam, live source) of each instance.  The first layer's
        # Fourier part is the same for every beam and is computed once per
        # live source (k_src_first); the rest of the network per row (k_mlp_wa)
        _, _, lay = sim.surrogate_params()
        F, E, H, D = (sim._mlp[k] for k in ("n_freq", "emb_dim", "width", "depth"))
        d0p = int(lay[-1])
        macs_row = (D - 1) * H * H + H * 8
        macs_src = 2 * F * H
        rows_step = float(np.sum(live.astype(np.float64) * w.n_ant))
        src_step = float(np.sum(live.astype(np.float64)))
        n_b, ms_b = prof["beam"]
        mlp_tf = 2.0 * (macs_row * rows_step + macs_src * src_step) * args.steps / (ms_b / 1e3) / 1e12
        err = float((V - Vg).abs().max() / Vg.abs().max())
        learned.update({"network_rows_per_step": rows_step, "flop_per_row": 2 * macs_row,
                        "flop_per_source": 2 * macs_src,
                        "flop_per_row_unshared": 2 * (d0p * H + (D - 1) * H * H + H * 8),
                        "surrogate_vs_grid_rel_err": err,
                        "surrogate_ms_per_instance": ms_max / args.steps / n_instances(w, pairs)})
        roof = {"bound": "tensor", "achieved": mlp_tf, "peak": sustained, "unit": "TFLOP/s",
                "frac": mlp_tf / sustained,
                "traffic": MLP_DRAM_BYTES_PER_LAUNCH, "traffic_unit": "B per launch",
                "kernel": "k_mlp_wa (learned-beam forward + WA, tcgen05; FLOPs as executed, with k_src_first)",
                "launches": n_b, "avg_launch_ms": ms_b / max(n_b, 1),
                "peak_source": f"{src} bf16 sustained (kernels timed inside a long step)"}
    metric = METRIC if n_unique is None else \
        "vis/s (bl·chan·time) represented by one value per redundant baseline group (Appendix A)"
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": w.name, "instances_per_step": n_instances(w, pairs),
                       "live_sources_mean": float(live.mean()), "precision": args.precision,
                       "l2": "inputs larger than L2: Z planes of one batch ~4.5 GB, re-streamed each step",
                       "parallelism": f"{world} replica(s), instances simulated independently"},
            "gpu_launches": launches, "roofline": roof, "clocks": clk, "herk_tuning": tuning, "learned_beam": learned,
            "redundant_groups": unique_info,
            # two feeds: every baseline carries n_feed^2 polarisation products
            "pol_products_per_s": value * nf * nf if nf > 1 else None,
            "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()}}

    if rank == 0 and not args.no_e2e:
        # end to end through the public API: model inputs from pinned host
        # memory each step (sky, beam, antennas), V back to pinned host memory
        pinned_keep = []

        def pinned(x):  # a page-locked copy, as a numpy view
            t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
            pinned_keep.append(t)
            return t.numpy()
        ra, dec, fl = (pinned(np.asarray(x, dtype=np.float64)) for x in (w.ra, w.dec, w.flux_ref))
        si = None if w.spec_idx is None else pinned(np.asarray(w.spec_idx, dtype=np.float64))
        beam = w.beam
        if beam[0] == "grid":
            beam = (beam[0], pinned(np.asarray(beam[1], dtype=np.complex64))) + tuple(beam[2:])
        enu = pinned(w.enu)
        Vh = torch.empty(tuple(V.shape), dtype=torch.complex64).pin_memory()
        h2d = sum(x.nbytes for x in (ra, dec, fl, enu)) + (0 if si is None else si.nbytes) + \
            (beam[1].nbytes if beam[0] == "grid" else 0)
        d2h = Vh.numel() * 8
        def e2e_step():
            sim.init_sky(ra, dec, fl, si, w.nu_ref)
            sim.set_beam(beam)
            sim.set_antennas(enu, None, w.lat)
            if n_unique is not None:
                sim.set_redundancy(1e-3)  # the plan belongs to the antennas just set
            run(w.lsts, w.freqs, args.precision, out=Vh, host=True)
        e2e_step()  # warm-up: the host-output staging buffer and its captured launch sequence
        e2e_steps = max(1, min(args.steps, 3))
        times = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            e2e_step()
            times.append(time.perf_counter() - t0)
        dt = sum(times)
        line["e2e"] = {"value": vis_step * e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "ms_per_step": [round(1e3 * x, 2) for x in times],
                       "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}
    if fp32_arm is not None:
        line["fp32_value"] = fp32_arm["value"]
        line["speedup_vs_fp32"] = fp32_arm["speedup_vs_fp32"]
        line["fp32_arm"] = {k: v for k, v in fp32_arm.items() if k != "v_first"}
    if rank == 0 and not args.no_cpu_baseline:
        keep = {}
        line["cpu_baseline"] = cpu_baseline(w, keep=keep, min_seconds=10.0)
        if v_first is not None:
            # accuracy of this run against the FP64 oracle on every baseline of
            # the first instance (LST 0, first channel)
            line["max_rel_err"] = max_rel_err(v_first, keep, nf)
            line["max_rel_err_sample"] = (f"{keep['a'].size} baselines (a >= b) x {nf * nf} feed products of the "
                                          f"first instance, against the FP64 oracle")
            if fp32_arm is not None:
                line["fp32_arm"]["max_rel_err"] = max_rel_err(fp32_arm["v_first"], keep, nf)
    if rank == 0:
        print(json.dumps(line), flush=True)
    d.close()


if __name__ == "__main__":
    main()
