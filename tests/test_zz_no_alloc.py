"""The allocation-free horizon cut (mv_horizon_cull_static) against the
regular path (needs a GB300).

Callers that cannot allocate device memory when they run this step (hosts
whose device memory all belongs to a framework's pool, latency-critical loops
that cannot take cudaMalloc's device synchronisation) use
mv_horizon_cull_static, whose scratch is a static device array.  Its live
count must equal the regular simulate path's (an integer decision:
bit-exact), its live list must be the catalogue indices with Up > 0 in order,
its East-North-Up and (az, za) outputs must match the oracle's, and two calls
in a row must agree.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import simulator
from paper_2312_09763_gb300 import synth

pytestmark = pytest.mark.gpu


def test_static_cull_matches_regular_path_twice():
    import torch
    from paper_2312_09763_gb300 import binding
    lib = binding.load_library()
    w = synth.hera_like(n_ant=20, n_src=100_000, n_chan=1, n_times=3, n_za=31, n_az=60)
    lsts = np.array([0.3, 2.9])
    # regular path: live counts through mv_simulate / mv_last_live_counts
    sim = simulator(w)
    sim.simulate(lsts, w.freqs, "fp32")
    want_counts = sim.last_live_counts(len(lsts))
    xeq = torch.from_numpy(np.ascontiguousarray(oracle.xeq(w.ra, w.dec).T)).cuda()   # [3][n_src]
    n = w.n_src
    for call, lst in enumerate(np.concatenate([lsts, lsts])):   # two calls in a row per LST
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        enu = torch.zeros((3, n), dtype=torch.float64, device="cuda")
        azza = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        nl = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        st = torch.cuda.current_stream().cuda_stream or 1
        rc = lib.mv_horizon_cull_static(n, ctypes.c_void_p(xeq.data_ptr()), float(lst), float(w.lat),
                                        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(enu.data_ptr()),
                                        ctypes.c_void_p(azza.data_ptr()), ctypes.c_void_p(nl.data_ptr()),
                                        ctypes.c_void_p(st))
        assert rc == 0, lib.mv_last_error().decode()
        torch.cuda.synchronize()
        k = int(nl.item())
        assert k == want_counts[call % 2]
        enu_o = oracle.to_topo(oracle.rotation(lst, w.lat), oracle.xeq(w.ra, w.dec))
        live = np.nonzero(enu_o[:, 2] > 0)[0]
        assert np.array_equal(idx[:k].cpu().numpy(), live)
        assert np.abs(enu[:, :k].cpu().numpy().T - enu_o[live]).max() < 1e-15
        # (az, za) in FP32: za directly, az through the horizontal direction it
        # names (sin za weights it, since az is undefined at the zenith)
        az_o, za_o = oracle.azza(enu_o[live])
        got = azza[:k].cpu().numpy().astype(np.float64)
        assert np.abs(got[:, 1] - za_o).max() < 1e-6
        daz = np.angle(np.exp(1j * (got[:, 0] - az_o)))
        assert np.abs(daz * np.sin(za_o)).max() < 1e-6
        assert np.all((got[:, 0] >= 0) & (got[:, 0] <= 2 * np.pi))


def test_static_cull_rejects_sizes_beyond_its_maximum():
    from paper_2312_09763_gb300 import binding
    lib = binding.load_library()
    dummy = ctypes.c_void_p(16)
    rc = lib.mv_horizon_cull_static(2_097_153, dummy, 0.0, 0.0, dummy, dummy, dummy, dummy, None)
    assert rc == 1 and b"2097152" in lib.mv_last_error()
    # a latitude the regular path refuses is refused here too
    rc = lib.mv_horizon_cull_static(1000, dummy, 0.0, 1.6, dummy, dummy, dummy, dummy, None)
    assert rc == 1 and b"latitude" in lib.mv_last_error()
