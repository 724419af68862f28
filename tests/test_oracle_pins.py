"""Pins of the FP64 oracle against closed forms and invariants (no GPU).

The paper prints no numeric visibilities, so the oracle is pinned by what the
mathematics fixes: the rotation of eq. "rotation", the single-zenith-source
and east-west-fringe closed forms, Hermitian symmetry, the outer-product
identity of eq. "zz", the Keys kernel values, interpolation exactness and
convergence, linearity, translation invariance and redundancy.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2312_09763_gb300 import synth

DEG = np.pi / 180
C = 299792458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(n_ant=6, n_src=300, beam=("gaussian", 10 * DEG), seed=3, spec=True):
    g = np.random.default_rng(seed)
    enu = np.zeros((n_ant, 3))
    enu[:, :2] = g.uniform(-30, 30, size=(n_ant, 2))
    enu[:, 2] = g.uniform(-0.5, 0.5, size=n_ant)
    ra = g.uniform(0, 2 * np.pi, n_src)
    dec = np.arcsin(g.uniform(-1, 1, n_src))
    flux = g.uniform(0.1, 10, n_src)
    si = g.normal(-0.8, 0.2, n_src) if spec else None
    return oracle.Problem(ra=ra, dec=dec, flux_ref=flux, enu=enu, lat=-30.7 * DEG, beam=beam,
                          spec_idx=si, nu_ref=150e6)


def grid_beam(n_feed=1, n_ax=1, n_nu=8, n_za=31, n_az=72, fn=None, interp="cubic", nu0=140e6, dnu=2e6):
    dza = (np.pi / 2) / (n_za - 1)
    daz = 2 * np.pi / n_az
    nu = nu0 + dnu * np.arange(n_nu)
    za = dza * np.arange(n_za)
    az = daz * np.arange(n_az)
    NU, ZA, AZ = np.meshgrid(nu, za, az, indexing="ij")
    vals = np.zeros((1, n_feed, n_ax, n_nu, n_za, n_az), dtype=np.complex128)
    for p in range(n_feed):
        for k in range(n_ax):
            vals[0, p, k] = fn(p, k, AZ, ZA, NU)
    return ("grid", vals, nu0, dnu, dza, daz, interp)


# ------------------------------------------------------------ rotation


@pytest.mark.parametrize("lst,lat", [(0.3, -30.7 * DEG), (4.0, 52 * DEG), (6.1, 0.0)])
def test_rotation_orthonormal(lst, lat):
    R = oracle.rotation(lst, lat)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15, rtol=0)
    assert abs(np.linalg.det(R) - 1.0) < 1e-15


def test_rotation_maps_meridian_at_latitude_to_zenith():
    for lst, lat in [(0.0, -30.7 * DEG), (1.234, 10 * DEG), (5.5, -80 * DEG)]:
        x = oracle.xeq([lst], [lat])
        enu = oracle.to_topo(oracle.rotation(lst, lat), x)[0]
        assert np.allclose(enu, [0, 0, 1], atol=1e-15)


def test_rotation_matches_hour_angle_formula():
    # textbook alt-az from hour angle h = LST - RA, written independently
    g = np.random.default_rng(0)
    ra = g.uniform(0, 2 * np.pi, 500)
    dec = np.arcsin(g.uniform(-1, 1, 500))
    for lst, lat in [(0.7, -30.7 * DEG), (3.3, 45 * DEG)]:
        h = lst - ra
        east = -np.cos(dec) * np.sin(h)
        north = np.cos(lat) * np.sin(dec) - np.sin(lat) * np.cos(dec) * np.cos(h)
        up = np.sin(lat) * np.sin(dec) + np.cos(lat) * np.cos(dec) * np.cos(h)
        enu = oracle.to_topo(oracle.rotation(lst, lat), oracle.xeq(ra, dec))
        assert np.abs(enu - np.stack([east, north, up], 1)).max() < 1e-14


def test_azza_convention():
    enu = np.array([[0, 1, 0], [1, 0, 0], [0, -1, 0], [-1, 0, 0], [0, 0, 1.0]])
    az, za = oracle.azza(enu)
    assert np.allclose(az[:4], [0, np.pi / 2, np.pi, 3 * np.pi / 2], atol=1e-15)
    assert np.allclose(za, [np.pi / 2] * 4 + [0], atol=1e-15)


def test_cull_count_matches_independent_up():
    p = small_problem(n_src=5000)
    for lst in [0.1, 2.0, 4.4]:
        h = lst - p.ra
        up = np.sin(p.lat) * np.sin(p.dec) + np.cos(p.lat) * np.cos(p.dec) * np.cos(h)
        assert oracle.count_live(p, lst) == int(np.sum(up > 0))


# ------------------------------------------------------------ closed forms


@pytest.mark.parametrize("beam", [("gaussian", 10 * DEG), ("uniform",)])
def test_single_zenith_source(beam):
    lst, lat = 1.1, -30.7 * DEG
    enu = np.zeros((5, 3))
    enu[:, :2] = np.random.default_rng(1).uniform(-40, 40, (5, 2))
    p = oracle.Problem(ra=[lst], dec=[lat], flux_ref=[3.5], enu=enu, lat=lat, beam=beam)
    V = oracle.vis(p, lst, 150e6)
    # V_ab = I A(0)^2 for every pair: A(0) = 1 for both beams
    assert np.abs(V - 3.5).max() < 1e-12


def test_single_zenith_source_grid_beam_jones():
    # constant Jones beam J: V^{pq} = I sum_k J_pk conj(J_qk)
    J = np.array([[0.9 + 0.1j, -0.2 + 0.05j], [0.15 - 0.3j, 0.8 + 0.0j]])
    beam = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU: J[p, k] + 0 * AZ)
    lst, lat = 0.4, -30.7 * DEG
    enu = np.zeros((3, 3))
    enu[:, 0] = [0, 14.6, 29.2]
    p = oracle.Problem(ra=[lst], dec=[lat], flux_ref=[2.0], enu=enu, lat=lat, beam=beam)
    V = oracle.vis(p, lst, 145e6).reshape(3, 2, 3, 2)
    want = 2.0 * J @ J.conj().T
    for a in range(3):
        for b in range(3):
            assert np.abs(V[a, :, b, :] - want).max() < 1e-12


def test_east_west_fringe_phase_and_rate():
    bl, nu, lat = 14.6, 150e6, -30.7 * DEG
    ra, dec = 1.0, -20 * DEG
    enu = np.array([[0, 0, 0], [bl, 0, 0.0]])
    p = oracle.Problem(ra=[ra], dec=[dec], flux_ref=[1.7], enu=enu, lat=lat, beam=("uniform",))
    lsts = ra + np.linspace(-0.5, 0.5, 11)
    v = np.array([oracle.vis(p, t, nu, pairs=([0], [1]))[0, 0, 0] for t in lsts])
    # b_01 = x_0 - x_1 = (-bl, 0, 0) and East = cos(dec) sin(ra - LST), so
    # V_01 = I exp(-2 pi i (nu/c) b_01 . s) = I exp(+2 pi i (nu/c) bl cos(dec) sin(ra - LST))
    want = 1.7 * np.exp(2j * np.pi * (nu / C) * bl * np.cos(dec) * np.sin(ra - lsts))
    assert np.abs(v - want).max() < 1e-12
    # fringe rate d(phase)/dLST = -2 pi (nu / c) bl cos(dec) cos(ra - LST)
    t0, dt = ra + 0.2, 1e-6
    ph = [np.angle(oracle.vis(p, t, nu, pairs=([0], [1]))[0, 0, 0]) for t in (t0 - dt, t0 + dt)]
    rate = (ph[1] - ph[0]) / (2 * dt)
    assert abs(rate + 2 * np.pi * (nu / C) * bl * np.cos(dec) * np.cos(ra - t0)) < 1e-6


# ------------------------------------------------------------ invariants


def test_hermitian_real_nonnegative_autos():
    p = small_problem()
    V = oracle.vis(p, 0.9, 150e6)
    assert np.abs(V - V.conj().T).max() <= 1e-14 * np.abs(V).max()
    assert np.all(np.diag(V).imag == 0) or np.abs(np.diag(V).imag).max() < 1e-14 * np.abs(V).max()
    assert np.all(np.diag(V).real >= 0)


@pytest.mark.parametrize("beam", [("gaussian", 20 * DEG), "grid_jones"])
def test_direct_sum_equals_outer_product(beam):
    if beam == "grid_jones":
        beam = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU:
                         (np.cos(ZA) * np.cos(AZ + 0.3 * p) + 0.2j * k) * np.exp(-ZA ** 2) * (NU / 150e6))
    p = small_problem(n_ant=5, n_src=200, beam=beam)
    for lst in [0.2, 3.0]:
        Vd = oracle.vis(p, lst, 147.3e6)
        Vo = oracle.vis_outer(p, lst, 147.3e6)
        assert np.abs(Vd - Vo).max() <= 1e-12 * np.abs(Vo).max()


def test_linearity_in_flux_and_additivity():
    p = small_problem()
    V = oracle.vis(p, 1.3, 160e6)
    p2 = small_problem()
    p2.flux_ref = 2.5 * p.flux_ref
    assert np.abs(oracle.vis(p2, 1.3, 160e6) - 2.5 * V).max() <= 1e-13 * np.abs(V).max()
    half = p.ra.size // 2
    pa, pb = small_problem(), small_problem()
    pa.flux_ref = np.where(np.arange(p.ra.size) < half, p.flux_ref, 0.0)
    pb.flux_ref = np.where(np.arange(p.ra.size) >= half, p.flux_ref, 0.0)
    Vs = oracle.vis(pa, 1.3, 160e6) + oracle.vis(pb, 1.3, 160e6)
    assert np.abs(Vs - V).max() <= 1e-13 * np.abs(V).max()


def test_translation_invariance_far_from_origin():
    p = small_problem()
    V = oracle.vis(p, 2.2, 150e6)
    q = small_problem()
    q.enu = q.enu + np.array([10_000.0, -7_000.0, 3.0])
    Vq = oracle.vis(q, 2.2, 150e6)
    assert np.abs(Vq - V).max() <= 1e-10 * np.abs(V).max()


def test_redundant_baselines_equal():
    enu = synth.hex_array(19, 14.6)
    g = np.random.default_rng(5)
    ra = g.uniform(0, 2 * np.pi, 400)
    dec = np.arcsin(g.uniform(-1, 1, 400))
    p = oracle.Problem(ra=ra, dec=dec, flux_ref=g.uniform(0.1, 5, 400), enu=enu, lat=-30.7 * DEG,
                       beam=("gaussian", 15 * DEG))
    V = oracle.vis(p, 0.5, 150e6)
    groups = {}
    for a in range(19):
        for b in range(19):
            key = tuple(np.round(enu[a] - enu[b], 6))
            groups.setdefault(key, []).append((a, b))
    n_checked = 0
    for pairs in groups.values():
        vals = np.array([V[a, b] for a, b in pairs])
        assert np.abs(vals - vals[0]).max() <= 1e-11 * np.abs(V).max()
        n_checked += len(pairs) > 1
    assert n_checked > 10


def test_lst_period():
    p = small_problem()
    V0 = oracle.vis(p, 0.4, 150e6)
    V1 = oracle.vis(p, 0.4 + 2 * np.pi, 150e6)
    assert np.abs(V1 - V0).max() <= 1e-11 * np.abs(V0).max()


def test_flux_spectrum_power_law():
    lst, lat = 0.5, -30.7 * DEG
    p = oracle.Problem(ra=[lst], dec=[lat], flux_ref=[4.0], enu=np.zeros((2, 3)), lat=lat,
                       beam=("uniform",), spec_idx=[-0.7], nu_ref=150e6)
    for nu in [100e6, 150e6, 200e6]:
        assert abs(oracle.vis(p, lst, nu)[0, 1] - 4.0 * (nu / 150e6) ** -0.7) < 1e-12


# ------------------------------------------------------------ beams


def test_keys_kernel_golden():
    data = np.loadtxt(os.path.join(GOLDEN, "keys_kernel.txt"))
    for x, w in data:
        assert oracle.keys(x) == w


def test_gaussian_beam_half_width():
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=("gaussian", 10 * DEG))
    A = oracle.beam_eval(p, [0.0, 0.0, 0.0], [0.0, 5 * DEG, 10 * DEG], 150e6)[0, 0, 0]
    assert np.allclose(A.real, [1.0, 0.5, 0.5 ** 4], rtol=1e-14)


def test_grid_exact_at_nodes():
    beam = grid_beam(fn=lambda p, k, AZ, ZA, NU: np.sin(3 * AZ) * ZA + 1j * np.cos(ZA) * NU / 1e8)
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam)
    vals, nu0, dnu, dza, daz = beam[1], beam[2], beam[3], beam[4], beam[5]
    for (m, i, j) in [(2, 0, 0), (3, 5, 71), (5, 30, 13), (2, 17, 36)]:
        got = oracle.beam_eval(p, [j * daz], [i * dza], nu0 + m * dnu)[0, 0, 0, 0]
        assert abs(got - vals[0, 0, 0, m, i, j]) < 1e-15


@pytest.mark.parametrize("interp", ["cubic", "bilinear"])
def test_grid_reproduces_polynomials(interp):
    # Keys' kernel reproduces quadratics exactly in every axis; the bilinear
    # scheme reproduces linear functions in az and za.
    deg = 2 if interp == "cubic" else 1
    fn = lambda p, k, AZ, ZA, NU: (1.0 + 0.3 * AZ + 0.05 * AZ ** deg) * (2.0 - ZA + 0.4 * ZA ** deg) \
        * (1 + (NU - 150e6) / 1e7 + ((NU - 150e6) / 1e7) ** 2)
    beam = grid_beam(fn=fn, interp=interp)
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam)
    g = np.random.default_rng(2)
    az = g.uniform(0.5, 5.5, 50)       # away from the az wrap
    za = g.uniform(0.2, 1.3, 50)       # away from the pole and the last row
    for nu in [143.1e6, 150.0e6, 151.7e6]:
        got = oracle.beam_eval(p, az, za, nu)[0, 0, 0]
        want = fn(0, 0, az, za, nu)
        assert np.abs(got - want).max() < 1e-11


def test_grid_cubic_convergence_order():
    f = lambda AZ, ZA: np.exp(-(ZA / 0.5) ** 2) * (1 + 0.3 * np.sin(ZA) * np.cos(AZ))
    errs = []
    g = np.random.default_rng(4)
    az = g.uniform(0, 2 * np.pi, 400)
    za = g.uniform(0.05, 1.4, 400)
    for n_za, n_az in [(19, 72), (37, 144)]:
        beam = grid_beam(n_za=n_za, n_az=n_az, fn=lambda p, k, AZ, ZA, NU: f(AZ, ZA))
        p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam)
        errs.append(np.abs(oracle.beam_eval(p, az, za, 150e6)[0, 0, 0] - f(az, za)).max())
    assert 6.0 < errs[0] / errs[1] < 20.0


def test_pole_vector_components_flip_sign():
    # E-field of an x-directed dipole at the zenith: theta and phi components
    # cos(za) cos(az) and -sin(az).  Across the pole (theta, phi) flip sign,
    # so interpolation straight through the zenith stays smooth only if the
    # reflected stencil rows are negated.
    fn = lambda p, k, AZ, ZA, NU: np.cos(ZA) * np.cos(AZ) if k == 0 else -np.sin(AZ) + 0 * ZA
    beam = grid_beam(n_ax=2, n_za=46, n_az=180, fn=fn)
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam)
    az = np.linspace(0.1, 6.2, 40)
    za = np.full(40, 0.6 * DEG)
    A = oracle.beam_eval(p, az, za, 150e6)[0, 0]
    assert np.abs(A[0] - np.cos(za) * np.cos(az)).max() < 1e-4
    assert np.abs(A[1] + np.sin(az)).max() < 1e-4
    # the same theta component read as a single-axis beam (no flip) is wrong
    beam1 = grid_beam(n_ax=1, n_za=46, n_az=180, fn=lambda p, k, AZ, ZA, NU: np.cos(ZA) * np.cos(AZ))
    p1 = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam1)
    A1 = oracle.beam_eval(p1, az, za, 150e6)[0, 0, 0]
    assert np.abs(A1 - np.cos(za) * np.cos(az)).max() > 1e-2


def test_scalar_beam_even_in_za_is_exact_through_pole():
    fn = lambda p, k, AZ, ZA, NU: 1.0 - 0.7 * ZA ** 2 + 0 * AZ
    beam = grid_beam(fn=fn)
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((1, 3)), lat=0, beam=beam)
    az = np.linspace(0, 6.2, 30)
    za = np.full(30, 0.9 * DEG)
    A = oracle.beam_eval(p, az, za, 150e6)[0, 0, 0]
    assert np.abs(A - (1 - 0.7 * za ** 2)).max() < 1e-13


def test_frequency_outside_grid_rejected():
    beam = grid_beam(fn=lambda p, k, AZ, ZA, NU: 1 + 0 * AZ)
    p = oracle.Problem(ra=[0], dec=[0], flux_ref=[1], enu=np.zeros((2, 3)), lat=0, beam=beam)
    with pytest.raises(ValueError):
        oracle.vis(p, 0.0, 140.5e6)   # needs the node below 140 MHz


def test_hera_like_generator_shapes():
    w = synth.hera_like(n_ant=37, n_src=2000, n_chan=4, n_times=3, n_za=31, n_az=60)
    assert w.enu.shape == (37, 3) and np.all(w.enu[:, 2] == 0)
    d = np.linalg.norm(w.enu[:, None, :2] - w.enu[None, :, :2], axis=-1)
    assert abs(np.min(d[d > 0]) - 14.6) < 1e-9
    assert np.all((w.flux_ref >= 0.01) & (w.flux_ref <= 100))
    assert w.beam[1].shape == (1, 1, 1, 105, 31, 60)


def test_per_antenna_beam_index():
    # two unique constant beams (Sec. 3.1 beam indirection a_i -> iota):
    # a zenith source gives V_ab = I A_{beta(a)}(0) conj(A_{beta(b)}(0))
    g0, g1 = 0.8 + 0.2j, 0.5 - 0.4j
    beam = grid_beam(fn=lambda p, k, AZ, ZA, NU: 1 + 0 * AZ)
    vals = np.concatenate([beam[1] * g0, beam[1] * g1], axis=0)
    beam = ("grid", vals) + beam[2:]
    lst, lat = 2.0, -30.7 * DEG
    enu = np.zeros((4, 3))
    enu[:, 1] = [0, 10, 20, 30]
    bidx = np.array([0, 1, 1, 0])
    p = oracle.Problem(ra=[lst], dec=[lat], flux_ref=[1.5], enu=enu, lat=lat, beam=beam, beam_idx=bidx)
    V = oracle.vis(p, lst, 150e6)
    gains = np.array([g0, g1])[bidx]
    assert np.abs(V - 1.5 * np.outer(gains, gains.conj())).max() < 1e-12


def test_batched_uneven_generator_live_range():
    w = synth.batched_uneven(n_pairs=64, n_src=20_000, n_za=31, n_az=60)
    assert w.lsts.size == w.freqs.size == 64
    assert np.all((w.freqs >= 50e6) & (w.freqs <= 250e6))
    lat = w.lat
    up = [np.sum(np.sin(lat) * np.sin(w.dec) + np.cos(lat) * np.cos(w.dec) * np.cos(t - w.ra) > 0)
          for t in np.linspace(0, 2 * np.pi, 25)]
    # 40 % uniform + 60 % clustered: about 20 % to 80 % of the catalogue above the horizon
    assert 0.15 * 20_000 < min(up) < 0.30 * 20_000 and 0.75 * 20_000 < max(up) <= 0.85 * 20_000


# ------------------------------------------------------------ tabulated beams
# vis_with_beam_fn is the checker of every learned-beam visibility test: it
# takes the beams of a caller's model at the live sources (a table in
# catalogue order of the live sources, [beam][feed][ax][n_live]) instead of
# the grid.  Fed the oracle's own grid interpolation at those directions it
# must reproduce oracle.vis to rounding; a table in another source order or a
# dropped per-antenna beam index (Sec. 3.1 indirection a_i -> iota) must not.


def _two_beam_problem(n_feed=1, n_ax=1, stokes=False, n_src=400, seed=9):
    if n_ax == 1:
        fn = lambda p, k, AZ, ZA, NU: (np.cos(ZA) ** 2 * (1 + 0.3 * np.sin(2 * AZ))
                                       + 0.1j * np.sin(ZA) * np.cos(AZ)) * (NU / 150e6)
    else:
        fn = lambda p, k, AZ, ZA, NU: ((np.cos(ZA) * np.cos(AZ + 0.4 * p) if k == 0 else -np.sin(AZ + 0.4 * p))
                                       * np.exp(-ZA ** 2) * (1 + 0.05j * (p + k)) * (NU / 150e6))
    b = grid_beam(n_feed=n_feed, n_ax=n_ax, fn=fn)
    vals = np.concatenate([b[1], b[1] * (0.6 - 0.5j) + 0.05 * np.roll(b[1], 7, axis=-1)], axis=0)
    beam = ("grid", vals) + b[2:]
    p = small_problem(n_ant=7, n_src=n_src, beam=beam, seed=seed)
    p.beam_idx = np.array([0, 1, 1, 0, 1, 0, 0], dtype=np.int32)
    if stokes:
        g = np.random.default_rng(seed + 1)
        frac = g.uniform(0, 0.5, n_src)
        ang = g.uniform(0, 2 * np.pi, n_src)
        p.stokes_quv = np.stack([frac * np.cos(ang), frac * np.sin(ang), 0.1 * g.uniform(-1, 1, n_src)]) * p.flux_ref
    return p


@pytest.mark.parametrize("n_feed,n_ax,stokes", [(1, 1, False), (2, 2, False), (2, 2, True)])
def test_tabulated_beam_path_equals_gridded_path(n_feed, n_ax, stokes):
    p = _two_beam_problem(n_feed, n_ax, stokes)
    for lst, nu in [(0.4, 147.3e6), (3.9, 151.1e6)]:
        V = oracle.vis(p, lst, nu)
        Vt = oracle.vis_with_beam_fn(p, lst, nu, lambda az, za, f: oracle.beam_eval(p, az, za, f))
        assert np.abs(Vt - V).max() <= 1e-14 * np.abs(V).max()
        # live directions in catalogue order of the live sources
        az, za = oracle.live_directions(p, lst)
        assert az.size == oracle.count_live(p, lst)


def test_tabulated_beam_path_catches_source_order_and_beam_index_slips():
    p = _two_beam_problem()
    lst, nu = 0.4, 147.3e6
    V = oracle.vis(p, lst, nu)
    good = lambda az, za, f: oracle.beam_eval(p, az, za, f)
    # a table of the live sources in reverse order
    rev = lambda az, za, f: oracle.beam_eval(p, az, za, f)[..., ::-1]
    assert np.abs(oracle.vis_with_beam_fn(p, lst, nu, rev) - V).max() > 1e-3 * np.abs(V).max()
    # the per-antenna beam index dropped: every antenna on beam 0
    q = _two_beam_problem()
    q.beam_idx = None
    Vq = oracle.vis_with_beam_fn(q, lst, nu, good)
    assert np.abs(Vq - V).max() > 1e-3 * np.abs(V).max()


def test_tabulated_beam_zenith_source_closed_form():
    # one source at the zenith, a caller's table of one complex value per beam
    # and component: V_ab^{pq} = I sum_k A_{beta(a)}^{pk} conj(A_{beta(b)}^{qk})
    lst, lat = 1.7, -30.7 * DEG
    tab = np.array([[[[0.8 + 0.3j], [0.1 - 0.2j]], [[-0.3 + 0.1j], [0.7 + 0.0j]]],
                    [[[-0.2 + 0.9j], [0.4 + 0.4j]], [[0.5 - 0.1j], [-0.6 + 0.2j]]]])   # [beam][feed][ax][1]
    enu = np.zeros((4, 3))
    enu[:, 0] = [0.0, 14.6, 29.2, -7.3]
    bidx = np.array([1, 0, 1, 0], dtype=np.int32)
    grid = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU: 1 + 0 * AZ)
    p = oracle.Problem(ra=[lst], dec=[lat], flux_ref=[2.5], enu=enu, lat=lat, beam=grid, beam_idx=bidx)
    V = oracle.vis_with_beam_fn(p, lst, 150e6, lambda az, za, f: tab).reshape(4, 2, 4, 2)
    J = tab[..., 0]
    for a in range(4):
        for b in range(4):
            want = 2.5 * J[bidx[a]] @ J[bidx[b]].conj().T
            assert np.abs(V[a, :, b, :] - want).max() < 1e-13


# ------------------------------------------------------------ sincos polynomials
# The Z build evaluates cos(2 pi x) and sin(2 pi x) for x in [-1/8, 1/8] turn
# with polynomials in x^2 whose coefficients sit in csrc/zcore.cuh.  They were
# fitted (least squares on Chebyshev nodes) to sin(2 pi x) / x and cos(2 pi x)
# with an error below 2e-9 in FP64; rounded to FP32 the coefficients give
# polynomials within 3.0e-8 (sin) and 6.7e-9 (cos) of the exact functions, about
# half an FP32 ulp of values near 0.7.  This pin reads the coefficients from the
# source and checks that bound in FP64, so a mistyped or reordered coefficient
# fails here on the CPU.


def _zcore_coefficients():
    import re
    src = open(os.path.join(os.path.dirname(GOLDEN), "..", "paper_2312_09763_gb300", "csrc", "zcore.cuh")).read()
    body = src[src.index("cos_sin_turns"):]
    sp = body[body.index("const float sp"):body.index(";", body.index("const float sp"))]
    cp = body[body.index("const float cp"):body.index(";", body.index("const float cp"))]
    num = r"(-?\d+\.\d+(?:e-?\d+)?)f"
    s = [float(v) for v in re.findall(num, sp)]
    c = [float(v) for v in re.findall(num, cp)]
    return s, c


def test_sincos_polynomial_coefficients_meet_their_bound():
    s, c = _zcore_coefficients()
    # sin: ((s0 x2 + s1) x2 + s2) x2 + s3, times x; cos: (((c0 x2 + c1) x2 + c2) x2 + c3) x2 + c4
    assert len(s) == 4 and len(c) == 5
    x = np.linspace(-0.125, 0.125, 200_001)
    x2 = x * x
    ps = ((s[0] * x2 + s[1]) * x2 + s[2]) * x2 + s[3]
    pc = (((c[0] * x2 + c[1]) * x2 + c[2]) * x2 + c[3]) * x2 + c[4]
    assert np.abs(ps * x - np.sin(2 * np.pi * x)).max() < 3.1e-8
    assert np.abs(pc - np.cos(2 * np.pi * x)).max() < 7e-9
    # the quarter-turn reduction: |x| <= 1/8 keeps both within those bounds at the
    # ends, and sin / cos agree at x = 1/8 (both sqrt(1/2)) to the same order
    assert abs(ps[-1] * x[-1] - pc[-1]) < 4e-8
    # the leading terms are the Taylor ones to FP32 rounding (2 pi and 1, -(2 pi)^2 / 2)
    assert abs(s[3] - 2 * np.pi) < 1e-6 and c[4] == 1.0 and abs(c[3] + 2 * np.pi ** 2) < 1e-4
