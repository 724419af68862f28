"""Algorithm 1 (Sec. 2.3): perturbed equatorial coordinates, host logic, no GPU.

The oracle's perturb_sky is pinned by what the rotation fixes: the rigid
rotation at the reference LST applied to the perturbed coordinates gives back
the apparent direction it was fed; apparent directions that came from the
rigid rotation itself give back the original catalogue; the zenith, the north
and the east horizon points have closed forms.  The library's host call
mv_perturb_sky is then checked against the oracle on the same inputs, and its
input checks are exercised.
"""
import numpy as np
import pytest

import oracle

DEG = np.pi / 180
LAT = -30.7 * DEG


def enu_of(alt, az):
    """East-North-Up unit vectors of (alt, az), az from North through East."""
    return np.stack([np.cos(alt) * np.sin(az), np.cos(alt) * np.cos(az), np.sin(alt)], 1)


def apparent(n, seed=0):
    g = np.random.default_rng(seed)
    alt = np.arcsin(g.uniform(-1, 1, n))
    az = g.uniform(0, 2 * np.pi, n)
    return alt, az


@pytest.mark.parametrize("lst,lat", [(0.3, LAT), (4.1, 52 * DEG), (6.0, 0.0), (2.2, -89 * DEG)])
def test_rigid_rotation_of_perturbed_coordinates_gives_the_apparent_direction(lst, lat):
    alt, az = apparent(2000)
    ra, dec = oracle.perturb_sky(alt, az, lst, lat)
    x = oracle.to_topo(oracle.rotation(lst, lat), oracle.xeq(ra, dec))
    assert np.abs(x - enu_of(alt, az)).max() < 2e-15
    assert np.all((ra >= 0) & (ra < 2 * np.pi)) and np.all(np.abs(dec) <= np.pi / 2)


def test_unperturbed_directions_return_the_catalogue():
    g = np.random.default_rng(3)
    ra0 = g.uniform(0, 2 * np.pi, 3000)
    dec0 = np.arcsin(g.uniform(-0.999, 0.999, 3000))
    lst = 1.9
    x = oracle.to_topo(oracle.rotation(lst, LAT), oracle.xeq(ra0, dec0))
    az, za = oracle.azza(x)
    ra, dec = oracle.perturb_sky(np.pi / 2 - za, az, lst, LAT)
    dra = np.angle(np.exp(1j * (ra - ra0)))
    assert np.abs(dra * np.cos(dec0)).max() < 1e-13 and np.abs(dec - dec0).max() < 1e-13


@pytest.mark.parametrize("lst,lat", [(0.7, LAT), (3.0, 40 * DEG)])
def test_closed_forms(lst, lat):
    # zenith: RA = LST, Dec = latitude
    ra, dec = oracle.perturb_sky([np.pi / 2], [0.4], lst, lat)
    assert abs(np.angle(np.exp(1j * (ra[0] - lst)))) < 1e-15 and abs(dec[0] - lat) < 1e-15
    # north point of the horizon: on the meridian (below the pole north of
    # the equator), Dec = 90 deg - |latitude|
    ra, dec = oracle.perturb_sky([0.0], [0.0], lst, lat)
    want_ra = lst + (np.pi if lat > 0 else 0.0)
    assert abs(np.angle(np.exp(1j * (ra[0] - want_ra)))) < 1e-15
    assert abs(dec[0] - (np.pi / 2 - abs(lat))) < 1e-15
    # east point of the horizon: on the equator, six hours east of the meridian
    ra, dec = oracle.perturb_sky([0.0], [np.pi / 2], lst, lat)
    assert abs(np.angle(np.exp(1j * (ra[0] - lst - np.pi / 2)))) < 1e-15 and abs(dec[0]) < 1e-15


def test_a_fixed_frame_rotation_is_recovered_at_every_time():
    # apparent directions from a catalogue seen through a fixed small frame
    # rotation Q (a stand-in for precession): the perturbed catalogue is Q X_eq
    # itself, so the rigid rotation with it is exact at every LST, not only at
    # the reference time
    g = np.random.default_rng(8)
    ra0 = g.uniform(0, 2 * np.pi, 500)
    dec0 = np.arcsin(g.uniform(-1, 1, 500))
    th = 0.4 * DEG
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Q = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    Xq = oracle.xeq(ra0, dec0) @ Q.T
    lst_ref = 2.5
    az, za = oracle.azza(oracle.to_topo(oracle.rotation(lst_ref, LAT), Xq))
    ra, dec = oracle.perturb_sky(np.pi / 2 - za, az, lst_ref, LAT)
    for lst in (lst_ref, lst_ref + 0.5, lst_ref + 3.0):
        want = oracle.to_topo(oracle.rotation(lst, LAT), Xq)
        got = oracle.to_topo(oracle.rotation(lst, LAT), oracle.xeq(ra, dec))
        assert np.abs(got - want).max() < 3e-15
        unpert = oracle.to_topo(oracle.rotation(lst, LAT), oracle.xeq(ra0, dec0))
        assert np.abs(unpert - want).max() > 1e-3


def test_library_host_call_matches_oracle():
    from paper_2312_09763_gb300 import perturb_sky
    for lst, lat in [(0.3, LAT), (4.1, 52 * DEG), (6.2, -89.5 * DEG)]:
        alt, az = apparent(5000, seed=11)
        ra, dec = perturb_sky(alt, az, lst, lat)
        ra_o, dec_o = oracle.perturb_sky(alt, az, lst, lat)
        # compare directions (RA is ill-conditioned at the poles)
        assert np.abs(oracle.xeq(ra, dec) - oracle.xeq(ra_o, dec_o)).max() < 2e-15
        assert np.all((ra >= 0) & (ra < 2 * np.pi))


def test_library_host_call_rejects_bad_input():
    from paper_2312_09763_gb300 import MatvisError, perturb_sky
    alt, az = apparent(10)
    with pytest.raises(MatvisError, match="MV_ERR_ARG"):
        perturb_sky(alt, az, 0.0, 1.6)              # |latitude| > pi/2
    bad = alt.copy()
    bad[7] = np.nan
    with pytest.raises(MatvisError, match=r"\[7\]"):
        perturb_sky(bad, az, 0.0, LAT)
    with pytest.raises(MatvisError, match="MV_ERR_ARG"):
        perturb_sky([], [], 0.0, LAT)
