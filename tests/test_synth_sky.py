"""Synthetic diffuse sky: HEALPix RING geometry against Gorski et al. (2005)
closed forms and the random field's statistics (no GPU)."""
import numpy as np

from paper_2312_09763_gb300 import synth


def test_healpix_ring_geometry():
    nside = 8
    theta, phi = synth.healpix_ring_pix2ang(nside)
    assert theta.size == 12 * nside * nside
    z = np.round(np.cos(theta), 12)
    rings = np.unique(z)[::-1]
    assert rings.size == 4 * nside - 1
    # ring i (1-based from the north pole): z = 1 - i^2 / (3 nside^2) in the caps,
    # 4/3 - 2 i / (3 nside) in the belt; 4 i pixels per cap ring, 4 nside in the belt
    for i, zr in enumerate(rings, start=1):
        k = min(i, 4 * nside - i)
        want = (1 - k * k / (3.0 * nside * nside)) * (1 if i <= 2 * nside else -1) if k < nside else \
            4.0 / 3.0 - 2.0 * i / (3.0 * nside)
        assert abs(zr - want) < 1e-12, i
        n_in = np.sum(z == zr)
        assert n_in == (4 * k if k < nside else 4 * nside)
        ph = np.sort(phi[z == zr])
        assert np.allclose(np.diff(ph), 2 * np.pi / n_in)
    # equal areas: the mean of z over all pixels is zero, of z^2 is 1/3 (uniform sphere)
    assert abs(z.mean()) < 1e-12 and abs((z * z).mean() - 1.0 / 3.0) < 2e-3


def test_random_field_statistics():
    nside, lmax = 16, 40
    theta, phi = synth.healpix_ring_pix2ang(nside)
    ell = np.arange(lmax + 1.0)
    cl = np.where(ell >= 1, np.maximum(ell, 1) ** -2.5, 0.0)
    f = synth.gaussian_random_field(theta, phi, lmax, cl, np.random.default_rng(0))
    # variance of a field with spectrum C_l: sum (2l+1) C_l / (4 pi)
    want = np.sum((2 * ell + 1) * cl) / (4 * np.pi)
    assert 0.3 * want < f.var() < 3.0 * want
    # a field with power only at l = 2 lies in the span of the five real l = 2
    # harmonics (closed forms): 3z^2-1, z s cos(phi), z s sin(phi), s^2 cos(2phi), s^2 sin(2phi)
    cl2 = np.array([0.0, 0.0, 1.0])
    f2 = synth.gaussian_random_field(theta, phi, 2, cl2, np.random.default_rng(1))
    z = np.cos(theta)
    s = np.sin(theta)
    basis = np.stack([3 * z * z - 1, z * s * np.cos(phi), z * s * np.sin(phi),
                      s * s * np.cos(2 * phi), s * s * np.sin(2 * phi)], axis=1)
    coef = np.linalg.lstsq(basis, f2, rcond=None)[0]
    assert np.abs(basis @ coef - f2).max() <= 1e-10 * np.abs(f2).max()
    # and an l = 3 field is orthogonal to it (pixel sums approximate the sphere integral)
    cl3 = np.array([0.0, 0.0, 0.0, 1.0])
    f3 = synth.gaussian_random_field(theta, phi, 3, cl3, np.random.default_rng(2))
    assert abs(np.mean(f2 * f3)) <= 1e-3 * np.sqrt(np.mean(f2 ** 2) * np.mean(f3 ** 2))
    # the m = 0 normalisation: Y_20 = sqrt(5 / (16 pi)) (3 z^2 - 1) has unit mean square x 4 pi
    y20 = np.sqrt(5 / (16 * np.pi)) * (3 * z * z - 1)
    assert abs(4 * np.pi * np.mean(y20 ** 2) - 1.0) < 1e-2
