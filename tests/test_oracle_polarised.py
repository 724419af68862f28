"""Pins of the oracle's fully polarised sky (no GPU).

The coherency of Sec. 2.1, C = [[I + Q, U + iV], [U - iV, I - Q]] in the
beam's (theta, phi) basis, enters the direct sum as sum_kk' A^{pk} C_kk'
conj(A^{qk'}) (eq. "matvistensorprod") and the outer-product form through a
square root M M^dagger = C (eq. "fullz").  Pinned by closed forms (a zenith
source seen by an identity or a general constant Jones beam), the
unpolarised limit, linearity in (I, Q, U, V), Hermitian symmetry, the
spectral scaling and the factorisation itself.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import DEG, grid_beam, small_problem


def coherency(I, Q, U, V):
    return np.array([[I + Q, U + 1j * V], [U - 1j * V, I - Q]])


def test_coherency_square_root():
    g = np.random.default_rng(0)
    cases = [(2.0, 0.3, -0.4, 0.1), (1.0, -1.0, 0.0, 0.0), (1.0, 0.6, 0.8, 0.0), (3.0, 0.0, 0.0, 0.0),
             (1.0, 0.0, 0.0, -1.0)]
    for _ in range(50):
        I = g.uniform(0.1, 5)
        d = g.normal(size=3)
        d *= g.uniform(0, 1) * I / np.linalg.norm(d)
        cases.append((I, *d))
    for I, Q, U, V in cases:
        M = oracle.coherency_sqrt(I, Q, U, V)
        assert M[0, 1] == 0
        assert np.abs(M @ M.conj().T - coherency(I, Q, U, V)).max() <= 1e-13 * I


def zenith_problem(beam, stokes, flux=2.0, spec=None):
    lst, lat = 0.4, -30.7 * DEG
    enu = np.zeros((3, 3))
    enu[:, 0] = [0, 14.6, 29.2]
    return oracle.Problem(ra=[lst], dec=[lat], flux_ref=[flux], enu=enu, lat=lat, beam=beam,
                          stokes_quv=np.array(stokes, dtype=float).reshape(3, 1),
                          spec_idx=None if spec is None else [spec], nu_ref=150e6), lst


def test_zenith_source_identity_beam_gives_the_coherency():
    # feed p sees only axis p: V^{pq} = C_pq exactly for every baseline
    beam = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU: float(p == k) + 0 * AZ)
    P, lst = zenith_problem(beam, [0.3, -0.5, 0.2], flux=2.0)
    V = oracle.vis(P, lst, 145e6).reshape(3, 2, 3, 2)
    want = np.array([[2.3, -0.5 + 0.2j], [-0.5 - 0.2j, 1.7]])
    for a in range(3):
        for b in range(3):
            assert np.abs(V[a, :, b, :] - want).max() < 1e-12


def test_zenith_source_general_jones():
    J = np.array([[0.9 + 0.1j, -0.2 + 0.05j], [0.15 - 0.3j, 0.8 + 0.0j]])
    beam = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU: J[p, k] + 0 * AZ)
    P, lst = zenith_problem(beam, [0.4, 0.7, -0.3], flux=1.5)
    V = oracle.vis(P, lst, 145e6).reshape(3, 2, 3, 2)
    want = J @ coherency(1.5, 0.4, 0.7, -0.3) @ J.conj().T
    assert np.abs(V[1, :, 2, :] - want).max() < 1e-12
    # outer-product form through M
    Vo = oracle.vis_outer(P, lst, 145e6).reshape(3, 2, 3, 2)
    assert np.abs(Vo[0, :, 2, :] - want).max() < 1e-12


def jones_beam():
    return grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU:
                     (np.cos(ZA) * np.cos(AZ + 0.3 * p + 0.9 * k) + 0.2j * (k - p)) * np.exp(-ZA ** 2)
                     * (NU / 150e6))


def polarised_problem(n_ant=5, n_src=200, frac=0.6, seed=4):
    P = small_problem(n_ant=n_ant, n_src=n_src, beam=jones_beam(), seed=seed)
    g = np.random.default_rng(seed + 100)
    d = g.normal(size=(3, n_src))
    d *= frac * g.uniform(0, 1, n_src) * P.flux_ref / np.linalg.norm(d, axis=0)
    P.stokes_quv = d
    return P


def test_unpolarised_limit():
    P = polarised_problem()
    P.stokes_quv = np.zeros_like(P.stokes_quv)
    Vp = oracle.vis(P, 0.7, 151e6)
    P.stokes_quv = None
    Vu = oracle.vis(P, 0.7, 151e6)
    assert np.abs(Vp - Vu).max() <= 1e-14 * np.abs(Vu).max()


def test_direct_sum_equals_outer_product_polarised():
    P = polarised_problem()
    for lst in [0.2, 3.0]:
        Vd = oracle.vis(P, lst, 147.3e6)
        Vo = oracle.vis_outer(P, lst, 147.3e6)
        assert np.abs(Vd - Vo).max() <= 1e-12 * np.abs(Vo).max()


def test_linearity_in_stokes():
    # the direct sum is linear in C, so V(I, Q, U, V) = V(I) + V(Q) + V(U) + V(V)
    P = polarised_problem()
    V = oracle.vis(P, 1.1, 146e6)
    quv = P.stokes_quv.copy()
    parts = []
    for i in range(4):
        Pi = polarised_problem()
        Pi.flux_ref = P.flux_ref if i == 0 else 0 * P.flux_ref
        Pi.stokes_quv = np.zeros_like(quv)
        if i > 0:
            Pi.stokes_quv[i - 1] = quv[i - 1]
        parts.append(oracle.vis(Pi, 1.1, 146e6))
    assert np.abs(sum(parts) - V).max() <= 1e-13 * np.abs(V).max()
    # Stokes V alone (C = [[0, iV], [-iV, 0]], Hermitian) still gives a Hermitian V
    Vv = parts[3].reshape(5, 2, 5, 2)
    assert np.abs(Vv - np.conj(np.transpose(Vv, (2, 3, 0, 1)))).max() <= 1e-14 * np.abs(Vv).max()


def test_hermitian_polarised():
    P = polarised_problem()
    V = oracle.vis(P, 2.2, 142e6)
    assert np.abs(V - V.conj().T).max() <= 1e-14 * np.abs(V).max()
    assert np.all(np.diag(V).real >= 0)


def test_stokes_follow_the_flux_spectrum():
    beam = grid_beam(n_feed=2, n_ax=2, fn=lambda p, k, AZ, ZA, NU: (1.0 + 0.3j * (p != k)) + 0 * AZ)
    P, lst = zenith_problem(beam, [0.2, 0.1, 0.3], flux=1.0, spec=-2.5)
    V1 = oracle.vis(P, lst, 150e6)
    V2 = oracle.vis(P, lst, 145e6)
    assert np.abs(V2 - (145 / 150) ** -2.5 * V1).max() <= 1e-13 * np.abs(V2).max()


def test_single_axis_beam_rejected():
    P = small_problem(n_ant=3, n_src=10)
    P.stokes_quv = np.zeros((3, 10))
    with pytest.raises(ValueError, match="two-axis"):
        oracle.vis(P, 0.1, 150e6)
