"""Pins of the oracle's real spherical-harmonic basis (App. B.1) against closed
forms, identities and scipy's complex spherical harmonics."""
import math

import numpy as np
import pytest


def _dirs(n, seed=0):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_y00_closed_form(oracle_mod):
    Y = oracle_mod.sh_basis(1, _dirs(50))
    assert np.allclose(Y[:, 0], 1.0 / (2.0 * math.sqrt(math.pi)), rtol=0, atol=1e-15)


def test_degree1_cartesian_signs(oracle_mod):
    # With the Condon-Shortley phase in P_l^m and the (-1)^m of the real basis,
    # the degree-1 functions are +y, +z, +x times sqrt(3/(4 pi)).
    d = _dirs(200, 1)
    Y = oracle_mod.sh_basis(4, d)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    assert np.allclose(Y[:, 1], c1 * d[:, 1], atol=1e-14)
    assert np.allclose(Y[:, 2], c1 * d[:, 2], atol=1e-14)
    assert np.allclose(Y[:, 3], c1 * d[:, 0], atol=1e-14)


def test_degree2_cartesian(oracle_mod):
    d = _dirs(200, 2)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    Y = oracle_mod.sh_basis(9, d)
    a = 0.5 * math.sqrt(15.0 / math.pi)
    exp = np.stack([a * x * y, a * y * z, 0.25 * math.sqrt(5.0 / math.pi) * (3 * z * z - 1),
                    a * x * z, 0.25 * math.sqrt(15.0 / math.pi) * (x * x - y * y)], axis=1)
    assert np.allclose(Y[:, 4:9], exp, atol=1e-14)


@pytest.mark.parametrize("lmax", [0, 1, 2, 3, 4])
def test_unsold_identity(oracle_mod, lmax):
    d = _dirs(300, 3 + lmax)
    K = (lmax + 1) ** 2
    Y = oracle_mod.sh_basis(K, d)
    for l in range(lmax + 1):
        s = (Y[:, l * l:(l + 1) * (l + 1)] ** 2).sum(axis=1)
        assert np.allclose(s, (2 * l + 1) / (4 * math.pi), atol=1e-13)


def test_orthonormal_by_quadrature(oracle_mod):
    # Gauss-Legendre in cos(theta) (exact for polynomials of degree <= 2*20-1)
    # times the uniform rule in phi (exact for trigonometric degree < 40).
    K = 25
    xg, wg = np.polynomial.legendre.leggauss(20)
    nphi = 40
    phi = 2 * math.pi * np.arange(nphi) / nphi
    ct = np.repeat(xg, nphi)
    st = np.sqrt(1 - ct * ct)
    ph = np.tile(phi, len(xg))
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    w = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    Y = oracle_mod.sh_basis(K, d)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(K), atol=1e-12)


def test_against_scipy_complex_harmonics(oracle_mod):
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    d = _dirs(100, 9)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    K = 25
    Y = oracle_mod.sh_basis(K, d)
    for l in range(5):
        for m in range(-l, l + 1):
            cplx = sp.sph_harm_y(l, abs(m), theta, phi)   # includes the Condon-Shortley phase
            if m < 0:
                ref = math.sqrt(2) * (-1) ** m * cplx.imag
            elif m == 0:
                ref = cplx.real
            else:
                ref = math.sqrt(2) * (-1) ** m * cplx.real
            assert np.allclose(Y[:, l * l + l + m], ref, atol=1e-13), (l, m)


def test_poles(oracle_mod):
    d = np.array([[0, 0, 1.0], [0, 0, -1.0]])
    Y = oracle_mod.sh_basis(16, d)
    for l in range(4):
        for m in range(-l, l + 1):
            if m != 0:
                assert abs(Y[0, l * l + l + m]) < 1e-15 and abs(Y[1, l * l + l + m]) < 1e-15
        # Y_l^0(pole) = sqrt((2l+1)/(4pi)) * (+-1)^l
        assert Y[0, l * l + l] == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), abs=1e-14)
        assert Y[1, l * l + l] == pytest.approx((-1) ** l * math.sqrt((2 * l + 1) / (4 * math.pi)),
                                                abs=1e-14)
