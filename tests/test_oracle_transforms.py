"""Pins for the oracle's FFT and R2R transforms (Sec. 2.3 Eq. dft; Table 1 transform types).

Checks against the O(n^2) definitions written out here, numpy.fft / scipy.fft
(library routines with the same conventions), Parseval and the orthogonality
relations of the DST/DCT families.
"""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import fft, r2r


def direct_dft(x, sign):
    n = len(x)
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        s = 0.0j
        for j in range(n):
            s += x[j] * np.exp(sign * 2j * np.pi * j * k / n)
        out[k] = s
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 48, 64])
def test_fft_matches_definition(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    np.testing.assert_allclose(fft.dft(x), direct_dft(x, -1), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(fft.idft(x), direct_dft(x, +1) / n, rtol=0, atol=1e-12 * max(1, n))


@pytest.mark.parametrize("n", [96, 128, 384, 512, 1024, 1536, 2048])
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    ref = np.fft.fft(x, axis=-1)
    got = fft.dft(x, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # Parseval and round trip
    np.testing.assert_allclose(np.sum(np.abs(got) ** 2, axis=-1) / n, np.sum(np.abs(x) ** 2, axis=-1), rtol=1e-12)
    np.testing.assert_allclose(fft.idft(got, -1), x, rtol=0, atol=1e-12)


def test_fft_multi_axis():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(6, 8, 12))
    np.testing.assert_allclose(fft.dftn(x, [0, 1, 2]), np.fft.fftn(x), atol=1e-11)
    np.testing.assert_allclose(fft.idftn(fft.dftn(x, [2, 1]), [2, 1]).real, x, atol=1e-13)


KINDS = {"DST1": (1, "dst"), "DST2": (2, "dst"), "DST3": (3, "dst"), "DST4": (4, "dst"),
         "DCT1": (1, "dct"), "DCT2": (2, "dct"), "DCT3": (3, "dct"), "DCT4": (4, "dct")}


@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("n", [2, 3, 7, 16, 33, 255, 257])
def test_r2r_matches_scipy(kind, n):
    t, fam = KINDS[kind]
    rng = np.random.default_rng(n + t)
    x = rng.normal(size=(2, n))
    ref = getattr(sfft, fam)(x, type=t, axis=-1)
    got = r2r.apply(kind, x, -1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [4, 9, 64])
def test_r2r_inverse_pairs(n):
    eye = np.eye(n)
    # Table 1 forward/backward pairs with their scale give the identity
    for bc in "DN":
        for stag in (False, True):
            if bc == "N" and not stag and n < 2:
                continue
            fwd = r2r.forward(bc, stag, eye, 0)
            back = r2r.backward(bc, stag, fwd, 0)
            np.testing.assert_allclose(back, eye, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 48])
def test_r2r_inverse_pairs_mixed_faces(n):
    # Dirichlet-Neumann / Neumann-Dirichlet axes: forward then backward with its scale is the identity
    eye = np.eye(n)
    for bc in ("DN", "ND"):
        for stag in (False, True):
            back = r2r.backward(bc, stag, r2r.forward(bc, stag, eye, 0), 0)
            np.testing.assert_allclose(back, eye, atol=1e-12)


def test_dst1_eigenfunction():
    n = 15
    j = np.arange(n)
    for m in (1, 4, 15):
        x = np.sin(np.pi * (j + 1) * m / (n + 1))
        y = r2r.apply("DST1", x, 0)
        expect = np.zeros(n)
        expect[m - 1] = n + 1
        np.testing.assert_allclose(y, expect, atol=1e-12)


def test_dct2_constant():
    n = 10
    y = r2r.apply("DCT2", np.ones(n), 0)
    expect = np.zeros(n)
    expect[0] = 2 * n
    np.testing.assert_allclose(y, expect, atol=1e-12)
