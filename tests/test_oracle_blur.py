"""Pins of the oracle's scale space (Sec. 3, Sec. 4.1) against things other
than itself: scipy's Gaussian filter, numpy's symmetric padding, brute-force
2-D convolution, and the transpose identity for the adjoint."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

SIGMAS = [0.5, 0.8, 1.0, 1.6, 2.3, 4.096, 7.88, 11.64]


@pytest.mark.parametrize("sigma", SIGMAS)
def test_kernel_sums_to_one_and_is_symmetric(sigma):
    r = oracle.radius(sigma, 4.0)
    w = oracle.gauss_kernel(sigma, r)
    assert len(w) == 2 * r + 1
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.array_equal(w, w[::-1])
    assert np.all(w > 0)
    assert np.all(np.diff(w[r:]) < 0)


@pytest.mark.parametrize("sigma", SIGMAS)
def test_kernel_equals_scipy_impulse_response(sigma):
    # scipy's 1-D Gaussian filter of a unit impulse reproduces its kernel.
    r = oracle.radius(sigma, 4.0)
    n = 4 * r + 9
    x = np.zeros(n)
    x[n // 2] = 1.0
    y = ndi.gaussian_filter1d(x, sigma, mode="constant", truncate=4.0)
    w = oracle.gauss_kernel(sigma, r)
    np.testing.assert_allclose(y[n // 2 - r: n // 2 + r + 1], w, rtol=0, atol=1e-16)
    assert np.all(y[: n // 2 - r] == 0) and np.all(y[n // 2 + r + 1:] == 0)


def test_radius_rounding():
    # Sec. 4.1: radius = truncate * sigma, rounded half up; scipy uses the same.
    assert oracle.radius(0.8, 4.0) == 3
    assert oracle.radius(1.0, 4.0) == 4
    assert oracle.radius(0.875, 4.0) == 4   # 3.5 rounds up
    assert oracle.radius(7.88, 4.0) == 32
    assert oracle.radius(1.0, 5.0) == 5


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_reflect_matches_numpy_symmetric_pad(n):
    r = 3 * n + 4
    padded = np.pad(np.arange(n), r, mode="symmetric")
    for k, v in enumerate(padded):
        assert oracle.reflect(k - r, n) == v


def test_reflect_small_cases():
    assert [oracle.reflect(i, 3) for i in range(-7, 8)] == [0, 0, 1, 2, 2, 1, 0, 0, 1, 2, 2, 1, 0, 0, 1]


def _brute_blur(img, sigma, r):
    w = oracle.gauss_kernel(sigma, r)
    h, wd = img.shape
    pad = np.pad(img, r, mode="symmetric")
    out = np.zeros_like(img)
    for y in range(h):
        for x in range(wd):
            s = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    s += w[a + r] * w[b + r] * pad[y + r + a, x + r + b]
            out[y, x] = s
    return out


@pytest.mark.parametrize("shape,sigma", [((1, 1), 2.0), ((3, 7), 1.7), ((9, 5), 3.1), ((4, 4), 0.8)])
def test_separable_blur_equals_bruteforce_2d(shape, sigma):
    rng = np.random.default_rng(7)
    img = rng.random(shape)
    r = oracle.radius(sigma, 4.0)
    assert r >= min(shape) or shape == (4, 4)   # exercises multi-fold reflection
    got = oracle.blur(img, sigma, r)
    want = _brute_blur(img, sigma, r)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", [(33, 47), (64, 64), (7, 130)])
@pytest.mark.parametrize("sigma", [0.8, 1.6, 4.096, 10.48576])
def test_blur_equals_scipy_gaussian_filter(shape, sigma):
    rng = np.random.default_rng(11)
    img = rng.random(shape)
    r = oracle.radius(sigma, 4.0)
    got = oracle.blur(img, sigma, r)
    want = ndi.gaussian_filter(img, sigma, mode="reflect", truncate=4.0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_blur_of_constant_is_constant():
    img = np.full((20, 31), 0.37)
    for sigma in SIGMAS:
        out = oracle.blur(img, sigma, oracle.radius(sigma, 4.0))
        np.testing.assert_allclose(out, 0.37, rtol=0, atol=1e-15)


@pytest.mark.parametrize("shape", [(1, 1), (3, 7), (9, 5), (16, 23)])
def test_adjoint_is_matrix_transpose(shape):
    h, w = shape
    sigma = 2.2
    r = oracle.radius(sigma, 4.0)
    k = oracle.gauss_kernel(sigma, r)
    dk = oracle.gauss_kernel_dsigma(sigma, r)
    n = h * w
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = oracle.blur2(e.reshape(h, w), dk, k).ravel()
    rng = np.random.default_rng(3)
    a = rng.random((h, w))
    got = oracle.blur2_adjoint(a, dk, k).ravel()
    np.testing.assert_allclose(got, M.T @ a.ravel(), rtol=0, atol=1e-13)


def test_kernel_derivative_matches_finite_difference():
    for sigma in [0.9, 2.0, 6.5]:
        r = oracle.radius(sigma, 4.0)
        h = 1e-6
        fd = (oracle.gauss_kernel(sigma + h, r) - oracle.gauss_kernel(sigma - h, r)) / (2 * h)
        np.testing.assert_allclose(oracle.gauss_kernel_dsigma(sigma, r), fd, rtol=0, atol=1e-9)
        assert abs(oracle.gauss_kernel_dsigma(sigma, r).sum()) < 1e-14
