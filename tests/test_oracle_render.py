"""Pins of the oracle's synthetic sphere frames (Sec. 5 evaluates on rendered
spheres with Poisson and Gaussian noise; the shading is a stated reading, so
the frames are pinned by their own definition, not by the paper).

Philox4x32-10 against the known-answer vectors published with Random123
(Salmon et al., SC'11); the chord-length profile against its closed-form
integral (2/3) pi R^2 and its exact centre value; mirror symmetry; the noise
against its mean and variance."""
import numpy as np

import oracle


def test_philox_known_answers():
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert oracle.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == \
        [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert oracle.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_centre_value_and_integral():
    for R in (5.0, 9.5, 17.25):
        sph = np.array([[64.0, 64.0, R, 0.8]], np.float32)
        inten, _ = oracle.render_spheres(sph, 128, 128, ss=8, background=0.0, gain=1000.0, read_noise=0.0)
        # the integral of sqrt(1 - d^2/R^2) over the disc is (2/3) pi R^2
        want = 0.8 * 2.0 / 3.0 * np.pi * R * R
        assert abs(inten.astype(np.float64).sum() - want) <= 2e-3 * want
        # nothing outside the disc (plus the half pixel of the sub-samples)
        yy, xx = np.mgrid[0:128, 0:128]
        assert not np.any(inten[np.hypot(xx - 64, yy - 64) > R + 0.75])
    sph = np.array([[10.0, 12.0, 6.0, 0.7]], np.float32)
    inten, _ = oracle.render_spheres(sph, 24, 24, ss=1, background=0.1)
    assert inten[12, 10] == np.float32(0.1) + np.float32(0.7)     # d = 0 at the sample: chord 1


def test_mirror_symmetry():
    # centred spheres: mirrored pixels see negated offsets (their sub-samples
    # are summed in the opposite order, so equal up to rounding)
    sph = np.array([[31.5, 19.5, 11.0, 1.0], [31.5, 19.5, 4.0, 0.5]], np.float32)
    inten, _ = oracle.render_spheres(sph, 40, 64, ss=4, background=0.02)
    np.testing.assert_allclose(inten, inten[:, ::-1], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(inten, inten[::-1, :], rtol=1e-6, atol=1e-7)
    assert inten.max() > 0.9


def test_noise_mean_and_variance():
    # flat frame: counts ~ lambda + sqrt(lambda) z1 + sigma z2, rounded
    lam, sigma = 500.0, 5.0
    _, c = oracle.render_spheres(np.zeros((0, 4), np.float32), 256, 256, background=0.25, gain=2000.0,
                                 read_noise=sigma, seed=123)
    v = c.astype(np.float64)
    assert abs(v.mean() - lam) < 0.5
    assert abs(v.var() / (lam + sigma ** 2 + 1.0 / 12.0) - 1.0) < 0.03
    # a different seed gives a different frame, the same seed the same one
    _, c2 = oracle.render_spheres(np.zeros((0, 4), np.float32), 256, 256, background=0.25, gain=2000.0,
                                  read_noise=sigma, seed=124)
    _, c3 = oracle.render_spheres(np.zeros((0, 4), np.float32), 256, 256, background=0.25, gain=2000.0,
                                  read_noise=sigma, seed=123)
    assert not np.array_equal(c, c2) and np.array_equal(c, c3)
    # clipping at the 12-bit range
    _, hi = oracle.render_spheres(np.zeros((0, 4), np.float32), 8, 8, background=5.0, gain=2000.0)
    assert np.all(hi == 4095)
