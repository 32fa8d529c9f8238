"""Pins of the pipeline-step oracle (oracle/pipeline.py) to things other than itself: closed
forms of the interpolation window, exact results (identity and integer maps, linear data
under bilinear interpolation, constants, Cramer's rule), symmetry, numpy's FFT and finite
differences.  Each pin is chosen so that a plausible slip (a tap offset, a sign, a transposed
coordinate, a dropped weight or term) fails it."""
import math

import numpy as np
import pytest

from oracle import pipeline as po


def gauss_stamp(K, sigma, cx=0.0, cy=0.0):
    c = (K - 1) // 2
    y, x = np.mgrid[0:K, 0:K] - c
    g = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * sigma ** 2))
    return g / g.sum()


def affine(a, b, c, d, e, f, degree=1, x_ref=0.0, y_ref=0.0):
    """u = a + b x + c y, v = d + e x + f y."""
    cu = [a, b, c] + [0.0] * 7
    cv = [d, e, f] + [0.0] * 7
    return dict(degree=degree, x_ref=x_ref, y_ref=y_ref, cu=cu, cv=cv)


# ------------------------------------------------------------------ step 4: resampling


def test_lanczos3_closed_forms():
    pi2 = math.pi ** 2
    for t, ref in ((0.5, 6 / pi2), (1.5, -4 / (3 * pi2)), (2.5, 6 / (25 * pi2)), (0.0, 1.0),
                   (1.0, 0.0), (2.0, 0.0), (3.0, 0.0), (3.2, 0.0)):
        assert po.lanczos3(t) == pytest.approx(ref, abs=1e-15)
        assert po.lanczos3(-t) == pytest.approx(ref, abs=1e-15)


def test_warp_monomial_order():
    x, y, xr, yr = 7.0, 3.0, 2.0, 1.0
    dx, dy = x - xr, y - yr
    expect = [1, dx, dy, dx * dx, dx * dy, dy * dy, dx ** 3, dx * dx * dy, dx * dy * dy, dy ** 3]
    for j in range(10):
        cu = [0.0] * 10
        cu[j] = 1.0
        cv = [0.0] * 10
        cv[j] = 2.0
        u, v = po.warp_eval(dict(degree=3, x_ref=xr, y_ref=yr, cu=cu, cv=cv), x, y)
        assert u == expect[j] and v == 2 * expect[j]


def test_warp_jacobian_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = dict(degree=3, x_ref=50.0, y_ref=40.0, cu=list(rng.normal(0, 1e-3, 10)), cv=list(rng.normal(0, 1e-3, 10)))
    w["cu"][1] += 1.0
    w["cv"][2] += 1.0
    for x, y in ((10.0, 20.0), (90.0, 5.0)):
        J = po.warp_jacobian(w, x, y)
        h = 1e-4
        for k, (ex, ey) in enumerate(((h, 0.0), (0.0, h))):
            up, vp = po.warp_eval(w, x + ex, y + ey)
            um, vm = po.warp_eval(w, x - ex, y - ey)
            assert (up - um) / (2 * h) == pytest.approx(J[0, k], rel=1e-7, abs=1e-9)
            assert (vp - vm) / (2 * h) == pytest.approx(J[1, k], rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("method", [po.LANCZOS3, po.BILINEAR])
def test_identity_and_integer_shift_are_exact(method):
    rng = np.random.default_rng(1)
    img = rng.normal(size=(12, 15))
    mask = (rng.random((12, 15)) < 0.1).astype(np.uint8)
    out, om, _ = po.resample(img, affine(0, 1, 0, 0, 0, 1), (12, 15), mask, method)
    assert np.array_equal(np.where(mask == 0, img, 0.0), out) and np.array_equal(om, mask)
    # u = x + 3, v = y - 2: out[y, x] = img[y - 2, x + 3]; outside the template -> masked
    out, om, _ = po.resample(img, affine(3, 1, 0, -2, 0, 1), (12, 15), mask, method)
    ref = np.zeros_like(img)
    refm = np.ones_like(mask)
    ref[2:, :12] = np.where(mask[:10, 3:] == 0, img[:10, 3:], 0.0)
    refm[2:, :12] = mask[:10, 3:]
    assert np.array_equal(out, ref) and np.array_equal(om, refm)


def test_bilinear_reproduces_a_linear_ramp_under_an_affine_map():
    ny, nx = 30, 40
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    img = 0.7 * x - 1.3 * y + 5.0
    th = 0.3
    w = affine(6.0, 0.9 * math.cos(th), -0.9 * math.sin(th), 4.0, 0.9 * math.sin(th), 0.9 * math.cos(th))
    out, om, _ = po.resample(img, w, (20, 20), None, po.BILINEAR)
    for r in range(20):
        for s in range(20):
            u, v = po.warp_eval(w, float(s), float(r))
            if om[r, s] == 0:
                assert out[r, s] == pytest.approx(0.7 * u - 1.3 * v + 5.0, abs=1e-12)
    assert (om == 0).sum() > 200


def test_lanczos_keeps_a_constant_and_flux_scales_by_the_jacobian():
    img = np.full((40, 40), 3.0)
    s, th = 1.1, 0.4
    w = affine(20.0, s * math.cos(th), -s * math.sin(th), 2.0, s * math.sin(th), s * math.cos(th))
    out, om, _ = po.resample(img, w, (16, 16), None, po.LANCZOS3)
    outf, _, _ = po.resample(img, w, (16, 16), None, po.LANCZOS3, flux=True)
    good = om == 0
    assert good.sum() > 50
    assert np.allclose(out[good], 3.0, atol=1e-13)
    assert np.allclose(outf[good], 3.0 * s * s, atol=1e-12)


def test_half_pixel_shift_of_a_symmetric_profile_is_mirror_symmetric():
    K = 21
    img = gauss_stamp(K, 2.0)
    out, _, _ = po.resample(img, affine(-0.5, 1, 0, 0, 0, 1), (K, K), None, po.LANCZOS3, zero_outside=True)
    c = (K - 1) // 2
    # out(x) = img(x - 0.5) is symmetric about x = c + 0.5
    for k in range(c - 2):
        assert out[c, c + 1 + k] == pytest.approx(out[c, c - k], rel=1e-12)
    # and close to the shifted Gaussian itself (a smooth, well-sampled profile)
    assert np.abs(out - gauss_stamp(K, 2.0, cx=0.5)).max() < 5e-3 * img.max()


def test_mask_spreads_by_the_half_pixel_lanczos_weights():
    img = np.ones((9, 20))
    mask = np.zeros((9, 20), np.uint8)
    mask[4, 10] = 1
    _, om, frac = po.resample(img, affine(0.5, 1, 0, 0, 0, 1), (9, 20), mask, po.LANCZOS3)
    # taps at distances -2.5 .. 2.5: |L| = 6/(25 pi^2), 4/(3 pi^2), 6/pi^2 (twice each)
    pi2 = math.pi ** 2
    wa = [6 / (25 * pi2), 4 / (3 * pi2), 6 / pi2, 6 / pi2, 4 / (3 * pi2), 6 / (25 * pi2)]
    tot = sum(wa)
    # out x reads u = x + 0.5 -> taps floor(u) - 2 .. floor(u) + 3 = x - 2 .. x + 3
    for x in range(7, 13):
        assert frac[4, x] == pytest.approx(wa[x - 7] / tot, rel=1e-12)
    expect = np.zeros_like(mask)
    expect[4, 7:13] = 1
    expect[:, :2] = 1   # taps left of column 0 on the left edge
    expect[:, 17:] = 1  # taps right of column 19
    assert np.array_equal(om, expect)


def test_align_psf_identity_and_quarter_turn():
    rng = np.random.default_rng(3)
    P = rng.random((9, 9))
    ident = affine(0, 1, 0, 0, 0, 1)
    assert np.array_equal(po.align_psf(P, ident, 100.0, 200.0), P)
    # u = x0 - y, v = y0 + x (a quarter turn): stamp offset (dx, dy) -> template (-dy, dx)
    rot = affine(500.0, 0, -1, 300.0, 1, 0)
    A = po.align_psf(P, rot, 100.0, 200.0)
    c = 4
    for r in range(9):
        for s in range(9):
            assert A[r, s] == pytest.approx(P[c + (s - c), c - (r - c)], abs=1e-15)


# ------------------------------------------------------------------ step 7: decorrelation


def _place(st, M):
    K = st.shape[0]
    c = (K - 1) // 2
    g = np.zeros((M, M))
    for a in range(K):
        for b in range(K):
            g[(a - c) % M, (b - c) % M] += st[a, b]
    return g


def test_matching_kernel_at_a_corner():
    L, dk = 3, 1
    rng = np.random.default_rng(4)
    th = rng.normal(size=3 * L * L + 3)
    K = po.matching_kernel(th, L, dk, (50, 80), 79.0, 0.0)  # xh = 1, yh = -1
    ref = th[:9] + th[9:18] - th[18:27]
    assert np.allclose(K.ravel(), ref, atol=1e-15)


def test_decorrelation_is_a_delta_without_template_noise_and_psf():
    Ps = gauss_stamp(11, 1.6)
    delta = np.zeros((1, 1)) + 1.0
    kern = gauss_stamp(5, 0.8) * 1.7
    phi, pd = po.decorrelation_kernel(Ps, delta, kern, 2.0, 0.0, 15)
    ref = np.zeros((15, 15))
    ref[7, 7] = 1.0
    assert np.abs(phi - ref).max() < 1e-14
    assert np.abs(pd - np.pad(Ps, 2)).max() < 1e-14


def test_decorrelation_whitens_the_difference_noise_spectrum():
    M = 25
    Ps, Pt = gauss_stamp(15, 1.4, 0.2, -0.1), gauss_stamp(13, 2.1, -0.3, 0.25)
    rng = np.random.default_rng(5)
    kern = gauss_stamp(7, 1.0) * 0.93 + rng.normal(0, 1e-3, (7, 7))
    ss, st = 1.3, 0.8
    phi, pd = po.decorrelation_kernel(Ps, Pt, kern, ss, st, M)
    F = lambda a: np.fft.fft2(_place(a, M))
    den = ss ** 2 * np.abs(F(Pt)) ** 2 + st ** 2 * np.abs(F(kern)) ** 2 * np.abs(F(Ps)) ** 2
    num = ss ** 2 + kern.sum() ** 2 * st ** 2
    # unit-gain whitening where the noise spectrum is above the floor, the capped gain below it
    g2 = np.abs(F(phi)) ** 2
    free = den >= 1e-8 * num
    assert free.sum() > M * M // 4 and (~free).sum() > 0
    assert np.allclose(g2[free] * den[free], num, rtol=1e-9)
    assert np.allclose(g2[~free], 1e8, rtol=1e-9)
    assert phi.sum() == pytest.approx(1.0, abs=1e-9)
    assert np.allclose(phi, phi[::-1, ::-1], atol=1e-12 * np.abs(phi).max())
    # the decorrelated science PSF is phi (x) P_S (x) P_T on the M grid
    ref = np.fft.ifft2(F(phi) * F(Ps) * F(Pt)).real
    assert np.allclose(_place(pd, M), ref, atol=1e-12)
    assert pd.sum() == pytest.approx(1.0, abs=1e-12)


# ------------------------------------------------------------------ step 9: photometry


@pytest.mark.parametrize("x,y,X,Y,fx,fy", [(2.5, 3.0, 3, 3, -0.5, 0.0), (2.49, -0.5, 2, 0, 0.49, -0.5),
                                           (10.0, 7.75, 10, 8, 0.0, -0.25)])
def test_source_pixel_rounding(x, y, X, Y, fx, fy):
    a = po.source_pixel(x, y)
    assert a[:2] == (X, Y) and a[2] == pytest.approx(fx, abs=1e-15) and a[3] == pytest.approx(fy, abs=1e-15)


def test_shifted_psf_zero_offset_is_the_stamp():
    P = gauss_stamp(13, 1.5)
    assert np.array_equal(po.shifted_psf(P, 0.0, 0.0), P)


@pytest.mark.parametrize("background", [False, True])
@pytest.mark.parametrize("weighted", [False, True])
def test_photometry_recovers_an_exact_source(background, weighted):
    rng = np.random.default_rng(6)
    P = gauss_stamp(11, 1.7)
    D = np.zeros((40, 50))
    D[12:23, 20:31] += 250.0 * P  # centre at (17, 25)
    if background:
        D += 3.5
    W = rng.uniform(0.5, 2.0, D.shape) if weighted else None
    f, sf, b, chi2, n = po.forced_photometry(D, P, 25.0, 17.0, W, None, background)
    assert f == pytest.approx(250.0, rel=1e-12)
    assert b == pytest.approx(3.5 if background else 0.0, abs=1e-9)
    assert chi2 < 1e-18 and n == 121


def test_photometry_closed_forms():
    rng = np.random.default_rng(7)
    P = gauss_stamp(9, 1.3)
    D = rng.normal(0, 1, (30, 30))
    W = rng.uniform(0.2, 3.0, D.shape)
    f, sf, b, chi2, n = po.forced_photometry(D, P, 14.0, 15.0, W)
    d, w = D[11:20, 10:19], W[11:20, 10:19]
    assert f == pytest.approx((w * P * d).sum() / (w * P * P).sum(), rel=1e-12)
    assert sf == pytest.approx(1.0 / math.sqrt((w * P * P).sum()), rel=1e-12)
    assert chi2 == pytest.approx((w * (d - f * P) ** 2).sum(), rel=1e-12)
    # with a background: Cramer's rule on the 2 x 2 normal equations
    f2, sf2, b2, _, _ = po.forced_photometry(D, P, 14.0, 15.0, W, None, True)
    a11, a12, a22 = (w * P * P).sum(), (w * P).sum(), w.sum()
    r1, r2 = (w * P * d).sum(), (w * d).sum()
    det = a11 * a22 - a12 * a12
    assert f2 == pytest.approx((r1 * a22 - a12 * r2) / det, rel=1e-10)
    assert b2 == pytest.approx((a11 * r2 - a12 * r1) / det, rel=1e-10)
    assert sf2 == pytest.approx(math.sqrt(a22 / det), rel=1e-10)


def test_photometry_ignores_masked_pixels_and_clips_at_the_edge():
    P = gauss_stamp(7, 1.2)
    rng = np.random.default_rng(8)
    D = rng.normal(size=(20, 20))
    M = np.zeros((20, 20), np.uint8)
    M[5, 6] = 1
    a = po.forced_photometry(D, P, 6.0, 5.0, None, M, True)
    D2 = D.copy()
    D2[5, 6] = 1e30
    b = po.forced_photometry(D2, P, 6.0, 5.0, None, M, True)
    assert a == b and a[4] == 48
    # a source in the corner: the footprint keeps its 4 x 4 in-frame quarter
    assert po.forced_photometry(D, P, 0.2, 19.4, None, None, False)[4] == 16
