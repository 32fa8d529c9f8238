"""FP64 CPU oracle for the pipeline steps around the fit (Sec. "Pipeline steps"):

* step 4, alignment and resampling of the template image, its detection mask and its PSF
  onto the science frame (``warp_eval``, ``lanczos3``, ``resample``, ``align_psf``);
* step 7, the decorrelation kernel and its application (``matching_kernel``,
  ``decorrelation_kernel``; the application is a convolution, ``oracle.convolve``);
* step 9, forced PSF photometry at a given position (``shifted_psf``, ``forced_photometry``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` are the only callers; the CUDA library never imports or calls it.

The paper names these steps but fixes neither an interpolation kernel, a coordinate model,
a decorrelation formula nor a photometry estimator.  The definitions below are the readings
this oracle and the CUDA path share (each stated in its function), written plainly in
numpy FP64 with explicit loops over taps and footprints.  Pins: tests/test_pipeline_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np

# Monomials of the coordinate polynomials: total degree, then the y power ascending --
# (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),(3,0),(2,1),(1,2),(0,3) -- as (p, q) = (x power, y power).
WARP_MONOMIALS = [(d - q, q) for d in range(4) for q in range(d + 1)]

LANCZOS3, BILINEAR = 0, 1
MASK_FRACTION = 0.01  # an output pixel is masked when more than 1 % of |weight| is on bad taps


# ----------------------------------------------------------------------------- step 4


def warp_eval(warp, x, y):
    """Template coordinates (u, v) of science pixel (x, y) (column, row; FP64).

    ``warp`` = dict(degree, x_ref, y_ref, cu, cv): u = sum_j cu[j] (x - x_ref)^p (y - y_ref)^q
    over the first npoly(degree) monomials of WARP_MONOMIALS, v likewise with cv.  A
    polynomial in pixel offsets covers the affine part of two WCS solutions and a low-order
    (SIP-like) distortion between them; the caller fits it from the two WCS."""
    dx, dy = x - warp["x_ref"], y - warp["y_ref"]
    n = (warp["degree"] + 1) * (warp["degree"] + 2) // 2
    u = v = 0.0
    for j in range(n):
        p, q = WARP_MONOMIALS[j]
        m = dx ** p * dy ** q
        u = u + warp["cu"][j] * m
        v = v + warp["cv"][j] * m
    return u, v


def warp_jacobian(warp, x, y):
    """d(u, v)/d(x, y) at (x, y): [[du/dx, du/dy], [dv/dx, dv/dy]] (FP64, term by term)."""
    dx, dy = x - warp["x_ref"], y - warp["y_ref"]
    n = (warp["degree"] + 1) * (warp["degree"] + 2) // 2
    J = np.zeros((2, 2))
    for j in range(n):
        p, q = WARP_MONOMIALS[j]
        ddx = p * dx ** (p - 1) * dy ** q if p > 0 else 0.0
        ddy = q * dx ** p * dy ** (q - 1) if q > 0 else 0.0
        J[0, 0] += warp["cu"][j] * ddx
        J[0, 1] += warp["cu"][j] * ddy
        J[1, 0] += warp["cv"][j] * ddx
        J[1, 1] += warp["cv"][j] * ddy
    return J


def lanczos3(t):
    """Lanczos window a = 3: sinc(t) sinc(t / 3) for |t| < 3, sinc(t) = sin(pi t) / (pi t);
    exactly 1 at t = 0 and exactly 0 at the other integers and for |t| >= 3."""
    if t == 0.0:
        return 1.0
    if abs(t) >= 3.0 or float(t).is_integer():
        return 0.0
    return math.sin(math.pi * t) * math.sin(math.pi * t / 3.0) * 3.0 / (math.pi * math.pi * t * t)


def _taps(f, method):
    """(offsets, weights) along one axis for fractional position f in [0, 1): Lanczos-3 uses
    the six samples floor - 2 .. floor + 3, bilinear the two samples floor, floor + 1."""
    if method == LANCZOS3:
        offs = range(-2, 4)
        return list(offs), [lanczos3(f - j) for j in offs]
    return [0, 1], [1.0 - f, f]


def _interp_one(img, mask, u, v, method, zero_outside):
    """One interpolated value at template coordinates (u, v) and its bad-weight fraction.

    Reading (the paper fixes no interpolation): separable taps w_ij = w_i(v) w_j(u); a tap
    is bad when it falls outside the template or on a masked pixel; bad taps contribute no
    value (their pixels are never read), the sum is normalised by the weight of ALL taps;
    with zero_outside the outside taps are plain zeros and not bad (PSF stamps)."""
    ny, nx = img.shape
    iu, iv = math.floor(u), math.floor(v)
    ox, wx = _taps(u - iu, method)
    oy, wy = _taps(v - iv, method)
    acc = wsum = wabs = wbad = 0.0
    for a, wa in zip(oy, wy):
        for b, wb in zip(ox, wx):
            w = wa * wb
            if w == 0.0:
                continue
            wsum += w
            wabs += abs(w)
            r, c = iv + a, iu + b
            inside = 0 <= r < ny and 0 <= c < nx
            if not inside:
                if not zero_outside:
                    wbad += abs(w)
                continue
            if mask is not None and mask[r, c] != 0:
                wbad += abs(w)
                continue
            acc += w * float(img[r, c])
    return acc / wsum, (wbad / wabs if wabs > 0 else 0.0)


def resample(img, warp, out_shape, mask=None, method=LANCZOS3, flux=False, zero_outside=False):
    """Resample the template onto the science grid (step 4).

    out[y, x] = interpolated template at (u, v) = warp(x, y), times |det J(x, y)| when
    ``flux`` (pixel values are fluxes and the pixel area changes); out_mask[y, x] = 1 when
    the fraction of |weight| on bad taps exceeds MASK_FRACTION.  Returns (out, out_mask,
    bad_fraction); the fraction lets a test tell decisions that sit on the threshold."""
    ny, nx = out_shape
    out = np.zeros(out_shape)
    frac = np.zeros(out_shape)
    for y in range(ny):
        for x in range(nx):
            u, v = warp_eval(warp, float(x), float(y))
            val, fr = _interp_one(img, mask, u, v, method, zero_outside)
            if flux:
                val *= abs(np.linalg.det(warp_jacobian(warp, float(x), float(y))))
            out[y, x], frac[y, x] = val, fr
    return out, (frac > MASK_FRACTION).astype(np.uint8), frac


def resample_pixels(img, warp, ys, xs, mask=None, method=LANCZOS3, flux=False, zero_outside=False):
    """resample() at the listed output pixels only (any frame size): (values, bad fractions)."""
    vals, fracs = [], []
    for y, x in zip(ys, xs):
        u, v = warp_eval(warp, float(x), float(y))
        val, fr = _interp_one(img, mask, u, v, method, zero_outside)
        if flux:
            val *= abs(np.linalg.det(warp_jacobian(warp, float(x), float(y))))
        vals.append(val)
        fracs.append(fr)
    return np.array(vals), np.array(fracs)


def psf_warp(warp, x, y, K):
    """The affine map that aligns a K x K template PSF stamp (centre c = (K - 1) / 2) to the
    science frame at science position (x, y): stamp offset d maps to J(x, y) d, i.e.
    u = c + J00 (s - c) + J01 (r - c), v = c + J10 (s - c) + J11 (r - c) for output stamp
    pixel (r, s)."""
    J = warp_jacobian(warp, x, y)
    c = (K - 1) / 2.0
    cu = [c, J[0, 0], J[0, 1]] + [0.0] * 7
    cv = [c, J[1, 0], J[1, 1]] + [0.0] * 7
    return dict(degree=1, x_ref=c, y_ref=c, cu=cu, cv=cv)


def align_psf(psf, warp, x, y, method=LANCZOS3):
    """Template PSF stamp resampled onto the science pixel grid at (x, y) (step 4 aligns the
    template's PSF with its image): zeros outside the stamp, flux-conserving (|det J|)."""
    K = psf.shape[0]
    out, _, _ = resample(psf, psf_warp(warp, x, y, K), (K, K), None, method, flux=True, zero_outside=True)
    return out


# ----------------------------------------------------------------------------- step 7


def matching_kernel(theta, L, dk, nxy, x, y):
    """The fitted matching kernel at pixel (x, y): K(dy, dx) = sum_pq a_{pq,(dx,dy)} w_pq(x, y)
    with w_pq = xh^p yh^q, xh = 2x/(Nx-1) - 1, yh = 2y/(Ny-1) - 1 (theta's kernel block: pq-major
    blocks of L^2 lags, dy outer).  Returned as an L x L array indexed [dy + h, dx + h]."""
    ny, nx = nxy
    xh = 2.0 * x / (nx - 1) - 1.0 if nx > 1 else 0.0
    yh = 2.0 * y / (ny - 1) - 1.0 if ny > 1 else 0.0
    Kk = np.zeros((L, L))
    npk = (dk + 1) * (dk + 2) // 2
    for idx in range(npk):
        p, q = _mono(idx)
        w = xh ** p * yh ** q
        Kk += w * np.asarray(theta[idx * L * L:(idx + 1) * L * L], dtype=np.float64).reshape(L, L)
    return Kk


def _mono(idx):
    d = 0
    while (d + 1) * (d + 2) // 2 <= idx:
        d += 1
    q = idx - d * (d + 1) // 2
    return d - q, q


def _dft2_centred(stamp, M):
    """DFT on the M x M cyclic grid of a centred odd stamp: value at offset d sits at index
    d mod M; X(k) = sum_d x(d) exp(-2 pi i k.d / M), written as explicit DFT matrices."""
    K = stamp.shape[0]
    c = (K - 1) // 2
    g = np.zeros((M, M))
    for a in range(K):
        for b in range(K):
            g[(a - c) % M, (b - c) % M] += stamp[a, b]
    n = np.arange(M)
    F = np.exp(-2j * np.pi * np.outer(n, n) / M)
    return F @ g @ F.T


def _idft2_centred(X, M):
    """Real part of the inverse DFT, returned as an M x M stamp centred on (M - 1) / 2."""
    n = np.arange(M)
    Fi = np.exp(2j * np.pi * np.outer(n, n) / M)
    g = (Fi @ X @ Fi.T).real / (M * M)
    c = (M - 1) // 2
    out = np.zeros((M, M))
    for a in range(M):
        for b in range(M):
            out[a, b] = g[(a - c) % M, (b - c) % M]
    return out


def decorrelation_kernel(psf_sci, psf_tmpl, kern, sigma_sci, sigma_tmpl, M, floor=1e-8):
    """Decorrelation kernel on the M x M grid (step 7) and the decorrelated science PSF.

    Reading (the paper cites the kernel without a formula): the fit matches S' = S (x) P_T
    against T' = T (x) P_S, so white pixel noise sigma_S, sigma_T leaves D = S' - K (x) T' with
    the noise spectrum  den(k) = sigma_S^2 |P_T(k)|^2 + sigma_T^2 |K(k)|^2 |P_S(k)|^2.  The filter
    whitens it at unit gain for a flux:
        Phi(k) = sqrt(num / max(den(k), floor * num)),  num = sigma_S^2 + K(0)^2 sigma_T^2,
    so Phi(0) = 1 for unit-sum stamps.  phi = IDFT(Phi) on the M x M grid (M odd, every stamp
    centred on it), returned centred; the decorrelated science PSF is IDFT(P_S P_T Phi)."""
    for s in (psf_sci, psf_tmpl, kern):
        if s.shape[0] > M or s.shape[0] % 2 == 0:
            raise ValueError("stamps must be odd and no larger than M")
    Ps, Pt, Kh = _dft2_centred(psf_sci, M), _dft2_centred(psf_tmpl, M), _dft2_centred(kern, M)
    num = sigma_sci ** 2 + (Kh[0, 0].real ** 2) * sigma_tmpl ** 2
    den = sigma_sci ** 2 * np.abs(Pt) ** 2 + sigma_tmpl ** 2 * np.abs(Kh) ** 2 * np.abs(Ps) ** 2
    Phi = np.sqrt(num / np.maximum(den, floor * num))
    return _idft2_centred(Phi, M), _idft2_centred(Ps * Pt * Phi, M)


# ----------------------------------------------------------------------------- step 9


def source_pixel(x, y):
    """Footprint centre of a source at (x, y): the nearest pixel, halves rounded up
    (floor(x + 0.5)), and the remaining offset (fx, fy) in [-0.5, 0.5)."""
    X, Y = math.floor(x + 0.5), math.floor(y + 0.5)
    return X, Y, x - X, y - Y


def shifted_psf(psf, fx, fy):
    """The PSF stamp moved by the sub-pixel offset (fx, fy): model(a, b) = psf interpolated
    (Lanczos-3, zeros outside the stamp) at stamp position (c + a - fy, c + b - fx)."""
    K = psf.shape[0]
    c = (K - 1) // 2
    out = np.zeros((K, K))
    for a in range(-c, c + 1):
        for b in range(-c, c + 1):
            out[a + c, b + c], _ = _interp_one(psf, None, c + b - fx, c + a - fy, LANCZOS3, True)
    return out


def forced_photometry(D, psf, x, y, weight=None, mask=None, background=False):
    """Weighted least-squares PSF flux at a fixed position (step 9).

    Reading: over the K x K footprint around source_pixel(x, y) (pixels inside the frame,
    unmasked, weight > 0), minimise sum w (D - f P - b)^2 with P = shifted_psf(psf, fx, fy),
    b = 0 unless ``background``.  Returns (f, sigma_f, b, chi2, n): sigma_f the formal error
    sqrt([(A^T W A)^-1]_ff) for inverse-variance weights, chi2 = sum w r^2, n pixels used."""
    ny, nx = D.shape
    X, Y, fx, fy = source_pixel(x, y)
    P = shifted_psf(psf, fx, fy)
    K = psf.shape[0]
    c = (K - 1) // 2
    rows, rhs, wts = [], [], []
    for a in range(-c, c + 1):
        for b in range(-c, c + 1):
            r, s = Y + a, X + b
            if not (0 <= r < ny and 0 <= s < nx):
                continue
            if mask is not None and mask[r, s] != 0:
                continue
            w = 1.0 if weight is None else float(weight[r, s])
            if w <= 0.0:
                continue
            rows.append([P[a + c, b + c], 1.0] if background else [P[a + c, b + c]])
            rhs.append(float(D[r, s]))
            wts.append(w)
    A, d, w = np.array(rows), np.array(rhs), np.array(wts)
    sw = np.sqrt(w)
    sol, *_ = np.linalg.lstsq(A * sw[:, None], d * sw, rcond=None)
    cov = np.linalg.inv((A * w[:, None]).T @ A)
    r = d - A @ sol
    f = sol[0]
    bg = sol[1] if background else 0.0
    return f, math.sqrt(cov[0, 0]), bg, float(np.sum(w * r * r)), len(d)
