"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws and renders data: stars, point-spread functions, sky, noise and
masks.  It holds none of the fit or subtraction arithmetic and imports nothing else from
the package, so both the CUDA path and the CPU oracle can take their inputs from it.

The paper's images are OpenUniverse 2024 Roman simulations (Sec. "Statement of need"),
which are not available here; these generators stand in for them, using the Roman frame
size 4088 x 4088 (Sec. "GPU acceleration and performance") and cutouts no smaller than the
1000 x 1000 px the paper still calls high quality (same section).

Recipes (seed fixes everything, numpy PCG64):
  * ``gaussian_pair``  -- 64 x 64 float64: template = 30 Gaussian stars (sigma 1.2 px,
    lognormal flux mu=8, sigma=1, uniform positions) + sky 100 + N(0, 3) noise;
    science = template cyclically convolved with a fixed 5 x 5 positive unit-sum kernel
    + 2.5 + N(0, 3).
  * ``roman_pair``     -- float32 frames with Moffat (beta=2.5) stars whose FWHM varies
    linearly 1.8 -> 2.4 px along x in the template and along y in the science image,
    Poisson(sky 80 e- + stars) with the known sky subtracted afterwards, and a union of two
    Bernoulli(0.005) masks (byte 1 = masked).
  * ``psf_field`` / ``psf_stamps`` / ``psf_grid_pair`` -- training data of the warm-start
    network: a random pair of spatially varying elliptical Moffat PSF fields (FWHM linear
    in the normalised coordinates, within 1.6 .. 2.8 px; ellipticity <= 0.15 at a random
    position angle), their 32 x 32 stamps at the 3 x 3 cell centres, and a noise-free
    frame pair with stars on a regular grid drawn with those fields (stamps scaled to unit
    mean).
  * ``cnn_init`` -- seeded He-normal initial weights of that network.
"""
from __future__ import annotations

import numpy as np

MOFFAT_BETA = 2.5


def moffat_alpha(fwhm: float, beta: float = MOFFAT_BETA) -> float:
    """Moffat core width alpha for a given FWHM: FWHM = 2 alpha sqrt(2^(1/beta) - 1)."""
    return fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))


def _render(ny, nx, xs, ys, flux, profile, radius):
    """Sum unit-normalised stamps (pixel-centre sampling) into a cyclic ny x nx frame."""
    img = np.zeros(ny * nx, dtype=np.float64)
    off = np.arange(-radius, radius + 1)
    oy, ox = np.meshgrid(off, off, indexing="ij")
    batch = 256
    for s in range(0, len(xs), batch):
        x = xs[s:s + batch, None, None]
        y = ys[s:s + batch, None, None]
        cx = np.floor(x + 0.5).astype(np.int64)
        cy = np.floor(y + 0.5).astype(np.int64)
        px = cx + ox[None]
        py = cy + oy[None]
        r2x = (px - x) ** 2
        r2y = (py - y) ** 2
        prof = profile(r2x, r2y, s, s + batch)
        prof /= prof.sum(axis=(1, 2), keepdims=True)
        prof *= flux[s:s + batch, None, None]
        flat = (np.mod(py, ny) * nx + np.mod(px, nx)).ravel()
        np.add.at(img, flat, prof.ravel())
    return img.reshape(ny, nx)


def fixed_kernel5() -> np.ndarray:
    """The fixed 5 x 5 positive, unit-sum kernel used to make the small science image."""
    off = np.arange(-2, 3)
    dy, dx = np.meshgrid(off, off, indexing="ij")
    k = np.exp(-((dx - 0.3) ** 2 + (dy + 0.2) ** 2) / (2.0 * 0.9 ** 2))
    return k / k.sum()


def _cyclic_convolve(img, kern):
    """out(u) = sum_d kern(d) img((u - d) mod N), d centred on the kernel's middle."""
    h = kern.shape[0] // 2
    out = np.zeros_like(img)
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            out += kern[dy + h, dx + h] * np.roll(img, shift=(dy, dx), axis=(0, 1))
    return out


def gaussian_pair(seed: int = 0, size: int = 64, n_stars: int = 30):
    """Small float64 pair: returns (sci, tmpl, kernel5, background)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(0, size, n_stars)
    ys = rng.uniform(0, size, n_stars)
    flux = np.exp(rng.normal(8.0, 1.0, n_stars))
    sig = 1.2

    def gauss(r2x, r2y, a, b):
        return np.exp(-(r2x + r2y) / (2 * sig * sig))

    stars = _render(size, size, xs, ys, flux, gauss, radius=6)
    tmpl = stars + 100.0 + rng.normal(0.0, 3.0, (size, size))
    kern = fixed_kernel5()
    bg = 2.5
    sci = _cyclic_convolve(tmpl, kern) + bg + rng.normal(0.0, 3.0, (size, size))
    return sci.astype(np.float64), tmpl.astype(np.float64), kern, bg


def roman_pair(ny: int = 4088, nx: int = 4088, seed: int = 1000, n_stars: int | None = None,
               fwhm=(1.8, 2.4), sky: float = 80.0, mask_frac: float = 0.005,
               flux_mode: str = "lognormal", dtype=np.float32, radius: int = 12, field=None):
    """Roman-like pair: returns (sci, tmpl, mask) with mask bytes 1 = masked.

    ``n_stars`` defaults to 3000 per 4088^2 frame, scaled by area.  ``flux_mode`` is
    "lognormal" (exp N(8, 1) e-) or "dynamic" (log-uniform over 1e2..1e7 e-, a 1e5 range).
    ``field`` (a PSF-field pair as ``psf_field`` / ``roman_field`` return) draws each star
    with the field's PSF at its position instead of the default fields (FWHM along x in the
    template, along y in the science image).
    """
    if field is not None:
        return _roman_pair_field(ny, nx, seed, n_stars, field, sky, mask_frac, flux_mode, dtype, radius)
    rng = np.random.Generator(np.random.PCG64(seed))
    if n_stars is None:
        n_stars = max(1, int(round(3000 * ny * nx / 4088.0 ** 2)))
    xs = rng.uniform(0, nx, n_stars)
    ys = rng.uniform(0, ny, n_stars)
    if flux_mode == "lognormal":
        flux = np.exp(rng.normal(8.0, 1.0, n_stars))
    elif flux_mode == "dynamic":
        flux = 10.0 ** rng.uniform(2.0, 7.0, n_stars)
    else:
        raise ValueError(flux_mode)
    f0, f1 = fwhm
    ax_t = moffat_alpha(f0 + (f1 - f0) * xs / max(nx - 1, 1))  # template: varies along x
    ax_s = moffat_alpha(f0 + (f1 - f0) * ys / max(ny - 1, 1))  # science: varies along y

    def moffat(alpha):
        def prof(r2x, r2y, a, b):
            al = alpha[a:b, None, None]
            return (1.0 + (r2x + r2y) / (al * al)) ** (-MOFFAT_BETA)
        return prof

    tmpl_model = _render(ny, nx, xs, ys, flux, moffat(ax_t), radius)
    sci_model = _render(ny, nx, xs, ys, flux, moffat(ax_s), radius)
    tmpl = rng.poisson(tmpl_model + sky).astype(np.float64) - sky
    sci = rng.poisson(sci_model + sky).astype(np.float64) - sky
    m1 = rng.random((ny, nx)) < mask_frac
    m2 = rng.random((ny, nx)) < mask_frac
    mask = (m1 | m2).astype(np.uint8)
    return sci.astype(dtype), tmpl.astype(dtype), mask


def _roman_pair_field(ny, nx, seed, n_stars, field, sky, mask_frac, flux_mode, dtype, radius):
    """``roman_pair`` with the stars drawn by a given pair of PSF fields (same random stream
    for positions, fluxes, noise and masks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if n_stars is None:
        n_stars = max(1, int(round(3000 * ny * nx / 4088.0 ** 2)))
    xs = rng.uniform(0, nx, n_stars)
    ys = rng.uniform(0, ny, n_stars)
    if flux_mode == "lognormal":
        flux = np.exp(rng.normal(8.0, 1.0, n_stars))
    elif flux_mode == "dynamic":
        flux = 10.0 ** rng.uniform(2.0, 7.0, n_stars)
    else:
        raise ValueError(flux_mode)
    xh = 2.0 * xs / max(nx - 1, 1) - 1.0
    yh = 2.0 * ys / max(ny - 1, 1) - 1.0
    models = {}
    for key in ("tmpl", "sci"):
        fd = field[key]
        al = moffat_alpha(_fwhm_at(fd, xh, yh))
        models[key] = np.zeros(ny * nx)
        for s0 in range(0, n_stars, 512):
            sl = slice(s0, s0 + 512)
            models[key] += _render_signed(ny, nx, xs[sl], ys[sl], flux[sl], al[sl], fd["e"], fd["phi"],
                                          radius).ravel()
    tmpl = rng.poisson(models["tmpl"].reshape(ny, nx) + sky).astype(np.float64) - sky
    sci = rng.poisson(models["sci"].reshape(ny, nx) + sky).astype(np.float64) - sky
    m1 = rng.random((ny, nx)) < mask_frac
    m2 = rng.random((ny, nx)) < mask_frac
    mask = (m1 | m2).astype(np.uint8)
    return sci.astype(dtype), tmpl.astype(dtype), mask


def linear_field(theta_sci: float, theta_tmpl: float, fwhm=(1.8, 2.4)):
    """Round Moffat fields whose FWHM runs linearly from fwhm[0] to fwhm[1] across the frame
    along the direction theta (radians from the x axis), one direction per image;
    ``roman_field`` is theta_sci = pi/2, theta_tmpl = 0."""
    c, g = 0.5 * (fwhm[0] + fwhm[1]), 0.5 * (fwhm[1] - fwhm[0])

    def one(th):
        cx, sy = np.cos(th), np.sin(th)
        n = abs(cx) + abs(sy)  # the extreme of cx xh + sy yh over [-1, 1]^2
        return dict(f0=c, fx=g * cx / n, fy=g * sy / n, e=0.0, phi=0.0)

    return dict(sci=one(theta_sci), tmpl=one(theta_tmpl))


def cutout_sizes(n: int, seed: int, choices=(512, 1024, 1536, 2048)):
    """Square cutout sizes drawn uniformly from ``choices``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(c) for c in rng.choice(np.asarray(choices), size=n)]


# ---------------------------------------------------------------------------------------
# PSF fields and stamps for the warm-start network

STAMP = 32
GRID3 = (-2.0 / 3.0, 0.0, 2.0 / 3.0)  # normalised coordinates of the 3 x 3 cell centres


def _moffat_ell(dx, dy, alpha, e, phi, beta=MOFFAT_BETA):
    """Elliptical Moffat with axis ratio 1 - e and the area of the round profile of width
    alpha (semi-axes alpha / sqrt(1 - e), alpha sqrt(1 - e))."""
    q = 1.0 - e
    a, b = alpha / np.sqrt(q), alpha * np.sqrt(q)
    c, s = np.cos(phi), np.sin(phi)
    u = c * dx + s * dy
    v = -s * dx + c * dy
    return (1.0 + (u / a) ** 2 + (v / b) ** 2) ** (-beta)


def _draw_field(rng, fwhm_range, e_max):
    lo, hi = fwhm_range
    f0 = rng.uniform(lo + 0.05, hi - 0.05)
    r = min(f0 - lo, hi - f0)
    fx, fy = rng.uniform(-r, r, 2)
    if abs(fx) + abs(fy) > r:
        sc = r / (abs(fx) + abs(fy))
        fx, fy = fx * sc, fy * sc
    return dict(f0=f0, fx=fx, fy=fy, e=rng.uniform(0.0, e_max), phi=rng.uniform(0.0, np.pi))


def psf_field(seed: int, fwhm_range=(1.6, 2.8), e_max: float = 0.15):
    """A random (science, template) pair of PSF fields: FWHM(xh, yh) = f0 + fx xh + fy yh
    stays inside ``fwhm_range`` over [-1, 1]^2; ellipticity and angle are constant."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return dict(sci=_draw_field(rng, fwhm_range, e_max), tmpl=_draw_field(rng, fwhm_range, e_max))


def roman_field(fwhm=(1.8, 2.4)):
    """The PSF fields ``roman_pair`` draws with: round Moffats, FWHM linear along x in the
    template and along y in the science image."""
    f0, f1 = fwhm
    c, g = 0.5 * (f0 + f1), 0.5 * (f1 - f0)
    return dict(sci=dict(f0=c, fx=0.0, fy=g, e=0.0, phi=0.0), tmpl=dict(f0=c, fx=g, fy=0.0, e=0.0, phi=0.0))


def _fwhm_at(fd, xh, yh):
    return fd["f0"] + fd["fx"] * xh + fd["fy"] * yh


def psf_stamps(field, size: int = STAMP) -> np.ndarray:
    """float32 [18][size][size]: stamps of unit mean (sum size^2, so that the network sees
    values of order one) centred on pixel (size/2, size/2) at the 3 x 3 cell centres
    (row-major, yh outer), science then template for each cell."""
    off = np.arange(size) - size // 2
    dy, dx = np.meshgrid(off, off, indexing="ij")
    out = np.zeros((18, size, size), dtype=np.float64)
    k = 0
    for yh in GRID3:
        for xh in GRID3:
            for key in ("sci", "tmpl"):
                fd = field[key]
                st = _moffat_ell(dx, dy, moffat_alpha(_fwhm_at(fd, xh, yh)), fd["e"], fd["phi"])
                out[k] = st * (size * size / st.sum())
                k += 1
    return out.astype(np.float32)


def psf_grid_pair(field, seed: int, size: int = 256, spacing: int = 32, flux: float = 1e4,
                  radius: int = 12, dtype=np.float32):
    """Noise-free (sci, tmpl) frames with one star per ``spacing`` x ``spacing`` cell (random
    sub-pixel offset), each drawn with the field's PSF at its position."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.arange(spacing // 2, size, spacing, dtype=np.float64)
    ys, xs = np.meshgrid(c, c, indexing="ij")
    xs = xs.ravel() + rng.uniform(-0.5, 0.5, xs.size)
    ys = ys.ravel() + rng.uniform(-0.5, 0.5, ys.size)
    fl = np.full(xs.size, flux)
    xh = 2.0 * xs / (size - 1) - 1.0
    yh = 2.0 * ys / (size - 1) - 1.0

    out = []
    for key in ("sci", "tmpl"):
        fd = field[key]
        al = moffat_alpha(_fwhm_at(fd, xh, yh))
        out.append(_render_signed(size, size, xs, ys, fl, al, fd["e"], fd["phi"], radius))
    return out[0].astype(dtype), out[1].astype(dtype)


def _render_signed(ny, nx, xs, ys, flux, alpha, e, phi, radius):
    """Like ``_render`` for elliptical profiles (which need signed offsets)."""
    img = np.zeros(ny * nx, dtype=np.float64)
    off = np.arange(-radius, radius + 1)
    oy, ox = np.meshgrid(off, off, indexing="ij")
    x = xs[:, None, None]
    y = ys[:, None, None]
    cx = np.floor(x + 0.5).astype(np.int64)
    cy = np.floor(y + 0.5).astype(np.int64)
    px = cx + ox[None]
    py = cy + oy[None]
    prof = _moffat_ell(px - x, py - y, alpha[:, None, None], e, phi)
    prof /= prof.sum(axis=(1, 2), keepdims=True)
    prof *= flux[:, None, None]
    np.add.at(img, (np.mod(py, ny) * nx + np.mod(px, nx)).ravel(), prof.ravel())
    return img.reshape(ny, nx)


def training_sample(seed: int, size: int = 256):
    """One training sample of the warm-start network: (sci, tmpl, stamps) float32 for the PSF
    field pair ``psf_field(seed)`` (frames from ``psf_grid_pair``, stamps from ``psf_stamps``)."""
    field = psf_field(seed)
    S, T = psf_grid_pair(field, seed=seed, size=size)
    return S, T, psf_stamps(field)


def training_chunk(args):
    """Training samples seed0 .. seed0 + count - 1 stacked: (sci, tmpl, stamps).  A process-
    pool worker function: it needs numpy only."""
    seed0, count, size = args
    out = [training_sample(seed0 + i, size) for i in range(count)]
    return tuple(np.stack([o[j] for o in out]) for j in range(3))


def cnn_init(n_out: int, seed: int) -> np.ndarray:
    """Seeded He-normal weights (zero biases) of the warm-start network, as one flat float32
    vector in the network's parameter order: 4 x (conv W [32][cin][3][3], b [32]) with
    cin = 18, 32, 32, 32, then linear W [n_out][128], b [n_out]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for cin in (18, 32, 32, 32):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (cin * 9)), (32, cin, 3, 3)).ravel())
        parts.append(np.zeros(32))
    parts.append(rng.normal(0.0, np.sqrt(2.0 / 128), (n_out, 128)).ravel())
    parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float32)


def psf_stamp_at(field, key: str, xh: float, yh: float, K: int = 25) -> np.ndarray:
    """float32 K x K (K odd) unit-sum stamp of the ``key`` ("sci" or "tmpl") PSF of a field
    at normalised position (xh, yh), centred on the middle element (cross-convolution,
    decorrelation and photometry inputs)."""
    off = np.arange(K) - K // 2
    dy, dx = np.meshgrid(off, off, indexing="ij")
    fd = field[key]
    st = _moffat_ell(dx, dy, moffat_alpha(_fwhm_at(fd, xh, yh)), fd["e"], fd["phi"])
    return (st / st.sum()).astype(np.float32)
