"""Steps 4, 7 and 9 of the pipeline (Sec. "Pipeline steps") through the C ABI against the
FP64 oracle (oracle/pipeline.py).

Tolerances, from the arithmetic:
* resampling: FP32 weights and sums over at most 36 taps and a coordinate error of a few
  1e-6 pixel (FP32 Taylor part about each tile corner) -> |out - ref| <= 1e-5 max|ref|;
  masks bit-exact except where the oracle's bad-weight fraction lies within 1e-4 of the
  1 % threshold (there FP32 and FP64 may decide differently; both answers are valid);
* decorrelation kernel: FP64 DFTs, FP32 output -> |phi - ref| <= 1e-6 max|ref|; applied
  with sfft_cross_convolve (FP32) -> 1e-5 max|ref| like the cross-convolution;
* photometry: FP32 model weights (relative error ~1e-7), FP64 sums -> flux and its error
  within 1e-5 relative, background within 1e-5 of (|b| + sigma_f), chi^2 within 1e-4
  relative, pixel counts and status exact.
Sizes cross several 32 x 32 tiles with ragged edges; the full-size cases (4088^2) compare
sampled pixels and jobs."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import pipeline as po
from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    sfft_build.build()
    sfft.load_library()


def moffat_stamp(K, fwhm, seed):
    rng = np.random.default_rng(seed)
    off = np.arange(K) - K // 2
    dy, dx = np.meshgrid(off, off, indexing="ij")
    cy, cx = rng.uniform(-0.4, 0.4, 2)
    al = synth.moffat_alpha(fwhm)
    p = (1.0 + ((dx - cx) ** 2 + (dy - cy) ** 2) / al ** 2) ** (-synth.MOFFAT_BETA)
    return (p / p.sum()).astype(np.float32)


def warp_dict(w: sfft.sfft_warp):
    return dict(degree=w.degree, x_ref=w.x_ref, y_ref=w.y_ref, cu=list(w.cu), cv=list(w.cv))


def rot_warp(th, s, tx, ty, xr, yr, cubic=0.0):
    c, sn = s * math.cos(th), s * math.sin(th)
    cu = [xr + tx, c, -sn, 0, 0, 0, cubic, 0, 0, 0]
    cv = [yr + ty, sn, c, 0, 0, 0, 0, 0, cubic, 0]
    return sfft.make_warp(3 if cubic else 1, cu, cv, xr, yr)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def check_mask(got, ref, frac):
    settled = np.abs(frac - po.MASK_FRACTION) > 1e-4
    assert np.array_equal(got[settled], ref[settled])


# ------------------------------------------------------------------ step 4


RES_CASES = [
    # in shape, out shape, warp, method, flags, dtype, masked, pitch pad
    ((110, 120), (96, 130), rot_warp(0.21, 1.03, 2.7, -1.4, 60, 48), sfft.LANCZOS3, 0, np.float32, True, 0),
    ((110, 120), (100, 100), rot_warp(-0.4, 0.97, 5.2, 3.1, 50, 50, 2e-6), sfft.BILINEAR, sfft.RESAMPLE_FLUX,
     np.float32, True, 0),
    ((64, 80), (70, 90), rot_warp(0.0, 1.0, 0.0, 0.0, 0, 0), sfft.LANCZOS3, 0, np.float32, True, 0),       # identity
    ((64, 80), (64, 80), rot_warp(0.0, 1.0, -3.0, 2.0, 0, 0), sfft.LANCZOS3, 0, np.float64, True, 6),     # integer shift
    ((90, 70), (50, 60), rot_warp(1.1, 1.2, 10.5, 3.25, 30, 20, -4e-6), sfft.LANCZOS3,
     sfft.RESAMPLE_FLUX, np.float64, False, 0),
    ((40, 40), (33, 17), rot_warp(0.0, 1.0, 5e9, 0.0, 0, 0), sfft.LANCZOS3, 0, np.float32, True, 0),     # far outside
]


@pytest.mark.parametrize("case", range(len(RES_CASES)))
def test_resample_matches_oracle(case):
    ishape, oshape, w, method, flags, dt, masked, pad = RES_CASES[case]
    S, T, M = synth.roman_pair(*ishape, seed=31 + case, n_stars=ishape[0] * ishape[1] // 250)
    img = T.astype(dt)
    mask = M if masked else None
    ref, refm, frac = po.resample(img.astype(np.float64), warp_dict(w), oshape, mask,
                                  po.LANCZOS3 if method == sfft.LANCZOS3 else po.BILINEAR,
                                  flux=bool(flags & sfft.RESAMPLE_FLUX))
    pitch = ishape[1] + pad
    src = np.zeros((ishape[0], pitch), dt)
    src[:, :ishape[1]] = img
    msk = np.zeros((ishape[0], pitch), np.uint8)
    if masked:
        msk[:, :ishape[1]] = M
    out = torch.full((oshape[0], oshape[1] + pad), 7.0, dtype=torch.float64 if dt == np.float64 else torch.float32,
                     device=DEV)
    om = torch.full((oshape[0], oshape[1] + pad), 9, dtype=torch.uint8, device=DEV)
    sfft.sfft_resample(w, dev(src), out, dev(msk) if masked else None, om, method, flags,
                       sfft.F64 if dt == np.float64 else sfft.F32, in_shape=ishape, out_shape=oshape,
                       in_pitch=pitch, out_pitch=oshape[1] + pad)
    torch.cuda.synchronize()
    got = out.cpu().numpy()[:, :oshape[1]].astype(np.float64)
    gm = om.cpu().numpy()[:, :oshape[1]]
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(got - ref).max() / scale
    print("resample case %d: max err / max|ref| = %.3e, masked %d" % (case, err, int(refm.sum())))
    assert err <= 1e-5
    check_mask(gm, refm, frac)
    if case in (2, 3):  # identity and integer shifts are exact
        assert np.array_equal(got, ref) and np.array_equal(gm, refm)
    if pad:
        assert np.all(om.cpu().numpy()[:, oshape[1]:] == 9)


def test_align_psf_matches_oracle():
    P = moffat_stamp(25, 2.0, 1)
    w = rot_warp(0.33, 1.05, 0, 0, 0, 0, 3e-7)
    out = torch.empty((25, 25), dtype=torch.float32, device=DEV)
    sfft.sfft_align_psf(w, 1500.0, 2200.0, dev(P), out)
    torch.cuda.synchronize()
    ref = po.align_psf(P.astype(np.float64), warp_dict(w), 1500.0, 2200.0)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_resample_rejects_bad_arguments():
    w = rot_warp(0.1, 1.0, 0, 0, 0, 0)
    a = torch.zeros((16, 16), device=DEV)
    b = torch.zeros((16, 16), device=DEV)
    for kw in (dict(method=5), dict(flags=8)):
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_resample(w, a, b, **kw)
        assert ei.value.status == sfft.ERR_INVALID_ARG
    with pytest.raises(sfft.SfftError):
        sfft.sfft_resample(w, a, a)  # aliasing
    bad = sfft.make_warp(1, [0, 1, 0], [0, 0, 1])
    bad.degree = 4
    with pytest.raises(sfft.SfftError):
        sfft.sfft_resample(bad, a, b)


@pytest.mark.slow
def test_resample_full_size_sampled():
    """4088^2 template with a 0.3 degree rotation, a 1e-4 scale change, a sub-pixel shift and
    a cubic distortion, Lanczos-3 with its mask; sampled pixels against the oracle."""
    S, T, M = synth.roman_pair(4088, 4088, seed=1001)
    w = rot_warp(math.radians(0.3), 1.0001, 3.37, -2.81, 2043.5, 2043.5, 1e-10)
    out = torch.empty((4088, 4088), dtype=torch.float32, device=DEV)
    om = torch.empty((4088, 4088), dtype=torch.uint8, device=DEV)
    sfft.sfft_resample(w, dev(T), out, dev(M), om, sfft.LANCZOS3, 0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    ys = np.concatenate([rng.integers(0, 4088, 3000), [0, 0, 4087, 4087, 2043]])
    xs = np.concatenate([rng.integers(0, 4088, 3000), [0, 4087, 0, 4087, 2043]])
    ref, frac = po.resample_pixels(T.astype(np.float64), warp_dict(w), ys, xs, M)
    got = out.cpu().numpy()[ys, xs].astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * float(np.abs(T).max())
    check_mask(om.cpu().numpy()[ys, xs], (frac > po.MASK_FRACTION).astype(np.uint8), frac)


# ------------------------------------------------------------------ step 7


DEC_CASES = [
    # L, dk, K, M, sigma_s, sigma_t, position
    (11, 2, 25, 25, 1.0, 0.8, (1000.5, 3000.0)),
    (11, 1, 21, 31, 2.5, 0.5, (0.0, 4087.0)),
    (5, 0, 1, 9, 1.0, 1.0, (17.0, 40.0)),     # delta PSFs: Phi from the kernel alone
    (15, 3, 25, 29, 1.3, 0.0, (2000.0, 10.0)),  # noiseless template
]


def kernel_theta(L, dk, seed, scale=0.93):
    """A matching kernel near a scaled delta with a weak spatial variation (test data)."""
    rng = np.random.default_rng(seed)
    nk = (dk + 1) * (dk + 2) // 2
    th = rng.normal(0, 2e-3, nk * L * L + 3)
    th[(L * L) // 2] += scale
    return th


@pytest.mark.parametrize("case", range(len(DEC_CASES)))
def test_decorrelation_kernel_matches_oracle(case):
    L, dk, K, M, ss, st, (x, y) = DEC_CASES[case]
    ny = nx = 4088
    if K == 1:
        Ps = Pt = np.ones((1, 1), np.float32)
    else:
        Ps, Pt = moffat_stamp(K, 1.9, 10 + case), moffat_stamp(K, 2.3, 20 + case)
    th = kernel_theta(L, dk, case)
    phi = torch.empty((M, M), dtype=torch.float32, device=DEV)
    pd = torch.empty((M, M), dtype=torch.float32, device=DEV)
    sfft.sfft_decorrelation_kernel(ny, nx, L, dk, dev(th), x, y, dev(Ps), dev(Pt), ss, st, phi, pd)
    torch.cuda.synchronize()
    Kk = po.matching_kernel(th, L, dk, (ny, nx), x, y)
    ref, pref = po.decorrelation_kernel(Ps.astype(np.float64), Pt.astype(np.float64), Kk, ss, st, M)
    e1 = np.abs(phi.cpu().numpy() - ref).max() / np.abs(ref).max()
    e2 = np.abs(pd.cpu().numpy() - pref).max() / np.abs(pref).max()
    print("decorrelation case %d: phi err %.3e, psf err %.3e, max|phi| %.3f" % (case, e1, e2, np.abs(ref).max()))
    assert e1 <= 1e-6 and e2 <= 1e-6


def test_decorrelation_applied_to_a_difference_image():
    """phi (x) D and phi (x) S' in one sfft_cross_convolve call against the oracle."""
    L, dk, K, M = 11, 2, 25, 25
    Ps, Pt = moffat_stamp(K, 1.9, 3), moffat_stamp(K, 2.3, 4)
    th = kernel_theta(L, dk, 9)
    phi = torch.empty((M, M), dtype=torch.float32, device=DEV)
    sfft.sfft_decorrelation_kernel(300, 280, L, dk, dev(th), 150.0, 140.0, dev(Ps), dev(Pt), 1.0, 0.7, phi)
    S, T, _ = synth.roman_pair(300, 280, seed=77, n_stars=300)
    D, Sc = dev(S - 0.93 * T), dev(S)
    Do, So = torch.empty_like(D), torch.empty_like(Sc)
    sfft.sfft_cross_convolve(300, 280, M, D, Sc, phi, phi, Do, So)
    torch.cuda.synchronize()
    p = phi.cpu().numpy().astype(np.float64)
    for got, X in ((Do, S - 0.93 * T), (So, S)):
        ref = oracle.convolve(X.astype(np.float32), p)
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_decorrelation_rejects_bad_arguments():
    z = torch.zeros((25, 25), dtype=torch.float32, device=DEV)
    th = dev(np.zeros(200))
    for args in ((11, 2, 25, 33), (11, 2, 25, 23), (11, 2, 24, 25), (12, 2, 25, 25)):
        L, dk, K, M = args
        with pytest.raises(sfft.SfftError):
            sfft.sfft_decorrelation_kernel(100, 100, L, dk, th, 0, 0, z[:K, :K], z[:K, :K], 1.0, 1.0,
                                           torch.zeros((M, M), dtype=torch.float32, device=DEV))
    with pytest.raises(sfft.SfftError):  # sigma_sci must be positive
        sfft.sfft_decorrelation_kernel(100, 100, 11, 2, th, 0, 0, z, z, 0.0, 1.0, z)


# ------------------------------------------------------------------ step 9


def _phot_compare(jobs_np, K, flags, res):
    for j, r in zip(jobs_np, res):
        ref = po.forced_photometry(j["D"], j["P"], j["x"], j["y"], j.get("W"), j.get("M"),
                                   bool(flags & sfft.PHOT_BACKGROUND))
        f, sf, b, chi2, n = ref
        assert r[5] == 0 and r[4] == n
        assert abs(r[0] - f) <= 1e-5 * abs(f) + 1e-7 * sf
        assert r[1] == pytest.approx(sf, rel=1e-5)
        assert abs(r[2] - b) <= 1e-5 * (abs(b) + sf)
        assert r[3] == pytest.approx(chi2, rel=1e-4, abs=1e-9)


@pytest.mark.parametrize("flags", [0, sfft.PHOT_BACKGROUND])
def test_forced_photometry_matches_oracle(flags):
    rng = np.random.default_rng(5 + flags)
    K = 25
    P = moffat_stamp(K, 2.1, 6)
    imgs = []
    for k, (ny, nx, dt) in enumerate(((200, 180, np.float32), (150, 260, np.float64), (64, 64, np.float32))):
        D = rng.normal(0, 1.0, (ny, nx)).astype(dt)
        W = rng.uniform(0.5, 2.0, (ny, nx)).astype(np.float32)
        M = (rng.random((ny, nx)) < 0.03).astype(np.uint8)
        imgs.append((D, W, M))
    jobs_np, jobs = [], []
    host = []
    for k, (x, y, img, use_w, use_m) in enumerate([
            (90.3, 100.7, 0, True, True), (12.5, 8.5, 0, False, False), (179.4, 199.49, 0, True, False),
            (130.0, 75.0, 1, True, True), (2.2, 148.8, 1, False, True), (31.75, 32.25, 2, True, True),
            (-20.0, 30.0, 2, False, False)]):
        D, W, M = imgs[img]
        D = D.copy()
        X, Y, fx, fy = po.source_pixel(x, y)
        src = po.shifted_psf(P.astype(np.float64), fx, fy) * (500.0 + 100 * k)
        c = K // 2
        for a in range(K):
            for b in range(K):
                r, s = Y - c + a, X - c + b
                if 0 <= r < D.shape[0] and 0 <= s < D.shape[1]:
                    D[r, s] += src[a, b] + (2.0 if flags else 0.0)
        tD, tW, tM, tP = dev(D), dev(W), dev(M), dev(P)
        host.append((tD, tW, tM, tP))
        jobs.append(dict(image=tD, psf=tP, x=x, y=y, weight=tW if use_w else None, mask=tM if use_m else None))
        jobs_np.append(dict(D=D.astype(np.float64), P=P.astype(np.float64), x=x, y=y,
                            W=W.astype(np.float64) if use_w else None, M=M if use_m else None))
    arr = sfft.phot_jobs(jobs)
    jd = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(DEV)
    res = torch.full((len(jobs), 8), -1.0, dtype=torch.float64, device=DEV)
    sfft.sfft_forced_photometry(jd, len(jobs), K, res, flags)
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    # the last job's footprint lies off the frame: status 1, zeros
    assert r[-1, 5] == 1 and r[-1, 4] == 0 and r[-1, 0] == 0
    _phot_compare(jobs_np[:-1], K, flags, r[:-1])


@pytest.mark.slow
def test_forced_photometry_many_stars_full_size():
    """2000 positions on a 4088^2 difference-like frame (field stars of step 8 plus the
    transient of step 9), 60 of them checked against the oracle."""
    rng = np.random.default_rng(11)
    D = rng.normal(0, 3.0, (4088, 4088)).astype(np.float32)
    P = moffat_stamp(31, 2.2, 12)
    xs, ys = rng.uniform(-10, 4098, 2000), rng.uniform(-10, 4098, 2000)
    tD, tP = dev(D), dev(P)
    arr = sfft.phot_jobs([dict(image=tD, psf=tP, x=x, y=y) for x, y in zip(xs, ys)])
    jd = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(DEV)
    res = torch.empty((2000, 8), dtype=torch.float64, device=DEV)
    sfft.sfft_forced_photometry(jd, 2000, 31, res, sfft.PHOT_BACKGROUND)
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    pick = rng.choice(2000, 60, replace=False)
    ok = [i for i in pick if r[i, 5] == 0]
    assert len(ok) > 45
    _phot_compare([dict(D=D, P=P.astype(np.float64), x=xs[i], y=ys[i]) for i in ok], 31, sfft.PHOT_BACKGROUND,
                  r[ok])


def test_edge_cases_of_the_pipeline_steps():
    """Zero photometry jobs (a no-op), the largest stamps (K = 63) for photometry and PSF
    alignment against the oracle, and empty frames rejected by the resampler."""
    res = torch.full((1, 8), -1.0, dtype=torch.float64, device=DEV)
    sfft.sfft_forced_photometry(None, 0, 25, res)
    torch.cuda.synchronize()
    assert float(res[0, 0]) == -1.0
    K = 63
    P = moffat_stamp(K, 6.0, 21)
    rng = np.random.default_rng(22)
    D = rng.normal(0, 1.0, (150, 170)).astype(np.float32)
    x, y = 84.3, 70.6
    X, Y, fx, fy = po.source_pixel(x, y)
    D[Y - 31:Y + 32, X - 31:X + 32] += 900.0 * po.shifted_psf(P.astype(np.float64), fx, fy).astype(np.float32)
    tD, tP = dev(D), dev(P)
    arr = sfft.phot_jobs([dict(image=tD, psf=tP, x=x, y=y)])
    jd = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(DEV)
    sfft.sfft_forced_photometry(jd, 1, K, res, sfft.PHOT_BACKGROUND)
    torch.cuda.synchronize()
    f, sf, b, chi2, n = po.forced_photometry(D.astype(np.float64), P.astype(np.float64), x, y, None, None, True)
    r = res.cpu().numpy()[0]
    assert r[5] == 0 and r[4] == n == K * K
    assert abs(r[0] - f) <= 1e-5 * abs(f) and abs(r[2] - b) <= 1e-5 * (abs(b) + sf)
    w = rot_warp(-0.7, 0.95, 0, 0, 0, 0)
    out = torch.empty((K, K), dtype=torch.float32, device=DEV)
    sfft.sfft_align_psf(w, 10.0, 20.0, tP, out)
    torch.cuda.synchronize()
    ref = po.align_psf(P.astype(np.float64), warp_dict(w), 10.0, 20.0)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    a = torch.zeros((16, 16), device=DEV)
    b2 = torch.zeros((16, 16), device=DEV)
    for shapes in (dict(in_shape=(0, 16)), dict(out_shape=(16, 0))):
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_resample(rot_warp(0.1, 1.0, 0, 0, 0, 0), a, b2, **shapes)
        assert ei.value.status == sfft.ERR_INVALID_ARG
