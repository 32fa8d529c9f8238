"""Cross-convolution (pipeline step 5) through the C ABI against the FP64 oracle.

sfft_cross_convolve computes sci (x) psf_tmpl and tmpl (x) psf_sci (cyclic, K x K stamps) in
FP32 arithmetic.  Tolerance: max |out_gpu - out_ref| <= 1e-5 max |out_ref| (the difference-
image scale the fit is held to), with the FP32 sums of K^2 products well inside it.  Sizes
cross several 256 x 32 output tiles with ragged tails, frames narrower than the stamp, every
stamp radius class, both dtypes and a pitched frame; the full-size case (4088^2, K = 25, the
Roman-like stamps) is checked on sampled pixels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    sfft_build.build()
    sfft.load_library()


def _stamp(K, fwhm, seed):
    """A unit-sum Moffat stamp of odd size K with a random sub-pixel centre (test data)."""
    rng = np.random.default_rng(seed)
    off = np.arange(K) - K // 2
    dy, dx = np.meshgrid(off, off, indexing="ij")
    cy, cx = rng.uniform(-0.5, 0.5, 2)
    al = synth.moffat_alpha(fwhm)
    p = (1.0 + ((dx - cx) ** 2 + (dy - cy) ** 2) / al ** 2) ** (-synth.MOFFAT_BETA)
    return (p / p.sum()).astype(np.float32)


def _run(S, T, Ps, Pt, pitch_pad=0):
    ny, nx = S.shape
    dt = sfft.F64 if S.dtype == np.float64 else sfft.F32
    pitch = nx + pitch_pad if pitch_pad else 0

    def dev(a):
        if pitch_pad:
            b = np.zeros((ny, nx + pitch_pad), a.dtype)
            b[:, :nx] = a
            a = b
        return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)

    St, Tt = dev(S), dev(T)
    So, To = torch.empty_like(St), torch.empty_like(Tt)
    sfft.sfft_cross_convolve(ny, nx, Ps.shape[0], St, Tt, torch.from_numpy(Ps).to(DEV), torch.from_numpy(Pt).to(DEV),
                             So, To, dtype=dt, pitch=pitch)
    torch.cuda.synchronize()
    return So.cpu().numpy()[:, :nx].astype(np.float64), To.cpu().numpy()[:, :nx].astype(np.float64)


CASES = [
    # ny, nx, K, dtype, pitch padding
    (300, 280, 25, np.float32, 0),   # two tile columns, ragged rows (300 = 9 * 32 + 12)
    (77, 530, 7, np.float32, 0),     # three tile columns, ragged
    (64, 64, 31, np.float64, 0),     # largest stamp, float64 frames
    (20, 13, 15, np.float32, 0),     # frame narrower than the stamp: the window wraps twice
    (129, 257, 1, np.float32, 0),    # K = 1: a scaling
    (100, 200, 11, np.float32, 24),  # pitched frame
]


@pytest.mark.parametrize("ny,nx,K,dtype,pad", CASES)
def test_cross_convolution_matches_oracle(ny, nx, K, dtype, pad):
    S, T, _ = synth.roman_pair(ny, nx, seed=ny + nx + K, n_stars=max(5, ny * nx // 300))
    S, T = S.astype(dtype), T.astype(dtype)
    Ps, Pt = _stamp(K, 1.9, 1), _stamp(K, 2.3, 2)
    So, To = _run(S, T, Ps, Pt, pad)
    So_ref, To_ref = oracle.convolve(S, Pt), oracle.convolve(T, Ps)
    for got, ref in ((So, So_ref), (To, To_ref)):
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print("cross-convolution %dx%d K=%d: max err / max|out| = %.3e" % (ny, nx, K, err))
        assert err <= 1e-5


def test_cross_convolution_one_half_and_argument_errors():
    S, T, _ = synth.roman_pair(64, 96, seed=5, n_stars=20)
    Ps, Pt = _stamp(9, 2.0, 3), _stamp(9, 2.2, 4)
    St, Tt = torch.from_numpy(S).to(DEV), torch.from_numpy(T).to(DEV)
    So = torch.full_like(St, 7.0)
    sfft.sfft_cross_convolve(64, 96, 9, St, None, None, torch.from_numpy(Pt).to(DEV), So, None)
    torch.cuda.synchronize()
    ref = oracle.convolve(S, Pt)
    assert np.abs(So.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    P8 = torch.zeros((8, 8), dtype=torch.float32, device=DEV)
    for kw in (dict(K=8), dict(K=33), dict(ny=0)):
        args = dict(ny=64, nx=96, K=9)
        args.update(kw)
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_cross_convolve(args["ny"], args["nx"], args["K"], St, Tt, P8, P8, So, torch.empty_like(Tt))
        assert ei.value.status == sfft.ERR_INVALID_ARG
    with pytest.raises(sfft.SfftError):
        sfft.sfft_cross_convolve(64, 96, 9, St, Tt, P8, P8, St, torch.empty_like(Tt))  # output aliases input


@pytest.mark.slow
def test_cross_convolution_full_size_sampled():
    """4088^2 Roman-like pair with 25 x 25 stamps (the frames' star radius), checked at
    sampled pixels including the four corners where the window wraps."""
    S, T, _ = synth.roman_pair(4088, 4088, seed=1000)
    Ps, Pt = _stamp(25, 2.1, 5), _stamp(25, 2.1, 6)
    So, To = _run(S, T, Ps, Pt)
    rng = np.random.default_rng(2)
    ys = np.concatenate([rng.integers(0, 4088, 200), [0, 0, 4087, 4087]])
    xs = np.concatenate([rng.integers(0, 4088, 200), [0, 4087, 0, 4087]])
    r = 12
    for got, X, P in ((So, S, Pt), (To, T, Ps)):
        # the oracle on a (4r + 1)^2 cyclic cutout centred on the pixel: its centre output
        # reads inputs within r of the centre only, so the cutout's own wrap never enters
        ref = []
        for y, x in zip(ys, xs):
            iy = (np.arange(-2 * r, 2 * r + 1) + y) % 4088
            ix = (np.arange(-2 * r, 2 * r + 1) + x) % 4088
            ref.append(oracle.convolve(X[np.ix_(iy, ix)], P)[2 * r, 2 * r])
        ref = np.array(ref)
        assert np.abs(got[ys, xs] - ref).max() <= 1e-5 * np.abs(got).max()
