"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Sizes are chosen so the oracle finishes in seconds yet the GPU path crosses several row
segments (P = 256, U = P - 2(L-1) useful columns each), ragged segment and y-tile tails,
frames narrower than one segment window, L = 1, and both input dtypes.

Tolerances:
  * difference image: max |D_gpu - D_ref| <= 1e-5 max |T| (the stated target) for the FP32
    path, 1e-10 max |T| (plus the output's own rounding) for the FP64 path;
  * coefficients, ||theta_gpu - theta_ref|| / ||theta_ref||: 1e-10 for the FP64 path; for the
    FP32 path 1e-6, the stated target.  The first FP32 solve carries the rounding of the
    FP32 segment spectra (1e-6 .. 4e-5 on these densely starred frames); the refinement
    pass removes it as long as its residual image is accurate to well below u |S| at the
    star cores, which the compensated residual kernel provides (exact products and a
    two-sum accumulator).  What remains is the FP32 rounding of the operands (the folded
    coefficients and xh^p T_m) and of the residual spectra: ~1e-7, amplified on small frames
    with few pixels per unknown.
  * normal-matrix entries (a diagnostic of the assembly, scaled by the diagonal):
    |N_gpu - N_ref|_ij <= tol sqrt(N_ii N_jj) with tol = 5e-7 for the FP32 path (random
    rounding of the FP32 segment FFTs, ~ u sqrt(log2 P) per spectral value, averaged by the
    lag sums; the systematic twiddle bias is removed by split twiddles), 1e-12 for FP64.
    The kernel x background block gets 2e-6: the background images m xh^p yh^q are smooth,
    so their spectra sit in a few large low-frequency bins whose FP32 rounding does not
    average out over the lag sums, and the more so the higher the degree (measured 2.8e-7
    at DB = 2, 7.8e-7 at DB = 4, with the coefficients still within 3e-7).
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


def _to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_normal(S, T, M, L, dk, db, precision=sfft.PREC_SPLIT):
    ny, nx = S.shape
    dtype = sfft.F64 if S.dtype == np.float64 else sfft.F32
    with sfft.sfft_plan(sfft.make_desc(ny, nx, L, dk, db, dtype=dtype, precision=precision)) as plan:
        n = plan.n
        N = torch.empty((n, n), dtype=torch.float64, device=DEV)
        b = torch.empty(n, dtype=torch.float64, device=DEV)
        St, Tt, Mt = _to_dev(S), _to_dev(T), _to_dev(M)
        sfft.sfft_normal(plan, St, Tt, Mt, N, b)
        torch.cuda.synchronize()
    return N.cpu().numpy(), b.cpu().numpy()


def gpu_fit_subtract(S, T, M, L, dk, db, precision=sfft.PREC_SPLIT, solver=sfft.SOLVE_CHOLESKY, x0=None,
                     refine=0):
    ny, nx = S.shape
    dtype = sfft.F64 if S.dtype == np.float64 else sfft.F32
    desc = sfft.make_desc(ny, nx, L, dk, db, dtype=dtype, precision=precision, solver=solver, refine=refine)
    with sfft.sfft_plan(desc) as plan:
        St, Tt, Mt = _to_dev(S), _to_dev(T), _to_dev(M)
        theta = torch.empty(plan.n, dtype=torch.float64, device=DEV)
        D = torch.empty_like(St)
        info = sfft.sfft_fit(plan, St, Tt, Mt, _to_dev(x0), theta, want_info=True)
        sfft.sfft_subtract(plan, St, Tt, theta, D)
        torch.cuda.synchronize()
    return theta.cpu().numpy(), D.cpu().numpy().astype(np.float64), info


def scaled_err(A, B):
    d = np.sqrt(np.abs(np.diag(B)))
    return np.max(np.abs(A - B) / np.outer(d, d))


def rhs_err(a, b, N):
    """|b_gpu - b_ref| relative to sqrt(N_ii) * ||S_m||, the Cauchy-Schwarz bound of b_i."""
    return np.max(np.abs(a - b) / np.sqrt(np.abs(np.diag(N))))


CASES = [
    # ny,  nx,   L, dk, db, masked, dtype
    (300, 280, 5, 2, 2, True, np.float32),    # 2 segments, ragged y tile (300 = 4*64 + 44)
    (130, 700, 11, 2, 2, True, np.float32),   # 3 segments, the config-1 basis (n = 732)
    (64, 64, 5, 0, 0, False, np.float64),     # small float64 shape
    (77, 51, 3, 1, 3, True, np.float32),      # frame narrower than one window: wraps several times
    (40, 500, 1, 0, 0, True, np.float32),     # L = 1, 3 segments
    (96, 244, 7, 3, 1, True, np.float32),     # nx == U for L = 7: exactly one segment
    (66, 300, 15, 1, 0, False, np.float32),   # largest supported L
    (128, 200, 5, 1, 4, True, np.float32),    # largest background degree, odd nP(DK)
]


def _inputs(ny, nx, masked, dtype, seed):
    S, T, M = synth.roman_pair(ny, nx, seed=seed, n_stars=max(8, ny * nx // 400))
    if not masked:
        M = None
    return S.astype(dtype), T.astype(dtype), M


@pytest.mark.parametrize("ny,nx,L,dk,db,masked,dtype", CASES)
def test_normal_equations_match_oracle(ny, nx, L, dk, db, masked, dtype):
    S, T, M = _inputs(ny, nx, masked, dtype, seed=ny + nx)
    N_ref, b_ref = oracle.normal_equations(S, T, M, L, dk, db)
    N, b = gpu_normal(S, T, M, L, dk, db)
    e_n, e_b = scaled_err(N, N_ref), rhs_err(b, b_ref, N_ref) / np.sqrt(np.sum((S.astype(np.float64) * (1 - (M if M is not None else 0))) ** 2))
    nker = L * L * (dk + 1) * (dk + 2) // 2
    d = np.sqrt(np.abs(np.diag(N_ref)))
    E = np.abs(N - N_ref) / np.outer(d, d)
    e_kk, e_kb, e_bb = E[:nker, :nker].max(), E[:nker, nker:].max(), E[nker:, nker:].max()
    print("N scaled err %.3e (kernel x kernel %.3e, kernel x background %.3e, background %.3e)  b err %.3e" % (
        e_n, e_kk, e_kb, e_bb, e_b))
    assert e_kk <= 5e-7 and e_bb <= 5e-7
    assert e_kb <= 2e-6
    assert e_b <= 5e-7
    assert np.array_equal(N, N.T)


@pytest.mark.parametrize("ny,nx,L,dk,db,masked,dtype", CASES)
def test_fit_and_difference_match_oracle(ny, nx, L, dk, db, masked, dtype):
    S, T, M = _inputs(ny, nx, masked, dtype, seed=ny * 3 + nx)
    th_ref = oracle.fit(S, T, M, L, dk, db)
    D_ref = oracle.subtract(S, T, th_ref, L, dk, db)
    th, D, info = gpu_fit_subtract(S, T, M, L, dk, db)
    rel = np.linalg.norm(th - th_ref) / np.linalg.norm(th_ref)
    derr = np.abs(D - D_ref).max() / np.abs(T).max()
    print("theta rel %.3e  D err %.3e  residual %.3e" % (rel, derr, info.rel_residual))
    assert info.status == 0
    assert rel <= 1e-6
    assert derr <= 1e-5


@pytest.mark.parametrize("ny,nx,L,dk,db,masked,dtype", [CASES[0], CASES[2], CASES[3]])
def test_fp64_path_matches_oracle_tightly(ny, nx, L, dk, db, masked, dtype):
    S, T, M = _inputs(ny, nx, masked, dtype, seed=5 * ny + nx)
    N_ref, b_ref = oracle.normal_equations(S, T, M, L, dk, db)
    N, b = gpu_normal(S, T, M, L, dk, db, precision=sfft.PREC_FP64)
    assert scaled_err(N, N_ref) <= 1e-12
    th_ref = oracle.cholesky_solve(N_ref, b_ref)
    th, D, _ = gpu_fit_subtract(S, T, M, L, dk, db, precision=sfft.PREC_FP64)
    assert np.linalg.norm(th - th_ref) <= 1e-10 * np.linalg.norm(th_ref)
    D_ref = oracle.subtract(S, T, th_ref, L, dk, db)
    # float32 frames carry a float32 difference image: allow its output rounding
    out_ulp = np.finfo(dtype).eps * np.abs(D_ref).max()
    assert np.abs(D - D_ref).max() <= 1e-10 * np.abs(T).max() + out_ulp


def test_small_float64_pair_workload():
    """64 x 64 float64 pair, fixed 5 x 5 kernel, L=5, DK=0, DB=0 (26 unknowns), FP64 path.
    The template keeps its sky of 100, so the constant background and the kernel sum are
    nearly collinear (cond(N) ~ 4e6): this workload needs the FP64 arithmetic mode."""
    S, T, k, bg = synth.gaussian_pair(seed=0)
    th_ref = oracle.fit(S, T, None, 5, 0, 0)
    th, D, info = gpu_fit_subtract(S, T, None, 5, 0, 0, precision=sfft.PREC_FP64)
    assert info.n == 26
    assert np.linalg.norm(th - th_ref) <= 1e-8 * np.linalg.norm(th_ref)
    D_ref = oracle.subtract(S, T, th_ref, 5, 0, 0)
    assert np.abs(D - D_ref).max() <= 1e-9 * np.abs(T).max()


def test_exact_recovery_through_gpu():
    """Noise-free science built from known coefficients (cyclic model, no mask)."""
    ny, nx, L, dk, db = 128, 300, 5, 1, 1
    rng = np.random.default_rng(4)
    T = (rng.gamma(2.0, 20.0, (ny, nx))).astype(np.float64)
    a = rng.normal(0, 0.3, (3, L * L))
    bc = np.array([2.0, -1.0, 0.5])
    xh = 2.0 * np.arange(nx) / (nx - 1) - 1.0
    yh = 2.0 * np.arange(ny) / (ny - 1) - 1.0
    mons = [np.ones((ny, nx)), np.outer(np.ones(ny), xh), np.outer(yh, np.ones(nx))]
    S = np.zeros_like(T)
    h = L // 2
    for i in range(3):
        for li in range(L * L):
            S += a[i, li] * np.roll(mons[i] * T, shift=(li // L - h, li % L - h), axis=(0, 1))
    for r in range(3):
        S += bc[r] * mons[r]
    th, D, info = gpu_fit_subtract(S, T, None, L, dk, db, precision=sfft.PREC_FP64)
    truth = np.concatenate([a.ravel(), bc])
    assert np.linalg.norm(th - truth) <= 1e-9 * np.linalg.norm(truth)
    assert np.abs(D).max() <= 1e-9 * np.abs(S).max()
    th32, D32, _ = gpu_fit_subtract(S, T, None, L, dk, db)
    # the template's mean of ~40 makes the constant background nearly collinear with the
    # kernel sum; the FP32 path stays within 1e-6 of the truth after refinement
    assert np.linalg.norm(th32 - truth) <= 1e-6 * np.linalg.norm(truth)


def test_mask_none_equals_all_good_mask():
    S, T, _ = _inputs(100, 260, False, np.float32, seed=3)
    M0 = np.zeros(S.shape, np.uint8)
    N1, b1 = gpu_normal(S, T, None, 5, 1, 1)
    N2, b2 = gpu_normal(S, T, M0, 5, 1, 1)
    assert np.array_equal(N1, N2) and np.array_equal(b1, b2)


def test_singular_design_reports_not_spd():
    S, T, _ = _inputs(64, 64, False, np.float32, seed=1)
    T = np.zeros_like(T)
    with pytest.raises(sfft.SfftError) as ei:
        gpu_fit_subtract(S, T, None, 3, 0, 0)
    assert ei.value.status == sfft.ERR_NOT_SPD


def test_invalid_descriptor_rejected():
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_plan(sfft.make_desc(64, 64, 4, 0, 0))
    assert ei.value.status == sfft.ERR_INVALID_ARG


def test_repeated_calls_are_deterministic():
    S, T, M = _inputs(150, 300, True, np.float32, seed=9)
    th1, D1, _ = gpu_fit_subtract(S, T, M, 5, 2, 1)
    th2, D2, _ = gpu_fit_subtract(S, T, M, 5, 2, 1)
    assert np.array_equal(th1, th2) and np.array_equal(D1, D2)


@pytest.mark.parametrize("ny,nx,L,dk,db", [(300, 280, 5, 2, 2), (512, 512, 11, 2, 2), (200, 260, 7, 1, 0)])
def test_pcg_matches_cholesky(ny, nx, L, dk, db):
    """The cluster PCG (FP32 Cholesky preconditioner, FP64 residuals) reaches the FP64
    Cholesky solution of the same normal equations without falling back."""
    S, T, M = _inputs(ny, nx, True, np.float32, seed=ny + 2 * nx)
    thc, _, ic = gpu_fit_subtract(S, T, M, L, dk, db, refine=-1)
    thp, _, ip = gpu_fit_subtract(S, T, M, L, dk, db, solver=sfft.SOLVE_PCG, refine=-1)
    assert ip.fallback == 0 and 1 <= ip.iterations <= 10
    assert np.linalg.norm(thp - thc) <= 1e-9 * np.linalg.norm(thc)
    assert ip.rel_residual <= 1e-12


def test_pcg_warm_start_and_refinement():
    S, T, M = _inputs(256, 300, True, np.float32, seed=77)
    th_ref = oracle.fit(S, T, M, 5, 2, 1)
    th0, _, i0 = gpu_fit_subtract(S, T, M, 5, 2, 1, solver=sfft.SOLVE_PCG, refine=-1)
    # a warm start 1e-3 away from the answer needs no more iterations than a cold start
    x0 = th0 * (1.0 + 1e-3 * np.random.default_rng(1).normal(size=th0.shape))
    thw, _, iw = gpu_fit_subtract(S, T, M, 5, 2, 1, solver=sfft.SOLVE_PCG, x0=x0, refine=-1)
    assert iw.fallback == 0 and iw.iterations <= i0.iterations
    assert np.linalg.norm(thw - th0) <= 1e-9 * np.linalg.norm(th0)
    # with the default residual refinement the PCG path meets the FP32-path tolerance
    thr, Dr, _ = gpu_fit_subtract(S, T, M, 5, 2, 1, solver=sfft.SOLVE_PCG)
    assert np.linalg.norm(thr - th_ref) <= 1e-6 * np.linalg.norm(th_ref)


def test_pcg_singular_design_falls_back_and_reports():
    S, T, _ = _inputs(64, 64, False, np.float32, seed=1)
    with pytest.raises(sfft.SfftError) as ei:
        gpu_fit_subtract(S, np.zeros_like(T), None, 3, 0, 0, solver=sfft.SOLVE_PCG)
    assert ei.value.status == sfft.ERR_NOT_SPD


@pytest.mark.parametrize("ny,nx,L,dk,db,masked,dtype", [CASES[0], CASES[1]])
def test_fp32_mode_without_refinement(ny, nx, L, dk, db, masked, dtype):
    """SFFT_PREC_FP32 runs the same kernels as SFFT_PREC_SPLIT but skips the refinement pass:
    its coefficients carry the FP32 spectra's rounding (amplified by cond(N)), so the bound is
    looser, while the difference image still meets 1e-5 of the template scale."""
    S, T, M = _inputs(ny, nx, masked, dtype, seed=7 * ny + nx)
    th_ref = oracle.fit(S, T, M, L, dk, db)
    th, D, info = gpu_fit_subtract(S, T, M, L, dk, db, precision=sfft.PREC_FP32)
    D_ref = oracle.subtract(S, T, th_ref, L, dk, db)
    assert info.status == 0
    assert np.linalg.norm(th - th_ref) <= 1e-4 * np.linalg.norm(th_ref)
    assert np.abs(D - D_ref).max() <= 1e-5 * np.abs(T).max()


@pytest.mark.parametrize("precision", [sfft.PREC_SPLIT, sfft.PREC_FP64])
def test_masked_pixels_never_enter_the_fit_whatever_they_hold(precision):
    """NaN or Inf at masked pixels of S and T leaves the coefficients unchanged (bit for bit)
    against zeros there: masked pixels are selected out, not multiplied by zero."""
    S, T, M = _inputs(200, 230, True, np.float32, seed=21)
    Sz, Tz = S.copy(), T.copy()
    Sz[M == 1] = 0
    Tz[M == 1] = 0
    Sn, Tn = S.copy(), T.copy()
    ys, xs = np.nonzero(M)
    Sn[ys[::2], xs[::2]] = np.nan
    Tn[ys[1::2], xs[1::2]] = np.inf
    th_z, _, iz = gpu_fit_subtract(Sz, Tz, M, 5, 2, 1, precision=precision)
    th_n, _, inn = gpu_fit_subtract(Sn, Tn, M, 5, 2, 1, precision=precision)
    assert iz.status == 0 and inn.status == 0
    assert np.array_equal(th_z, th_n)
