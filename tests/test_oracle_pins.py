"""Pins for the FP64 CPU oracle, against things other than the oracle itself.

Each test checks the oracle against something the mathematics fixes: brute-force dot
products of materialised basis images, correlation through numpy's FFT (a library
primitive), exact recovery of data synthesised from the model here in the test, closed
forms (one-parameter least squares, identity and pure-shift kernels, kernel sum = flux
ratio), the textbook polynomial least-squares solution via numpy.linalg.lstsq, and the
symmetric-positive-definite property of N.  A wrong sign or index in the lag direction,
a transposed pair in the assembly, a dropped mask factor or a wrong monomial order fails
at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2509_18544_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frames(ny, nx, seed, masked=True, frac=0.08):
    rng = np.random.default_rng(seed)
    T = rng.normal(0, 1, (ny, nx)) + 3 * rng.random((ny, nx)) ** 4
    S = rng.normal(0, 1, (ny, nx)) + 0.7 * T
    mask = (rng.random((ny, nx)) < frac).astype(np.uint8) if masked else None
    return S, T, mask


def _monomials_by_definition(ny, nx, d):
    """Monomials xh^p yh^q with p+q <= d, total degree first then q ascending (test-side)."""
    xh = 2.0 * np.arange(nx) / (nx - 1) - 1.0
    yh = 2.0 * np.arange(ny) / (ny - 1) - 1.0
    out = []
    for deg in range(d + 1):
        for q in range(deg + 1):
            p = deg - q
            out.append(np.outer(yh ** q, xh ** p))
    return out


def _synthesise(T, a, bcoef, L, dk, db):
    """S(u) = sum a[pq, d] (w_pq T)((u - d) mod N) + sum b_rs w_rs(u), written here with np.roll."""
    ny, nx = T.shape
    h = (L - 1) // 2
    wk = _monomials_by_definition(ny, nx, dk)
    wb = _monomials_by_definition(ny, nx, db)
    S = np.zeros_like(T)
    for i, w in enumerate(wk):
        for li in range(L * L):
            dy, dx = li // L - h, li % L - h
            S += a[i, li] * np.roll(w * T, shift=(dy, dx), axis=(0, 1))
    for r, w in enumerate(wb):
        S += bcoef[r] * w
    return S


def test_monomial_order():
    assert [oracle.mono_pq(i) for i in range(10)] == [
        (0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]
    assert oracle.n_unknowns(11, 2, 2) == 732
    assert oracle.n_unknowns(11, 2, 1) == 729
    assert oracle.n_unknowns(15, 3, 2) == 2256
    assert oracle.n_unknowns(5, 0, 0) == 26


@pytest.mark.parametrize("ny,nx,L,dk,db,masked", [
    (16, 16, 3, 1, 1, True),
    (12, 10, 5, 2, 1, True),
    (9, 11, 3, 0, 2, False),
    (7, 7, 7, 1, 0, True),   # lags reach the frame size: every cyclic wrap is exercised
])
def test_brute_force_equals_lag_structured(ny, nx, L, dk, db, masked):
    S, T, m = _frames(ny, nx, seed=ny * 100 + nx, masked=masked)
    N1, b1 = oracle.normal_equations(S, T, m, L, dk, db)
    N2, b2 = oracle.brute_normal_equations(S, T, m, L, dk, db)
    scale = np.abs(N2).max()
    assert np.abs(N1 - N2).max() <= 1e-13 * scale
    assert np.abs(b1 - b2).max() <= 1e-13 * np.abs(b2).max()
    assert np.array_equal(N1, N1.T)


def test_lag_tables_match_fft_correlation():
    """C_AB(d) = sum_u A(u) B(u + d) equals IFFT(conj(FFT A) FFT B) at lag d (numpy FFT)."""
    ny, nx, L, dk, db = 20, 18, 5, 2, 1
    S, T, m = _frames(ny, nx, seed=7)
    good = 1.0 - m
    wk = [w * T * good for w in _monomials_by_definition(ny, nx, dk)]
    wb = [w * good for w in _monomials_by_definition(ny, nx, db)]
    Sm = S * good
    tab = oracle.lag_tables(S, T, m, L, dk, db)

    def xcorr(A, B):
        return np.real(np.fft.ifft2(np.conj(np.fft.fft2(A)) * np.fft.fft2(B)))

    h, Lw = (L - 1) // 2, 2 * L - 1
    pr = 0
    for i in range(len(wk)):
        for j in range(i, len(wk)):
            c = xcorr(wk[i], wk[j])
            for ly in range(Lw):
                for lx in range(Lw):
                    dy, dx = ly - (L - 1), lx - (L - 1)
                    assert tab["Cww"][pr, ly, lx] == pytest.approx(c[dy % ny, dx % nx], rel=1e-10, abs=1e-9)
            pr += 1
    for i in range(len(wk)):
        cs = xcorr(wk[i], Sm)
        for ly in range(L):
            for lx in range(L):
                dy, dx = ly - h, lx - h
                assert tab["Cws"][i, ly, lx] == pytest.approx(cs[dy % ny, dx % nx], rel=1e-10, abs=1e-9)
                for r in range(len(wb)):
                    cg = xcorr(wk[i], wb[r])
                    assert tab["Cwg"][i, r, ly, lx] == pytest.approx(cg[dy % ny, dx % nx], rel=1e-10, abs=1e-9)
    for r in range(len(wb)):
        assert tab["Ggs"][r] == pytest.approx(np.sum(wb[r] * Sm), rel=1e-12)
        for r2 in range(len(wb)):
            assert tab["Ggg"][r, r2] == pytest.approx(np.sum(wb[r] * wb[r2]), rel=1e-12)


@pytest.mark.parametrize("ny,nx,L,dk,db", [(32, 28, 5, 2, 2), (24, 24, 3, 1, 0), (30, 20, 7, 0, 1)])
def test_exact_recovery_and_zero_difference(ny, nx, L, dk, db):
    """Noise-free S built from known coefficients: the fit returns them and D vanishes."""
    rng = np.random.default_rng(11)
    T = rng.normal(0, 1, (ny, nx)) + 2.0
    nk, nb = oracle.npoly(dk), oracle.npoly(db)
    a = rng.normal(0, 1, (nk, L * L))
    bcoef = rng.normal(0, 1, nb)
    S = _synthesise(T, a, bcoef, L, dk, db)
    theta = oracle.fit(S, T, None, L, dk, db)
    truth = np.concatenate([a.ravel(), bcoef])
    assert np.linalg.norm(theta - truth) <= 1e-9 * np.linalg.norm(truth)
    D = oracle.subtract(S, T, theta, L, dk, db)
    assert np.abs(D).max() <= 1e-9 * np.abs(S).max()


def test_kernel_sum_is_flux_ratio():
    """S = r (T convolved with a unit-sum kernel): DK=0 gives sum(a) = r; with DK=2 the
    constant block sums to r and every spatial block sums to 0."""
    ny = nx = 40
    rng = np.random.default_rng(3)
    T = rng.gamma(2.0, 1.0, (ny, nx))
    k = rng.random((5, 5))
    k /= k.sum()
    r = 1.37
    S = np.zeros_like(T)
    for ly in range(5):
        for lx in range(5):
            S += r * k[ly, lx] * np.roll(T, shift=(ly - 2, lx - 2), axis=(0, 1))
    th0 = oracle.fit(S, T, None, 5, 0, 0)
    assert th0[:25].sum() == pytest.approx(r, rel=1e-11)
    assert np.allclose(th0[:25].reshape(5, 5), r * k, atol=1e-10)
    th2 = oracle.fit(S, T, None, 5, 2, 1)
    blocks = th2[:6 * 25].reshape(6, 25)
    assert blocks[0].sum() == pytest.approx(r, rel=1e-10)
    assert np.abs(blocks[1:].sum(axis=1)).max() < 1e-10


def test_noisy_small_pair_recovers_kernel():
    """The 64 x 64 float64 workload: the fitted 5x5 kernel sums to 1 within the noise."""
    S, T, k, bg = synth.gaussian_pair(seed=0)
    th = oracle.fit(S, T, None, 5, 0, 0)
    assert th[:25].sum() == pytest.approx(1.0, abs=0.02)
    assert np.abs(th[:25].reshape(5, 5) - k).max() < 0.05


def test_normal_matrix_is_spd():
    S, T, m = _frames(24, 22, seed=5)
    N, b = oracle.normal_equations(S, T, m, 5, 2, 2)
    assert np.array_equal(N, N.T)
    ev = np.linalg.eigvalsh(N)
    assert ev.min() > 0.0
    x = oracle.cholesky_solve(N, b)
    assert np.allclose(x, np.linalg.solve(N, b), rtol=1e-8, atol=1e-10)


def test_not_spd_is_reported():
    S, T, _ = _frames(12, 12, seed=9, masked=False)
    with pytest.raises(oracle.OracleError):
        oracle.fit(S, np.zeros_like(T), None, 3, 0, 0)


def test_single_delta_closed_form():
    """L=1, DK=0, DB=0: unknowns (a, b) are the slope and intercept of the regression of
    S_m on T_m over the good pixels (Cramer's rule on the 2 x 2 normal equations)."""
    S, T, m = _frames(17, 13, seed=21)
    g = (1.0 - m).astype(bool)
    t, s_ = T[g], S[g]
    n, st, ss, stt, sts = len(t), t.sum(), s_.sum(), (t * t).sum(), (t * s_).sum()
    det = stt * n - st * st
    th = oracle.fit(S, T, m, 1, 0, 0)
    assert th[0] == pytest.approx((sts * n - st * ss) / det, rel=1e-11)
    assert th[1] == pytest.approx((stt * ss - st * sts) / det, rel=1e-11)


def test_identity_kernel_when_science_equals_template():
    S, T, m = _frames(18, 16, seed=4)
    L, dk, db = 3, 1, 1
    th = oracle.fit(T, T, m, L, dk, db)
    e = np.zeros_like(th)
    e[(L * L) // 2] = 1.0  # a_{00, (0,0)}
    assert np.abs(th - e).max() < 1e-10


def test_pure_shift_kernel():
    _, T, _ = _frames(20, 18, seed=8, masked=False)
    L, dy0, dx0 = 5, -1, 2
    S = np.roll(T, shift=(dy0, dx0), axis=(0, 1))  # S(u) = T(u - d0)
    th = oracle.fit(S, T, None, L, 1, 1)
    e = np.zeros_like(th)
    h = (L - 1) // 2
    e[(dy0 + h) * L + (dx0 + h)] = 1.0
    assert np.abs(th - e).max() < 1e-10


def test_background_block_is_textbook_polynomial_least_squares():
    """The Psi-Psi block of N and the Psi part of b are the normal equations of the plain
    polynomial fit of S_m on the masked monomial design matrix (numpy.linalg.lstsq)."""
    ny, nx, L, dk, db = 21, 19, 3, 1, 3
    S, T, m = _frames(ny, nx, seed=13)
    N, b = oracle.normal_equations(S, T, m, L, dk, db)
    nker = oracle.npoly(dk) * L * L
    Ngg, bg = N[nker:, nker:], b[nker:]
    good = (1.0 - m).ravel()
    X = np.stack([w.ravel() * good for w in _monomials_by_definition(ny, nx, db)], axis=1)
    coef, *_ = np.linalg.lstsq(X, S.ravel() * good, rcond=None)
    assert np.allclose(np.linalg.solve(Ngg, bg), coef, rtol=1e-9, atol=1e-12)


def test_sampled_entries_match_full_matrix():
    S, T, m = _frames(15, 17, seed=2)
    L, dk, db = 5, 2, 2
    N, b = oracle.normal_equations(S, T, m, L, dk, db)
    n = len(b)
    rng = np.random.default_rng(0)
    rows = rng.integers(0, n, 40)
    cols = rng.integers(0, n + 1, 40)
    got = oracle.normal_entries(S, T, m, L, dk, db, rows, cols)
    want = np.where(cols == n, b[rows], N[rows, np.minimum(cols, n - 1)])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_sampled_pixels_match_full_difference():
    S, T, m = _frames(14, 12, seed=6)
    L, dk, db = 3, 1, 1
    th = oracle.fit(S, T, m, L, dk, db)
    D = oracle.subtract(S, T, th, L, dk, db)
    idx = np.array([0, 5, 17, 100, 14 * 12 - 1])
    assert np.allclose(oracle.subtract_pixels(S, T, th, L, dk, db, idx), D.ravel()[idx], rtol=0, atol=1e-13)


def test_golden_hand_worked_example():
    """A 3 x 3 frame worked by hand (tests/golden/hand_3x3.txt)."""
    vals = {}
    with open(os.path.join(GOLDEN, "hand_3x3.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                vals[k.strip()] = np.array([float(t) for t in v.split()])
    T = vals["T"].reshape(3, 3)
    S = vals["S"].reshape(3, 3)
    mask = vals["mask"].reshape(3, 3).astype(np.uint8)
    th = oracle.fit(S, T, mask, 1, 0, 0)
    assert np.allclose(th, vals["theta_L1_DK0_DB0"], rtol=1e-14, atol=0)
    D = oracle.subtract(S, T, th, 1, 0, 0)
    assert np.allclose(D.ravel(), vals["D_L1_DK0_DB0"], rtol=0, atol=1e-13)
    th3 = oracle.fit(S, T, None, 1, 0, 0)
    assert np.allclose(th3, vals["theta_L1_DK0_DB0_nomask"], rtol=1e-14, atol=0)


def test_masked_pixels_never_enter_the_fit_whatever_they_hold():
    # the mask reading: masked pixels of S and T are zero in the fit, so NaN there changes nothing
    S, T = synth.gaussian_pair(seed=3)[:2]
    M = np.zeros(S.shape, np.uint8)
    M[5, 7] = M[20, 31] = M[40, 2] = 1
    Sz, Tz = S.copy(), T.copy()
    Sz[M == 1] = 0.0
    Tz[M == 1] = 0.0
    Sn, Tn = S.copy(), T.copy()
    Sn[5, 7] = np.nan
    Tn[20, 31] = np.nan
    Tn[40, 2] = np.inf
    a = oracle.fit(Sz, Tz, M, 5, 1, 1)
    b = oracle.fit(Sn, Tn, M, 5, 1, 1)
    assert np.array_equal(a, b)
    rows = np.arange(0, 26 * 3 + 3, 7)
    ea = oracle.normal_entries(Sz, Tz, M, 5, 1, 1, rows, rows[::-1])
    eb = oracle.normal_entries(Sn, Tn, M, 5, 1, 1, rows, rows[::-1])
    assert np.array_equal(ea, eb)


def test_band_lag_tables_are_row_restricted_sums():
    """The band routine (used to time the oracle on a full frame in slices): each band's
    table equals the lag sum restricted to the band's rows, written here with numpy rolls,
    and the bands of a partition of the rows add up to the full tables."""
    ny, nx, L, dk, db = 23, 19, 5, 1, 1
    S, T, m = _frames(ny, nx, seed=17)
    good = 1.0 - m
    wk = [w * T * good for w in _monomials_by_definition(ny, nx, dk)]
    bands = [(0, 4), (4, 13), (13, 23)]
    tabs = [oracle.lag_tables_band(S, T, m, L, dk, db, y0, y1) for y0, y1 in bands]
    full = oracle.lag_tables(S, T, m, L, dk, db)
    for k in full:
        tot = sum(t[k] for t in tabs)
        assert np.allclose(tot, full[k], rtol=1e-12, atol=1e-10 * np.abs(full[k]).max())
    # one entry by definition: C_{W_0,W_1}(dx=2, dy=-3) over rows 4..12 only
    y0, y1 = bands[1]
    prod = wk[0] * np.roll(wk[1], shift=(3, -2), axis=(0, 1))  # B((u + d) mod N) at u
    want = prod[y0:y1].sum()
    got = tabs[1]["Cww"][1, -3 + L - 1, 2 + L - 1]
    assert got == pytest.approx(want, rel=1e-12)
    with pytest.raises(oracle.OracleError):
        oracle.lag_tables_band(S, T, m, L, dk, db, 5, 5)


def test_convolution_pins():
    """Cross-convolution oracle: a centred delta is the identity, an off-centre delta is a
    cyclic shift (np.roll), and a random stamp equals numpy's FFT convolution (a library
    primitive) with the stamp placed cyclically around the origin."""
    rng = np.random.default_rng(3)
    X = rng.normal(size=(21, 17))
    K = 5
    P = np.zeros((K, K))
    P[2, 2] = 1.0
    assert np.array_equal(oracle.convolve(X, P), X)
    P = np.zeros((K, K))
    P[0, 3] = 1.0  # d = (-2, +1): out(u) = X(u - d)
    assert np.allclose(oracle.convolve(X, P), np.roll(X, shift=(-2, 1), axis=(0, 1)), rtol=0, atol=1e-15)
    P = rng.normal(size=(7, 7))
    kimg = np.zeros_like(X)
    for a in range(7):
        for b in range(7):
            kimg[(a - 3) % 21, (b - 3) % 17] += P[a, b]
    ref = np.real(np.fft.ifft2(np.fft.fft2(X) * np.fft.fft2(kimg)))
    assert np.allclose(oracle.convolve(X, P), ref, rtol=1e-12, atol=1e-12)
    with pytest.raises(oracle.OracleError):
        oracle.convolve(X, np.ones((4, 4)))
