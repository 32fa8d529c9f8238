"""Parity at the full 4088 x 4088 size, in the configuration the benchmark times.

The benchmark's first pair (Roman-like 4088^2 float32 frames, 0.5% masked, L = 11, DK = 2,
DB = 2, n = 732, FP32 spectra, default refinement) goes through the C ABI and is compared
with the FP64 oracle:
  * sampled normal-matrix entries and right-hand-side values, each evaluated by definition
    (direct spatial sums over the full frame), scaled as in the small-frame tests;
  * the coefficients against the oracle's full fit (lag tables by direct sums, FP64
    Cholesky): ||theta_gpu - theta_ref|| / ||theta_ref|| <= 1e-6, for the Cholesky and the
    PCG solvers;
  * difference-image pixels at sampled positions, including the frame edges where the
    cyclic window wraps, for the GPU's own coefficients: <= 1e-5 max |T|.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = torch.device("cuda:0")
NY = NX = 4088
L, DK, DB = 11, 2, 2


@pytest.fixture(scope="module")
def pair():
    sfft_build.build()
    sfft.load_library()
    S, T, M = synth.roman_pair(NY, NX, seed=1000)   # the benchmark's first pair on rank 0
    return S, T, M


@pytest.fixture(scope="module")
def theta_ref(pair):
    S, T, M = pair
    return oracle.fit(S, T, M, L, DK, DB)


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _fit(pair, solver):
    S, T, M = pair
    with sfft.sfft_plan(sfft.make_desc(NY, NX, L, DK, DB, solver=solver)) as p:
        St, Tt, Mt = _dev(S), _dev(T), _dev(M)
        th = torch.empty(p.n, dtype=torch.float64, device=DEV)
        D = torch.empty_like(St)
        info = sfft.sfft_fit(p, St, Tt, Mt, None, th, want_info=True)
        sfft.sfft_subtract(p, St, Tt, th, D)
        torch.cuda.synchronize()
        return th.cpu().numpy(), D, info


def test_sampled_normal_entries(pair):
    S, T, M = pair
    n = oracle.n_unknowns(L, DK, DB)
    with sfft.sfft_plan(sfft.make_desc(NY, NX, L, DK, DB)) as p:
        N = torch.empty((n, n), dtype=torch.float64, device=DEV)
        b = torch.empty(n, dtype=torch.float64, device=DEV)
        sfft.sfft_normal(p, _dev(S), _dev(T), _dev(M), N, b)
        torch.cuda.synchronize()
        N, b = N.cpu().numpy(), b.cpu().numpy()
    rng = np.random.default_rng(7)
    rows = rng.integers(0, n, 48)
    cols = rng.integers(0, n, 48)
    # the diagonal, the kernel/background block corner and the last unknown
    rows = np.concatenate([rows, [0, n - 1, 0, n - 7]])
    cols = np.concatenate([cols, [0, n - 1, n - 1, 3]])
    ref = oracle.normal_entries(S, T, M, L, DK, DB, rows, cols)
    diag = oracle.normal_entries(S, T, M, L, DK, DB, np.concatenate([rows, cols]), np.concatenate([rows, cols]))
    dr, dc = diag[:len(rows)], diag[len(rows):]
    err = np.abs(N[rows, cols] - ref) / np.sqrt(dr * dc)
    assert err.max() <= 5e-7, err.max()
    brows = rng.integers(0, n, 24)
    bref = oracle.normal_entries(S, T, M, L, DK, DB, brows, np.full(len(brows), n))
    bdiag = oracle.normal_entries(S, T, M, L, DK, DB, brows, brows)
    Sm = S.astype(np.float64) * (M == 0)
    berr = np.abs(b[brows] - bref) / np.sqrt(bdiag * np.sum(Sm * Sm))
    assert berr.max() <= 5e-7, berr.max()


@pytest.mark.parametrize("solver", [sfft.SOLVE_CHOLESKY, sfft.SOLVE_PCG])
def test_coefficients_and_sampled_pixels(pair, theta_ref, solver):
    S, T, M = pair
    th, D, info = _fit(pair, solver)
    assert info.status == 0
    rel = np.linalg.norm(th - theta_ref) / np.linalg.norm(theta_ref)
    assert rel <= 1e-6, rel
    rng = np.random.default_rng(11)
    ys = np.concatenate([rng.integers(0, NY, 400), [0, 0, NY - 1, NY - 1, 3, NY - 4]])
    xs = np.concatenate([rng.integers(0, NX, 400), [0, NX - 1, 0, NX - 1, NX - 2, 1]])
    flat = ys * NX + xs
    ref = oracle.subtract_pixels(S, T, th, L, DK, DB, flat)
    got = D.reshape(-1)[torch.from_numpy(flat).to(DEV)].cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(T).max()
