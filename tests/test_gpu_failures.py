"""Failure paths of the solvers, produced in the allowed forms: a solver that stops at its
iteration cap, and a bounded device-side wait that runs out.  Neither faults or hangs the
GPU: the kernels record a status word and return, and the tests then check that the same
process keeps working.
"""
import numpy as np
import pytest
import torch

from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    sfft_build.build()
    sfft.load_library()


def _pair(ny, nx, seed):
    S, T, M = synth.roman_pair(ny, nx, seed=seed, n_stars=max(8, ny * nx // 400))
    return tuple(torch.from_numpy(a).to(DEV) for a in (S, T, M))


def _fit(desc, S, T, M):
    with sfft.sfft_plan(desc) as plan:
        th = torch.empty(plan.n, dtype=torch.float64, device=DEV)
        info = sfft.sfft_fit(plan, S, T, M, None, th, want_info=True)
        torch.cuda.synchronize()
    return th.cpu().numpy(), info


def test_pcg_iteration_cap_reports_no_convergence_and_falls_back():
    """PCG on a positive-definite N with max_iter = 1 and an unreachable tolerance stops at
    its cap: the fit reports pcg_status = NO_CONVERGENCE and fallback = 1 and returns the
    FP64 Cholesky solution of the same equations (status OK)."""
    ny, nx, L, dk, db = 300, 280, 5, 2, 2
    S, T, M = _pair(ny, nx, seed=41)
    th_c, ic = _fit(sfft.make_desc(ny, nx, L, dk, db, refine=-1), S, T, M)
    th_p, ip = _fit(sfft.make_desc(ny, nx, L, dk, db, solver=sfft.SOLVE_PCG, max_iter=1, tol=1e-30, refine=-1),
                    S, T, M)
    assert ic.status == 0 and ic.pcg_status == 0
    assert ip.status == 0
    assert ip.fallback == 1
    assert ip.pcg_status == sfft.ERR_NO_CONVERGENCE
    assert np.linalg.norm(th_p - th_c) <= 1e-12 * np.linalg.norm(th_c)
    # the same plan shape with the default cap converges without a fallback
    _, ig = _fit(sfft.make_desc(ny, nx, L, dk, db, solver=sfft.SOLVE_PCG, refine=-1), S, T, M)
    assert ig.fallback == 0 and ig.pcg_status == 0


def test_pcg_cap_in_a_batch_is_reported_per_pair():
    ny, nx, L, dk, db = 200, 260, 5, 1, 1
    data = [_pair(ny, nx, seed=50 + k) for k in range(3)]
    n = L * L * 3 + 3
    th = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in data]
    Ds = [torch.empty_like(d[0]) for d in data]
    pairs = [sfft.make_pair(S, T, M, t, D, ny, nx) for (S, T, M), t, D in zip(data, th, Ds)]
    desc = sfft.make_desc(ny, nx, L, dk, db, solver=sfft.SOLVE_PCG, max_iter=1, tol=1e-30)
    with sfft.sfft_batch_create(desc, pairs, lanes=2) as b:
        infos = sfft.sfft_batch_info(b)
    assert all(i.status == 0 and i.fallback == 1 and i.pcg_status == sfft.ERR_NO_CONVERGENCE for i in infos)


def test_grid_barrier_wait_limit_returns_timeout_and_the_context_stays_usable():
    """spin_limit = 1 lets every wait of the cooperative Cholesky's grid barrier give up
    after one ~64 ns sleep.  CTA 0 factors each diagonal tile (tens of microseconds) while the
    other CTAs wait at the barrier, so they give up: the kernel records SFFT_ERR_TIMEOUT and
    every CTA returns; nothing is left waiting.  The next fit in the same process, with the
    default limit, runs normally and gives the usual answer."""
    ny, nx, L, dk, db = 300, 280, 5, 2, 2
    S, T, M = _pair(ny, nx, seed=43)
    th_ok, i_ok = _fit(sfft.make_desc(ny, nx, L, dk, db), S, T, M)
    with pytest.raises(sfft.SfftError) as ei:
        _fit(sfft.make_desc(ny, nx, L, dk, db, spin_limit=1), S, T, M)
    assert ei.value.status == sfft.ERR_TIMEOUT
    torch.cuda.synchronize()  # the device still answers
    th_again, i_again = _fit(sfft.make_desc(ny, nx, L, dk, db), S, T, M)
    assert i_ok.status == 0 and i_again.status == 0
    assert np.array_equal(th_ok, th_again)


def test_negative_spin_limit_is_rejected_on_the_host():
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_plan(sfft.make_desc(64, 64, 3, 0, 0, spin_limit=-1))
    assert ei.value.status == sfft.ERR_INVALID_ARG
