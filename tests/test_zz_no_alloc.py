"""The allocation-free difference-image entry point (sfft_subtract_noalloc) against the
planned one (sfft_subtract).

Callers that cannot allocate device memory where they need the difference image -- their
memory belongs to another allocator, or their path cannot take cudaMalloc's implicit
synchronisation -- use the no-allocation variant, whose scratch is a fixed device array.
This file is named so that pytest collects it last; it must pass alone in a fresh process
(the first call performs the per-device set-up) and after every other test.
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


def _planned(desc, St, Tt, Mt):
    with sfft.sfft_plan(desc) as plan:
        theta = torch.empty(plan.n, dtype=torch.float64, device=DEV)
        sfft.sfft_fit(plan, St, Tt, Mt, None, theta, want_info=True)
        D = torch.empty_like(St)
        sfft.sfft_subtract(plan, St, Tt, theta, D)
        torch.cuda.synchronize()
    return theta, D


def test_noalloc_matches_planned_subtract_on_two_calls():
    ny, nx, L, dk, db = 300, 280, 5, 2, 2
    S, T, M = synth.roman_pair(ny, nx, seed=31)
    St, Tt, Mt = (torch.from_numpy(a).to(DEV) for a in (S, T, M))
    desc = sfft.make_desc(ny, nx, L, dk, db)
    theta, D_ref = _planned(desc, St, Tt, Mt)
    tol = 1e-5 * float(np.abs(T).max())
    # first call (per-device set-up happens here), then a second call with other
    # coefficients, then the first coefficients again: the shared array carries nothing over
    theta2 = theta * 1.01
    D1 = torch.empty_like(St)
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta, D1)
    D2 = torch.empty_like(St)
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta2, D2)
    D3 = torch.empty_like(St)
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta, D3)
    torch.cuda.synchronize()
    with sfft.sfft_plan(desc) as plan:
        D2_ref = torch.empty_like(St)
        sfft.sfft_subtract(plan, St, Tt, theta2, D2_ref)
        torch.cuda.synchronize()
    assert float((D1 - D_ref).abs().max()) <= tol
    assert float((D2 - D2_ref).abs().max()) <= tol
    assert float((D3 - D_ref).abs().max()) <= tol


def test_noalloc_rejects_frames_beyond_its_scratch():
    desc = sfft.make_desc(8192, 8192, 15, 3, 2)  # needs ~30 MB of scratch
    x = torch.zeros(16, dtype=torch.float32, device=DEV)
    th = torch.zeros(16, dtype=torch.float64, device=DEV)
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_subtract_noalloc(desc, x, x, th, torch.zeros_like(x))
    assert ei.value.status == sfft.ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
