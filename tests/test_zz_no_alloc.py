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


def _frames(ny, nx, pitch, dtype, seed):
    """Seeded frames laid out with a row pitch of `pitch` elements (the padding columns hold
    values that must never be read as pixels)."""
    S, T, M = synth.roman_pair(ny, nx, seed=seed)
    out = []
    for a, fill in ((S, 1e30), (T, -1e30), (M, 1)):
        buf = np.full((ny, pitch), fill, dtype=a.dtype if a.dtype == np.uint8 else dtype)
        buf[:, :nx] = a
        out.append(torch.from_numpy(buf).to(DEV))
    return out, float(np.abs(T).max())


# (input dtype, precision, row pitch minus width): the FP32 path with SPLIT precision, the FP64
# path (FP64 scratch tables), and a pitched FP32 frame
VARIANTS = [(sfft.F32, sfft.PREC_SPLIT, 0), (sfft.F64, sfft.PREC_FP64, 0), (sfft.F32, sfft.PREC_SPLIT, 20)]


@pytest.mark.parametrize("dtype,precision,pad", VARIANTS)
def test_noalloc_matches_planned_subtract_on_two_calls(dtype, precision, pad):
    ny, nx, L, dk, db = 300, 280, 5, 2, 2
    npdt = np.float64 if dtype == sfft.F64 else np.float32
    (St, Tt, Mt), tmax = _frames(ny, nx, nx + pad, npdt, seed=31)
    desc = sfft.make_desc(ny, nx, L, dk, db, dtype=dtype, precision=precision, pitch=nx + pad if pad else 0)
    theta, D_ref = _planned(desc, St, Tt, Mt)
    # FP32 images: the stated 1e-5 of the template's flux scale; FP64: the FP64 path's bound
    tol = (1e-5 if dtype == sfft.F32 else 1e-10) * tmax
    theta2 = theta * 1.01
    with sfft.sfft_plan(desc) as plan:
        D2_ref = torch.empty_like(St)
        sfft.sfft_subtract(plan, St, Tt, theta2, D2_ref)
        torch.cuda.synchronize()
    D1, D2, D3 = (torch.empty_like(St) for _ in range(3))
    # the first call (per-device set-up, kernels loaded) ...
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta, D1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    # ... then two more in a row, with other coefficients and then the first ones again: the
    # shared array carries nothing over, and the device's free memory does not move
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta2, D2)
    sfft.sfft_subtract_noalloc(desc, St, Tt, theta, D3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0
    for got, ref in ((D1, D_ref), (D2, D2_ref), (D3, D_ref)):
        assert float((got[:, :nx] - ref[:, :nx]).abs().max()) <= tol


def test_noalloc_rejects_frames_beyond_its_scratch():
    desc = sfft.make_desc(8192, 8192, 15, 3, 2)  # needs ~30 MB of scratch
    x = torch.zeros(16, dtype=torch.float32, device=DEV)
    th = torch.zeros(16, dtype=torch.float64, device=DEV)
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_subtract_noalloc(desc, x, x, th, torch.zeros_like(x))
    assert ei.value.status == sfft.ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
