"""The difference image's row-segment FFT route (tuning field subtract_fft = 1) against the
FP64 oracle and against the direct kernel, on the same fitted coefficients.

Tolerance: D within 1e-5 max|T| of the oracle (the difference image's bound); the two GPU
routes differ only by FP32 rounding of different summation orders, within 1e-6 max|T|.
Shapes cross several 256-column segments and 32-row chunks with ragged edges, a frame
narrower than one segment, every DK the route has kernels for, L from 3 to 15, DB up to 4,
FP64 frames and a pitched frame."""
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


CASES = [
    # ny, nx, L, dk, db, dtype, pitch pad
    (300, 600, 11, 2, 2, np.float32, 0),
    (97, 180, 5, 1, 1, np.float32, 0),   # narrower than one segment
    (260, 530, 15, 0, 4, np.float64, 0),
    (130, 300, 3, 2, 0, np.float32, 12),  # pitched
]


@pytest.mark.parametrize("ny,nx,L,dk,db,dt,pad", CASES)
def test_fft_route_difference_image(ny, nx, L, dk, db, dt, pad):
    S, T, M = synth.roman_pair(ny, nx, seed=ny + L, n_stars=ny * nx // 300)
    S, T = S.astype(dt), T.astype(dt)
    pitch = nx + pad

    def dev(a, fill):
        b = np.full((ny, pitch), fill, dtype=a.dtype)
        b[:, :nx] = a
        return torch.from_numpy(b).to(DEV)

    St, Tt, Mt = dev(S, 1e30), dev(T, -1e30), dev(M, 1)
    dtype = sfft.F64 if dt == np.float64 else sfft.F32
    desc = sfft.make_desc(ny, nx, L, dk, db, dtype=dtype, pitch=pitch if pad else 0)
    out = {}
    for route in (0, 1):
        tn = sfft.sfft_tuning()
        tn.subtract_fft = route
        sfft.sfft_tuning_set(desc, tn)
        with sfft.sfft_plan(desc) as plan:
            th = torch.empty(plan.n, dtype=torch.float64, device=DEV)
            sfft.sfft_fit(plan, St, Tt, Mt, None, th, want_info=False)
            D = torch.full_like(St, 7.0)
            sfft.sfft_subtract(plan, St, Tt, th, D)
            torch.cuda.synchronize()
            out[route] = (th.cpu().numpy(), D.cpu().numpy())
    sfft.sfft_tuning_set(desc, sfft.sfft_tuning())
    th, Dfft = out[1]
    assert np.array_equal(out[0][0], th)  # the route changes only the difference image
    tmax = float(np.abs(T).max())
    ref = oracle.subtract(S.astype(np.float64), T.astype(np.float64), th, L, dk, db)
    err = np.abs(Dfft[:, :nx] - ref).max() / tmax
    err_direct = np.abs(Dfft[:, :nx] - out[0][1][:, :nx]).max() / tmax
    print("FFT-route D %dx%d L=%d dk=%d db=%d: vs oracle %.2e, vs direct %.2e" % (ny, nx, L, dk, db, err, err_direct))
    assert err <= 1e-5 and err_direct <= 1e-6
    if pad:
        assert np.all(Dfft[:, nx:] == 7.0)
