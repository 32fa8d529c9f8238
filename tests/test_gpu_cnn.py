"""The warm-start network's CUDA kernels against the FP64 reference (oracle/cnn_oracle.py),
and what the trained network gains the PCG solve.

Tolerances: the kernels compute in FP32 (sums of at most 32 x 9 x 2 = 576 products per
value in the forward pass, up to 64 x 256 in the weight gradients); the comparison allows
1e-5 of the largest magnitude for outputs and 1e-4 for gradients.
"""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as C
from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import learned, sfft, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    sfft_build.build()
    sfft.load_library()


def _case(n_out, batch, seed):
    rng = np.random.default_rng(seed)
    p = synth.cnn_init(n_out, seed).astype(np.float64)
    p += 0.02 * rng.normal(size=p.size)
    x = np.stack([synth.psf_stamps(synth.psf_field(seed * 100 + i)) for i in range(batch)]).astype(np.float64)
    x += 0.1 * rng.normal(size=x.shape)            # off-distribution values too
    t = 0.05 * rng.normal(size=(batch, n_out))
    return p.astype(np.float32), x.astype(np.float32), t.astype(np.float32)


def _net(n_out, batch, p):
    cnn = sfft.sfft_cnn_create(n_out, batch)
    assert sfft.sfft_cnn_param_count(cnn) == C.param_count(n_out)
    sfft.sfft_cnn_set_params(cnn, torch.from_numpy(p).to(DEV))
    return cnn


@pytest.mark.parametrize("n_out,batch", [(726, 4), (37, 3)])
def test_forward_matches_reference(n_out, batch):
    p, x, _ = _case(n_out, batch, seed=3)
    with _net(n_out, batch, p) as cnn:
        out = torch.empty((batch, n_out), dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_forward(cnn, torch.from_numpy(x).to(DEV), batch, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
    ref, _ = C.forward(p.astype(np.float64), x.astype(np.float64), n_out)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("n_out,batch", [(726, 5), (37, 2)])
def test_gradients_match_reference(n_out, batch):
    p, x, t = _case(n_out, batch, seed=4)
    with _net(n_out, batch, p) as cnn:
        g = torch.empty(p.size, dtype=torch.float32, device=DEV)
        gin = torch.empty(x.shape, dtype=torch.float32, device=DEV)
        loss = torch.empty(1, dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_gradients(cnn, torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV), batch, g, gin, loss)
        torch.cuda.synchronize()
        g, gin, loss = g.cpu().numpy().astype(np.float64), gin.cpu().numpy().astype(np.float64), float(loss.item())
    lref, gref, ginref = C.gradients(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), n_out)
    assert loss == pytest.approx(lref, rel=1e-5)
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in C.param_shapes(n_out)])
    for a, b in zip(bounds[:-1], bounds[1:]):       # layer by layer
        scale = np.abs(gref[a:b]).max()
        assert np.abs(g[a:b] - gref[a:b]).max() <= 1e-4 * scale, (a, b)
    assert np.abs(gin - ginref).max() <= 1e-4 * np.abs(ginref).max()


def test_adam_step_matches_reference():
    n_out, batch, lr = 37, 4, 1e-3
    p, x, t = _case(n_out, batch, seed=5)
    with _net(n_out, batch, p) as cnn:
        loss = torch.empty(1, dtype=torch.float32, device=DEV)
        xs, ts = torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV)
        sfft.sfft_cnn_train_step(cnn, xs, ts, batch, lr, loss)
        sfft.sfft_cnn_train_step(cnn, xs, ts, batch, lr, loss)
        p2 = torch.empty(p.size, dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_get_params(cnn, p2)
        p2 = p2.cpu().numpy().astype(np.float64)
    q = p.astype(np.float64)
    m = v = np.zeros(q.size)
    big = None
    for step in (1, 2):
        _, g, _ = C.gradients(q, x.astype(np.float64), t.astype(np.float64), n_out)
        # Adam normalises each gradient; where the reference gradient is tiny its FP32
        # value has no correct digits, so compare the well-determined entries only
        mask = np.abs(g) > 1e-3 * np.abs(g).max()
        big = mask if big is None else big & mask
        q, m, v = C.adam_step(q, g, m, v, step, lr)
    assert np.abs((p2 - p)[big] - (q - p)[big]).max() <= 2e-3 * lr * 2
    assert np.abs(p2 - p).max() <= 2 * lr * 1.01


def test_training_reduces_loss_and_warm_start_layout():
    stamps, targets, coeffs = learned.make_training_set(96, seed=11, size=128)
    n_out = targets.shape[1]
    assert n_out == 726
    cnn, losses = learned.train(stamps, targets, epochs=40, batch=32, lr=2e-3)
    with cnn:
        assert losses[-1] < 0.7 * losses[0], losses
        x0 = learned.warm_starts(cnn, stamps[:5], coeffs.shape[1])
        out = torch.empty((5, n_out), dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_forward(cnn, stamps[:5], 5, out)
        torch.cuda.synchronize()
        assert torch.equal(x0[:, :n_out], out.double())
        assert torch.count_nonzero(x0[:, n_out:]) == 0


def test_invalid_arguments_are_rejected():
    with pytest.raises(sfft.SfftError):
        sfft.sfft_cnn_create(0, 4)
    with sfft.sfft_cnn_create(10, 4) as cnn:
        x = torch.zeros((8, 18, 32, 32), device=DEV)
        out = torch.empty((8, 10), device=DEV)
        with pytest.raises(sfft.SfftError):
            sfft.sfft_cnn_forward(cnn, x, 8, out)       # batch above max_batch


@pytest.mark.slow
def test_trained_network_gains_the_pcg_solve():
    """Train on fits of random PSF fields, then warm-start PCG on a Roman-like pair whose
    fields the network never saw.  Against the cold start (the method without the network)
    the starting residual falls from 1 to below 0.25 and PCG needs no more iterations; the
    solution agrees with the FP64 Cholesky solve.  (With the FP32 Cholesky preconditioner
    each iteration cuts the residual by about 1e6, so a start that is better by a factor of
    ten saves an iteration only when it moves the last one across the tolerance.  On noisy
    frames the least-squares kernel carries noise-fitted wing terms no PSF-based prediction
    can know, so the starting residual cannot approach zero; the identity kernel is printed
    for context.)"""
    stamps, targets, _ = learned.make_training_set(2048, seed=1000, size=256)
    cnn, losses = learned.train(stamps, targets, epochs=40, batch=64, lr=1e-3)
    assert losses[-1] < 0.1 * losses[0], losses
    ny = nx = 1024
    S, T, M = synth.roman_pair(ny, nx, seed=77)
    St, Tt, Mt = (torch.from_numpy(a).to(DEV) for a in (S, T, M))
    field_stamps = torch.from_numpy(synth.psf_stamps(synth.roman_field())[None]).to(DEV)
    with cnn, sfft.sfft_plan(sfft.make_desc(ny, nx, 11, 2, 2, solver=sfft.SOLVE_PCG, refine=-1)) as plan, \
            sfft.sfft_plan(sfft.make_desc(ny, nx, 11, 2, 2, refine=-1)) as chol:
        n = plan.n
        x0 = learned.warm_starts(cnn, field_stamps, n)[0].contiguous()
        naive = torch.zeros(n, dtype=torch.float64, device=DEV)
        naive[60] = 1.0                                   # a_{00} at the centre lag: the identity kernel
        th = {k: torch.empty(n, dtype=torch.float64, device=DEV) for k in ("cold", "cnn", "naive", "chol")}
        info = {
            "cold": sfft.sfft_fit(plan, St, Tt, Mt, None, th["cold"]),
            "cnn": sfft.sfft_fit(plan, St, Tt, Mt, x0, th["cnn"]),
            "naive": sfft.sfft_fit(plan, St, Tt, Mt, naive, th["naive"]),
        }
        sfft.sfft_fit(chol, St, Tt, Mt, None, th["chol"])
        ref = th["chol"].cpu().numpy()
    for k in ("cold", "cnn", "naive"):
        assert info[k].status == 0 and info[k].fallback == 0
        assert np.linalg.norm(th[k].cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    print("start residual: cold %.3e naive %.3e cnn %.3e; iterations: cold %d naive %d cnn %d" % (
        info["cold"].start_residual, info["naive"].start_residual, info["cnn"].start_residual,
        info["cold"].iterations, info["naive"].iterations, info["cnn"].iterations))
    assert info["cold"].start_residual == 1.0
    assert info["cnn"].start_residual < 0.25
    assert info["cnn"].iterations <= info["cold"].iterations


def test_save_and_load_round_trip(tmp_path):
    """A saved network loads into a fresh one with the same outputs; a file for another
    output width, a truncated file or a foreign file is rejected."""
    n_out, batch = 37, 3
    p, x, _ = _case(n_out, batch, seed=8)
    path = str(tmp_path / "net.bin")
    xs = torch.from_numpy(x).to(DEV)
    with _net(n_out, batch, p) as a:
        sfft.sfft_cnn_save(a, path)
        out_a = torch.empty((batch, n_out), dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_forward(a, xs, batch, out_a)
    with sfft.sfft_cnn_create(n_out, batch) as b:
        sfft.sfft_cnn_load(b, path)
        got = torch.empty(C.param_count(n_out), dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_get_params(b, got)
        out_b = torch.empty((batch, n_out), dtype=torch.float32, device=DEV)
        sfft.sfft_cnn_forward(b, xs, batch, out_b)
        torch.cuda.synchronize()
        assert torch.equal(got.cpu(), torch.from_numpy(p))
        assert torch.equal(out_a, out_b)
    with sfft.sfft_cnn_create(n_out + 1, batch) as c:
        with pytest.raises(sfft.SfftError):
            sfft.sfft_cnn_load(c, path)
    raw = open(path, "rb").read()
    short = str(tmp_path / "short.bin")
    open(short, "wb").write(raw[:-4])
    foreign = str(tmp_path / "foreign.bin")
    open(foreign, "wb").write(b"NOTANNET" + raw[8:])
    with sfft.sfft_cnn_create(n_out, batch) as d:
        for bad in (short, foreign, str(tmp_path / "missing.bin")):
            with pytest.raises(sfft.SfftError):
                sfft.sfft_cnn_load(d, bad)
