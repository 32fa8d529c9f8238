"""Batches of S x T pairs with uneven cutout sizes: lanes, graph replay, per-pair status,
and the autotuner -- all through the C ABI, checked against single-pair plans and the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
L, DK, DB = 5, 1, 1
FRAME = 320


@pytest.fixture(scope="module", autouse=True)
def _built():
    sfft_build.build()
    sfft.load_library()


def _cutouts(sizes, seed):
    """Per pair: science/template/mask frames of FRAME x FRAME and the cutout origin; the
    pair's cutout (ny, nx) sits at (oy, ox) and is addressed with the frame's pitch."""
    out = []
    for k, (ny, nx) in enumerate(sizes):
        S, T, M = synth.roman_pair(FRAME, FRAME, seed=seed + k, n_stars=120)
        oy, ox = 8 * (k % 3), 4 * (k % 5)
        out.append(dict(S=torch.from_numpy(S).to(DEV), T=torch.from_numpy(T).to(DEV),
                        M=torch.from_numpy(M).to(DEV), ny=ny, nx=nx, oy=oy, ox=ox))
    return out


def _view(t, c):
    return t.reshape(-1)[c["oy"] * FRAME + c["ox"]:]


def _pairs(cuts, n, x0=None):
    pairs, coeffs, diffs = [], [], []
    for k, c in enumerate(cuts):
        th = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
        D = torch.full((c["ny"], FRAME), float("nan"), dtype=torch.float32, device=DEV)
        pairs.append(sfft.make_pair(_view(c["S"], c), _view(c["T"], c), _view(c["M"], c), th, D, c["ny"], c["nx"],
                                    pitch=FRAME, x0=None if x0 is None else x0[k]))
        coeffs.append(th)
        diffs.append(D)
    return pairs, coeffs, diffs


def _single(c, n, solver=sfft.SOLVE_CHOLESKY, x0=None):
    d = sfft.make_desc(c["ny"], c["nx"], L, DK, DB, pitch=FRAME, solver=solver)
    with sfft.sfft_plan(d) as p:
        th = torch.empty(n, dtype=torch.float64, device=DEV)
        D = torch.full((c["ny"], FRAME), float("nan"), dtype=torch.float32, device=DEV)
        sfft.sfft_fit(p, _view(c["S"], c), _view(c["T"], c), _view(c["M"], c), x0, th)
        sfft.sfft_subtract(p, _view(c["S"], c), _view(c["T"], c), th, D)
        torch.cuda.synchronize()
    return th, D


SIZES = [(128, 128), (192, 160), (256, 256), (160, 224), (128, 256), (256, 192)]   # 3 x 2 pairs


@pytest.mark.parametrize("flags,lanes", [(0, 1), (0, 3), (sfft.BATCH_GRAPH, 4)])
def test_batch_matches_single_pair_plans(flags, lanes):
    cuts = _cutouts(SIZES, seed=40)
    n = oracle.n_unknowns(L, DK, DB)
    pairs, coeffs, diffs = _pairs(cuts, n)
    base = sfft.make_desc(128, 128, L, DK, DB)
    with sfft.sfft_batch_create(base, pairs, lanes=lanes, flags=flags) as b:
        infos = sfft.sfft_batch_info(b)
        for k, c in enumerate(cuts):
            th, D = _single(c, n)
            assert infos[k].status == 0
            # same kernels, same launch shapes: identical results
            assert torch.equal(coeffs[k], th)
            assert torch.equal(diffs[k][:, :c["nx"]], D[:, :c["nx"]])
        # a replay reproduces the first run bit for bit, after the outputs were cleared
        first = [t.clone() for t in coeffs]
        for t in coeffs:
            t.fill_(float("nan"))
        sfft.sfft_batch_run(b)
        sfft.sfft_batch_info(b)
        for k in range(len(cuts)):
            assert torch.equal(coeffs[k], first[k])


def test_batch_results_match_oracle_and_report_a_singular_pair():
    cuts = _cutouts(SIZES[:4], seed=60)
    cuts[2]["T"] = torch.zeros_like(cuts[2]["T"])          # no template: rank-deficient design
    n = oracle.n_unknowns(L, DK, DB)
    pairs, coeffs, diffs = _pairs(cuts, n)
    infos = sfft.sfft_batch(sfft.make_desc(128, 128, L, DK, DB), 2, 2, pairs)
    assert [i.status for i in infos] == [0, 0, sfft.ERR_NOT_SPD, 0]
    for k in (0, 1, 3):
        c = cuts[k]
        sl = (slice(c["oy"], c["oy"] + c["ny"]), slice(c["ox"], c["ox"] + c["nx"]))
        S, T, M = (c[a][sl].cpu().numpy() for a in ("S", "T", "M"))
        ref = oracle.fit(S, T, M, L, DK, DB)
        th = coeffs[k].cpu().numpy()
        assert np.linalg.norm(th - ref) <= 1e-6 * np.linalg.norm(ref)
        Dref = oracle.subtract(S, T, th, L, DK, DB)
        assert np.abs(diffs[k][:, :c["nx"]].cpu().numpy() - Dref).max() <= 1e-5 * np.abs(T).max()


def test_graph_batch_with_pcg_warm_starts():
    cuts = _cutouts(SIZES, seed=80)
    n = oracle.n_unknowns(L, DK, DB)
    # warm starts: the cold solutions perturbed by 1e-3
    cold = [_single(c, n)[0] for c in cuts]
    x0 = [t * (1 + 1e-3) for t in cold]
    pairs, coeffs, _ = _pairs(cuts, n, x0=x0)
    base = sfft.make_desc(128, 128, L, DK, DB, solver=sfft.SOLVE_PCG)
    with sfft.sfft_batch_create(base, pairs, lanes=3, flags=sfft.BATCH_GRAPH) as b:
        for _ in range(2):
            sfft.sfft_batch_run(b)
        infos = sfft.sfft_batch_info(b)
    for k in range(len(cuts)):
        assert infos[k].status == 0 and infos[k].fallback == 0
        assert infos[k].start_residual < 1e-2
        assert torch.linalg.norm(coeffs[k] - cold[k]) <= 1e-6 * torch.linalg.norm(cold[k])


def test_autotune_stores_a_valid_shape_that_fits_correctly():
    S, T, M = synth.roman_pair(512, 512, seed=5)
    St, Tt, Mt = (torch.from_numpy(a).to(DEV) for a in (S, T, M))
    d = sfft.make_desc(512, 512, 11, 2, 2)
    t, ms = sfft.sfft_autotune(d, St, Tt, Mt, trials=2)
    got, cached = sfft.sfft_tuning_get(d)
    assert cached and ms > 0
    assert (got.ycorr_bins, got.ycorr_split, got.ycorr_scalar, got.subtract_ctas, got.pcg_cluster) == \
        (t.ycorr_bins, t.ycorr_split, t.ycorr_scalar, t.subtract_ctas, t.pcg_cluster)
    with sfft.sfft_plan(d) as p:
        th = torch.empty(p.n, dtype=torch.float64, device=DEV)
        sfft.sfft_fit(p, St, Tt, Mt, None, th)
    ref = oracle.fit(S, T, M, 11, 2, 2)
    assert np.linalg.norm(th.cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)


def test_batch_with_host_buffers_copies_in_and_out_on_the_lanes():
    """Pairs that carry pinned host buffers: each run copies the cutouts in (2-D copies with the
    frames' pitch) and theta and D out; the host results equal single-pair device runs."""
    cuts = _cutouts(SIZES[:4], seed=100)
    n = oracle.n_unknowns(L, DK, DB)
    pairs, refs = [], []
    for k, c in enumerate(cuts):
        refs.append(_single(c, n))
        hs = {a: c[a].cpu().pin_memory() for a in ("S", "T", "M")}
        dev = {a: torch.zeros_like(c[a]) for a in ("S", "T", "M")}      # the copies land here
        th = torch.empty(n, dtype=torch.float64, device=DEV)
        D = torch.empty((c["ny"], FRAME), dtype=torch.float32, device=DEV)
        host = dict(sci=_view(hs["S"], c), tmpl=_view(hs["T"], c), mask=_view(hs["M"], c),
                    coeffs=torch.full((n,), float("nan"), dtype=torch.float64).pin_memory(),
                    diff=torch.full((c["ny"], FRAME), float("nan"), dtype=torch.float32).pin_memory())
        c.update(host=host, keep=(hs, dev, th, D))
        pairs.append(sfft.make_pair(_view(dev["S"], c), _view(dev["T"], c), _view(dev["M"], c), th, D,
                                    c["ny"], c["nx"], pitch=FRAME, host=host))
    with sfft.sfft_batch_create(sfft.make_desc(128, 128, L, DK, DB), pairs, lanes=2, flags=sfft.BATCH_GRAPH) as b:
        for c in cuts:
            c["host"]["coeffs"].fill_(float("nan"))
        sfft.sfft_batch_run(b)
        sfft.sfft_batch_info(b)
    for c, (th, D) in zip(cuts, refs):
        assert torch.equal(c["host"]["coeffs"], th.cpu())
        assert torch.equal(c["host"]["diff"][:, :c["nx"]], D[:, :c["nx"]].cpu())


def test_batch_with_contiguous_host_frames():
    """Whole frames (pitch == nx) with pinned host buffers: the copies in and out are single
    contiguous transfers; the host results equal single-pair device runs bit for bit."""
    n = oracle.n_unknowns(L, DK, DB)
    pairs, refs, keep = [], [], []
    for k, (ny, nx) in enumerate([(160, 192), (224, 128), (128, 256)]):
        S, T, M = synth.roman_pair(ny, nx, seed=300 + k, n_stars=60)
        c = dict(S=torch.from_numpy(S).to(DEV), T=torch.from_numpy(T).to(DEV), M=torch.from_numpy(M).to(DEV))
        d = sfft.make_desc(ny, nx, L, DK, DB)
        with sfft.sfft_plan(d) as p:
            th = torch.empty(n, dtype=torch.float64, device=DEV)
            D = torch.empty((ny, nx), dtype=torch.float32, device=DEV)
            sfft.sfft_fit(p, c["S"], c["T"], c["M"], None, th)
            sfft.sfft_subtract(p, c["S"], c["T"], th, D)
            torch.cuda.synchronize()
        refs.append((th, D))
        host = dict(sci=torch.from_numpy(S).pin_memory(), tmpl=torch.from_numpy(T).pin_memory(),
                    mask=torch.from_numpy(M).pin_memory(),
                    coeffs=torch.full((n,), float("nan"), dtype=torch.float64).pin_memory(),
                    diff=torch.full((ny, nx), float("nan"), dtype=torch.float32).pin_memory())
        dev = [torch.zeros_like(c[a]) for a in ("S", "T", "M")]
        th2 = torch.empty(n, dtype=torch.float64, device=DEV)
        D2 = torch.empty((ny, nx), dtype=torch.float32, device=DEV)
        keep.append((host, dev, th2, D2))
        pairs.append(sfft.make_pair(dev[0], dev[1], dev[2], th2, D2, ny, nx, host=host))
    with sfft.sfft_batch_create(sfft.make_desc(128, 128, L, DK, DB), pairs, lanes=3, flags=sfft.BATCH_GRAPH) as b:
        sfft.sfft_batch_run(b)
        infos = sfft.sfft_batch_info(b)
    for (host, _, _, _), (th, D), info in zip(keep, refs, infos):
        assert info.status == 0
        assert torch.equal(host["coeffs"], th.cpu())
        assert torch.equal(host["diff"], D.cpu())


def test_batch_runs_the_warm_start_network_inside_the_graph():
    """Pairs that carry PSF stamps, with a warm-start network given to the batch: every run
    evaluates the network on the stamps (inside the graph) and starts those pairs' PCG solves
    from its warm starts.  The coefficients equal, bit for bit, a batch whose warm starts
    were computed beforehand by sfft_cnn_warm_start and passed as x0; a pair without stamps
    starts cold as before."""
    cuts = _cutouts(SIZES[:4], seed=300)
    n = oracle.n_unknowns(L, DK, DB)
    nker = L * L * (DK + 1) * (DK + 2) // 2
    cnn = sfft.sfft_cnn_create(nker, 8)
    sfft.sfft_cnn_set_params(cnn, torch.from_numpy(synth.cnn_init(nker, 3) * 0.05).to(DEV))
    stamps = torch.from_numpy(np.stack([synth.psf_stamps(synth.psf_field(40 + k)) for k in range(3)])).to(DEV)
    x0 = torch.zeros((3, n), dtype=torch.float64, device=DEV)
    sfft.sfft_cnn_warm_start(cnn, stamps, 3, n, x0)
    desc = sfft.make_desc(128, 128, L, DK, DB, solver=sfft.SOLVE_PCG)
    # reference: x0 given explicitly (the fourth pair cold)
    pairs_ref, th_ref, _ = _pairs(cuts, n, x0=[x0[0], x0[1], x0[2], None])
    with sfft.sfft_batch_create(desc, pairs_ref, lanes=2, flags=sfft.BATCH_GRAPH) as b:
        sfft.sfft_batch_run(b)
        i_ref = sfft.sfft_batch_info(b)
    # the network inside the batch, fed each pair's stamps
    pairs, th, _ = _pairs(cuts, n)
    for k in range(3):
        pairs[k].psf_stamps = stamps[k].data_ptr()
    with sfft.sfft_batch_create(desc, pairs, lanes=2, flags=sfft.BATCH_GRAPH, cnn=cnn) as b:
        for t in th:
            t.fill_(float("nan"))
        sfft.sfft_batch_run(b)
        infos = sfft.sfft_batch_info(b)
    for a, r in zip(th, th_ref):
        assert torch.equal(a, r)
    assert [i.iterations for i in infos] == [i.iterations for i in i_ref]
    assert [i.start_residual for i in infos] == [i.start_residual for i in i_ref]
    # a network whose width does not match the basis is rejected
    with sfft.sfft_cnn_create(nker + 1, 4) as bad:
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_batch_create(desc, pairs, lanes=2, cnn=bad)
        assert ei.value.status == sfft.ERR_INVALID_ARG
    cnn.close()
