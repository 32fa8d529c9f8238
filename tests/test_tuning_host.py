"""The launch-tuning cache is host logic: set/get, validation against the geometry's
limits, and the text round trip (no GPU work)."""
import pytest

from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sfft_build.build()
    sfft.load_library()


def _t(bins=0, split=0, scalar=0, ctas=0, cluster=0):
    t = sfft.sfft_tuning()
    t.ycorr_bins, t.ycorr_split, t.ycorr_scalar, t.subtract_ctas, t.pcg_cluster = bins, split, scalar, ctas, cluster
    return t


def _fields(t):
    return (t.ycorr_bins, t.ycorr_split, t.ycorr_scalar, t.subtract_ctas, t.pcg_cluster)


def test_set_get_and_validation():
    d = sfft.make_desc(1000, 900, 11, 2, 2)
    t, cached = sfft.sfft_tuning_get(d)
    assert not cached and _fields(t) == (0, 0, 0, 0, 0)
    sfft.sfft_tuning_set(d, _t(3, 3, 1, 3, 8))
    t, cached = sfft.sfft_tuning_get(d)
    assert cached and _fields(t) == (3, 3, 1, 3, 8)
    # entries are per descriptor
    assert not sfft.sfft_tuning_get(sfft.make_desc(1000, 900, 11, 2, 1))[1]
    for bad in (_t(bins=10_000), _t(split=10_000), _t(scalar=2), _t(ctas=5), _t(bins=-1), _t(cluster=4)):
        with pytest.raises(sfft.SfftError):
            sfft.sfft_tuning_set(d, bad)
    assert _fields(sfft.sfft_tuning_get(d)[0]) == (3, 3, 1, 3, 8)


def test_save_and_load_round_trip(tmp_path):
    d1 = sfft.make_desc(512, 512, 11, 2, 2)
    d2 = sfft.make_desc(2048, 1536, 7, 1, 1, solver=sfft.SOLVE_PCG)
    sfft.sfft_tuning_set(d1, _t(2, 1, 0, 1))
    sfft.sfft_tuning_set(d2, _t(3, 4, 1, 2, 16))
    path = str(tmp_path / "tuning.txt")
    sfft.sfft_tuning_save(path)
    sfft.sfft_tuning_set(d1, _t(1, 1, 1, 4))
    sfft.sfft_tuning_load(path)
    assert _fields(sfft.sfft_tuning_get(d1)[0]) == (2, 1, 0, 1, 0)
    assert _fields(sfft.sfft_tuning_get(d2)[0]) == (3, 4, 1, 2, 16)
    bad = tmp_path / "bad.txt"
    bad.write_text("512 512 0 11 2 2 0 0 0 0 : 1 2\n")
    with pytest.raises(sfft.SfftError):
        sfft.sfft_tuning_load(str(bad))


def test_workspace_size_follows_the_tuning():
    d = sfft.make_desc(1024, 1024, 11, 2, 2)
    base = sfft.sfft_workspace_size(d)
    sfft.sfft_tuning_set(d, _t(split=1))
    small = sfft.sfft_workspace_size(d)
    sfft.sfft_tuning_set(d, _t(split=8))
    big = sfft.sfft_workspace_size(d)
    assert small <= base <= big and small < big


def test_descriptor_limits():
    """The kernel instantiations cover DK <= 3, DB <= 4 and odd L <= 15 (the streaming
    residual and difference kernels, the y-correlation roles); the host rejects the rest
    before any GPU work: DK = 4 needs more than 256 work items per frequency."""
    for ny, nx, L, dk, db in ((64, 64, 1, 0, 0), (300, 280, 15, 3, 2), (128, 200, 5, 1, 4), (4088, 4088, 11, 2, 2)):
        assert sfft.sfft_workspace_size(sfft.make_desc(ny, nx, L, dk, db)) > 0
    for L, dk, db, what in ((11, 4, 0, "work items"), (11, 2, 5, "db=5"), (12, 2, 2, ""), (17, 1, 1, ""),
                            (11, -1, 0, "")):
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_workspace_size(sfft.make_desc(256, 256, L, dk, db))
        assert ei.value.status == sfft.ERR_INVALID_ARG and what in str(ei.value)
