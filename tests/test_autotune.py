"""Block-count autotuner: candidate layouts, the accuracy-guarded choice and the cache (host
logic, no GPU; the measured path runs in tests/test_gpu_batch.py)."""
import json

import pytest

from paper_1502_07806_b300 import autotune as at


@pytest.mark.parametrize("n", [1, 7, 200, 256, 1280, 3000, 9072])
def test_candidates_cover_the_width_range(n):
    c = at.candidates(n)
    assert c[0] == at.default_nblocks(n)
    assert len(c) == len(set(c))
    assert all(1 <= p <= n for p in c)
    if n >= 256:
        widths = {n / p for p in c}
        assert min(widths) < 100 and max(widths) > 180      # both ends of 64 .. 256 are tried


def test_default_layout_is_config4_rule():
    for n, want in [(200, 3), (640, 10), (1280, 10), (3000, 11), (100, 1)]:
        m = min(256, max(64, n // 10))
        assert at.default_nblocks(n) == max(1, n // m) == want


def test_choose_takes_fastest_within_the_residual_slack():
    meas = {10: (5.0, 1e-6), 8: (4.0, 1.5e-6), 20: (3.0, 5e-6), 5: (4.5, 1e-7)}
    # 20 is fastest but its residual is 5x the default's: rejected; 8 is next fastest
    assert at.choose(meas, 10) == 8
    meas[20] = (3.0, 2e-6)
    assert at.choose(meas, 10) == 20
    # ties in time go to the smaller block count; the default is always admissible
    assert at.choose({10: (1.0, 1e-3), 4: (1.0, 1e-12)}, 10) == 4
    assert at.choose({10: (9.0, 0.0), 4: (1.0, 1e-9)}, 10) == 10


def test_choose_needs_the_default():
    with pytest.raises(ValueError):
        at.choose({4: (1.0, 1e-9)}, 10)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    at._memory.clear()
    assert at.lookup("B300", 1280, 2, path) is None
    at.remember("B300", 1280, 2, 12, path)
    at._memory.clear()                                   # a fresh process reads the file
    assert at.lookup("B300", 1280, 2, path) == 12
    assert at.lookup("B300", 1290, 2, path) == 12        # same size class
    assert at.lookup("B300", 1280, 0, path) is None      # other form
    assert at.lookup("B300", 1500, 2, path) is None
    data = json.load(open(path))
    assert data == {at.cache_key("B300", 1280, 2): 12}
    at.remember("B300", 3000, 0, 11, path)
    assert len(json.load(open(path))) == 2
    at._memory.clear()
