"""The tile autotuner's host logic (no GPU): every step kernel has
candidate tiles, each a legal block for it; the tuner keeps the fastest
candidate, skips tiles the library rejects, caches its choice per (GPU,
lattice, precision, kind, size class) and takes it from the cache next time
without stepping.  The CUDA timing is replaced by a fake clock."""
import types

import pytest

import paper_2409_10399_gb300 as lbm
from paper_2409_10399_gb300 import autotune


@pytest.mark.parametrize("lat", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev", "fp64dev", "fp16ab"])
def test_every_kernel_has_legal_candidates(lat, prec):
    mt = lbm.tile_limit(lat, prec)
    tiles = autotune.CANDIDATES[(lat, mt)]
    assert tiles
    for tx, ty, tz in tiles:
        n = tx * ty * tz
        assert n % 32 == 0 and n <= mt, (lat, prec, (tx, ty, tz))
        if lat < 3:
            assert tz == 1
        if lat < 2:
            assert ty == 1


class _Fake:
    """A Simulation stand-in: set_tile (rejecting one tile), step advancing a
    fake clock by a per-tile cost."""

    def __init__(self, cost, reject):
        self.cost, self.reject = cost, reject
        self.tile, self.clock, self.steps = None, 0.0, 0

    def set_tile(self, *t):
        if t in self.reject:
            raise lbm.LBMError(-1, "lbm_set_tile")
        self.tile = t

    def step(self, n):
        self.clock += n * self.cost[self.tile]
        self.steps += n


def _fake_cuda(monkeypatch, obj):
    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = obj.clock

        def elapsed_time(self, other):
            return (other.t - self.t) * 1e3  # ms

    import torch
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "fake GPU")


def test_tune_keeps_the_fastest_and_caches(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tiles.json"))
    tiles = autotune.CANDIDATES[(2, 128)]
    cost = {t: 1e-4 * (1 + i) for i, t in enumerate(tiles)}
    best = tiles[3]
    cost[best] = 1e-5
    obj = _Fake(cost, reject={tiles[1]})
    _fake_cuda(monkeypatch, obj)
    tile, times = autotune.tune(obj, 2, "fp32", 1 << 20, "single", steps=10)
    assert tile == best and obj.tile == best
    assert tiles[1] not in times and set(times) == set(tiles) - {tiles[1]}
    for t, sec in times.items():
        assert sec == pytest.approx(cost[t])
    # the cache answers the same key without stepping; another size class tunes again
    steps = obj.steps
    obj.tile = None
    tile2, times2 = autotune.tune(obj, 2, "fp32", (1 << 20) + 5, "single", steps=10)
    assert tile2 == best and obj.tile == best and obj.steps == steps and times2 == times
    autotune.tune(obj, 2, "fp32", 1 << 22, "single", steps=10)
    assert obj.steps > steps
    assert autotune._size_class(1 << 20) == autotune._size_class((1 << 21) - 1) != autotune._size_class(1 << 21)
