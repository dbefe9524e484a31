"""Host logic of the autotuner against a fake timer (no GPU): coordinate
descent finds the fastest setting of a synthetic cost surface, keeps the
default when nothing beats it by the margin, caches by workload class,
never re-times a cached class, and round-trips through JSON."""
import json

import pytest

from paper_2602_06986_gb300 import autotune as at


class Fake:
    """A cost surface over settings; 'installed' is what run() sees."""

    def __init__(self, cost):
        self.cost = cost
        self.installed = None
        self.calls = 0
        self.runs = 0

    def install(self, cfg):
        self.installed = dict(cfg) if cfg else {}

    def run(self):
        self.runs += 1

    def timer(self, fn):
        fn()
        self.calls += 1
        return self.cost(self.installed)


def test_finds_minimum_of_each_parameter():
    # best at tile_group 4, seed_stride 128 (defaults: 8 and 64)
    def cost(c):
        g = c.get("tile_group", 8)
        s = c.get("seed_stride", 64)
        return 1.0 + 0.1 * abs(g - 4) + 0.05 * abs(s - 128) / 32

    f = Fake(cost)
    cache = {}
    e = at.tune("screen_tc", 20000, 16, f.run, cache=cache, timer=f.timer, install=f.install, reps=1)
    assert e["config"] == {"tile_group": 4, "seed_stride": 128}
    assert f.installed == {}  # defaults restored afterwards
    assert at.lookup(cache, "screen_tc", 20000, 16) == {"tile_group": 4, "seed_stride": 128}
    # one untimed warm-up run, then one run per timed setting
    assert f.runs == 1 + f.calls
    # same class: cached, not timed or run again
    n, r = f.calls, f.runs
    at.tune("screen_tc", 17000, 9, f.run, cache=cache, timer=f.timer, install=f.install)
    assert f.calls == n and f.runs == r
    # another class is tuned separately
    assert at.lookup(cache, "screen_tc", 500, 64) is None


def test_margin_keeps_defaults_against_noise():
    import random

    rnd = random.Random(0)
    f = Fake(lambda c: 1.0 + rnd.uniform(-0.005, 0.005))
    e = at.tune("batched", 800, 1, f.run, timer=f.timer, install=f.install, reps=3, margin=0.02)
    assert e["config"] == {}
    # the defaults, then every candidate value once
    assert len(e["tried"]) == 1 + len(at.CANDIDATES["batched"]["batch_job_samples"])


def test_buckets_and_keys():
    assert at.bucket_n(1) == 1 and at.bucket_n(1000) == 1024 and at.bucket_n(1024) == 1024
    assert at.bucket_n(20000) == 32768
    assert [at.bucket_t(t) for t in (1, 2, 7, 8, 16, 17, 64, 65)] == ["1", "2-7", "2-7", "8-16", "8-16", "17-32",
                                                                        "33-64", ">64"]
    assert at.key("screen_tc", 20000, 16) == "screen_tc|N32768|T8-16"
    with pytest.raises(ValueError):
        at.bucket_n(0)


def test_json_round_trip_and_apply(tmp_path):
    f = Fake(lambda c: 2.0 - 0.5 * (c.get("gram_max_n", 2048) == 16))
    cache = {}
    at.tune("screen_single", 1000, 1, f.run, cache=cache, timer=f.timer, install=f.install, reps=1)
    p = tmp_path / "tune.json"
    at.save(str(p), cache)
    back = at.load(str(p))
    assert back == json.loads(json.dumps(cache))
    got = at.apply(back, "screen_single", 900, 1, install=f.install)
    assert got == {"gram_max_n": 16} and f.installed == {"gram_max_n": 16}
    assert at.apply(back, "screen_single", 100, 1, install=f.install) is None and f.installed == {}
    assert at.load(str(tmp_path / "missing.json")) == {}


def test_tuning_fields_and_ranges_host():
    """dse_set_tuning / dse_get_tuning on the host (no GPU needed): every
    candidate value the tuner may install is accepted, values outside a
    field's range are rejected, and None restores the defaults."""
    from paper_2602_06986_gb300 import dse

    try:
        for cls, params in at.CANDIDATES.items():
            for field, values in params.items():
                assert field in dse.TUNING_FIELDS, (cls, field)
                for v in values:
                    dse.set_tuning({field: v})
                    assert dse.get_tuning()[field] == v, (cls, field, v)
        for bad in ({"gmt_cluster": 3}, {"gmt_group": 5000}, {"gram_max_n": 8}):
            with pytest.raises(dse.DseError):
                dse.set_tuning(bad)
        dse.set_tuning(None)
        t = dse.get_tuning()
        assert t["gmt_cluster"] == 2 and t["gmt_group"] == 2
    finally:
        dse.set_tuning(None)
