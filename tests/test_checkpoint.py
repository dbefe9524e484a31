"""Checkpoint/resume of the residual loop (host logic, no GPU): a stand-in
for the library's loop that chooses deterministically from the descriptors
fixed so far, so that an interrupted and resumed run can be compared with
an uninterrupted one; the fingerprint check; atomic writes."""
import os

import numpy as np
import pytest

from paper_2602_06986_gb300 import checkpoint as ck


class FakeSpace:
    """residual_loop: iteration D picks a descriptor from (y, fixed ids);
    records every call so that tests can see the one-iteration calls."""

    n_stored, n_total = 50, 5000

    def __init__(self):
        self.calls = []

    def residual_loop(self, y, n_iter, k, precision=0, sis_ids=None, fixed=()):
        fixed = [int(f) for f in fixed]
        self.calls.append((n_iter, list(fixed)))
        chosen = list(fixed)
        seed = int(np.sum(np.asarray(y) * 1e6)) % 9973
        for it in range(len(fixed), n_iter):
            chosen.append((seed * 31 + 7 * sum(chosen) + it) % self.n_total)
            sis_ids[it * k:(it + 1) * k] = np.arange(k, dtype=np.uint64) + np.uint64(chosen[-1])
        return {"chosen": chosen, "rmse": [1.0 / (i + 2) for i in range(n_iter)],
                "coefs": [[0.5] * (i + 2) for i in range(n_iter)],
                "stats": [{"screened": self.n_total, "reasons": {"valid": i}} for i in range(n_iter)]}


def test_interrupted_run_resumes_to_the_same_state(tmp_path):
    y = np.linspace(0.0, 1.0, 40)
    sp = FakeSpace()
    full = ck.residual_loop(sp, y, 3, 8, str(tmp_path / "a.npz"))
    sp2 = FakeSpace()
    p = str(tmp_path / "b.npz")
    part = ck.residual_loop(sp2, y, 3, 8, p, stop_after=1)
    assert len(part["chosen"]) == 1 and os.path.exists(p)
    resumed = ck.residual_loop(FakeSpace(), y, 3, 8, p)
    for key in ("chosen", "rmse", "coefs", "stats"):
        assert resumed[key] == full[key], key
    for a, b in zip(resumed["sis_ids"], full["sis_ids"]):
        np.testing.assert_array_equal(a, b)
    # one iteration per call, each resuming from the descriptors so far
    assert [c[0] for c in sp.calls] == [1, 2, 3]
    assert sp.calls[2][1] == full["chosen"][:2]
    # a finished checkpoint runs nothing more
    sp3 = FakeSpace()
    again = ck.residual_loop(sp3, y, 3, 8, p)
    assert sp3.calls == [] and again["chosen"] == full["chosen"]


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    p = str(tmp_path / "c.npz")
    ck.residual_loop(FakeSpace(), np.ones(10) * np.arange(10), 2, 4, p, stop_after=1)
    with pytest.raises(ValueError):
        ck.residual_loop(FakeSpace(), np.arange(10.0) + 1.0, 2, 4, p)
    with pytest.raises(ValueError):
        ck.residual_loop(FakeSpace(), np.ones(10) * np.arange(10), 2, 5, p)


def test_failed_write_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    p = str(tmp_path / "d.npz")
    y = np.arange(12.0)
    ck.residual_loop(FakeSpace(), y, 3, 4, p, stop_after=1)
    before = ck.load(p)

    def boom(src, dst):
        raise OSError("disk gone")

    monkeypatch.setattr(ck.os, "replace", boom)
    with pytest.raises(OSError):
        ck.residual_loop(FakeSpace(), y, 3, 4, p)
    monkeypatch.undo()
    after = ck.load(p)
    assert after["chosen"] == before["chosen"] and len(after["chosen"]) == 1
    done = ck.residual_loop(FakeSpace(), y, 3, 4, p)
    assert len(done["chosen"]) == 3
