"""The seeded generator of uneven batch workloads (host logic, CPU)."""
import numpy as np

from paper_2103_01767_gb300 import synth


def test_batch_members_follow_the_recipe():
    ms = synth.batch_members(64, seed=7)
    assert len(ms) == 64
    assert {m.m for m in ms} == {32, 64, 128}
    for m in ms:
        assert max(128, 2 * m.m) <= m.n <= 512          # N >= 2 x probe
        assert 64 <= m.K <= 1024
        assert (m.loss == 0 and m.peak == 0.0) or (m.loss == 1 and m.peak == 1e3)
    assert {m.loss for m in ms} == {0, 1}
    # reproducible
    assert synth.batch_members(64, seed=7) == ms
    assert synth.batch_members(64, seed=8) != ms


def test_batch_positions_stay_inside_and_count_K():
    for mem in synth.batch_members(64, seed=7):
        pos = synth.batch_positions(mem)
        assert pos.shape == (mem.K, 2) and pos.dtype == np.int32
        assert pos.min() >= 0 and pos.max() <= mem.n - mem.m
