"""The batch autotuner's host logic (no GPU): the fastest candidate wins, an
invalid candidate is skipped with its reason, the refinement stage re-times the
fastest few and can change the pick, and the result is cached per workload and
device."""
import pytest

from paper_1101_0809_gb300 import autotune as AT


def cands():
    return [dict(tile=t, ppb=p, K=k) for t in (8, 16) for p in (2048, 8192) for k in (3, 5)]


def sample_ms(c):
    # a made-up cost surface: the sample favours small blocks, tile 16 is invalid at ppb 2048 and K 3
    if c["tile"] == 16 and c["ppb"] == 2048 and c["K"] == 3:
        raise ValueError("tile larger than the smallest grid")
    return 10.0 + (c["ppb"] / 2048) * 0.1 + (1.0 if c["K"] == 3 else 0.0) - (0.2 if c["tile"] == 16 else 0.0)


def test_fastest_candidate_is_picked_and_invalid_ones_are_listed(tmp_path):
    path = str(tmp_path / "cache.json")
    best, table, cached = AT.tune("w", "gpu", cands(), sample_ms, path=path)
    assert not cached
    assert best == dict(tile=16, ppb=2048, K=5)
    bad = [t for t in table if t[1] is None]
    assert len(bad) == 1 and "smallest grid" in bad[0][2]
    assert len(table) == len(cands())


def test_refinement_retimes_the_fastest_few_and_can_change_the_pick(tmp_path):
    path = str(tmp_path / "cache.json")
    seen = []

    def cost(c):              # on the whole workload larger blocks pay
        return 20.0 - c["ppb"] / 1024

    def full_ms(c):
        seen.append(c)
        return cost(c)

    best, table, _ = AT.tune("w", "gpu", cands(), sample_ms, path=path, refine=full_ms, top=3)
    ranked = sorted([t for t in table if t[1] is not None and t[2] == ""], key=lambda t: t[1])[:3]
    assert seen == [t[0] for t in ranked]
    assert best == min(seen, key=cost)
    assert best["ppb"] == 8192
    assert sum(1 for t in table if t[2] == "refined") == 3


def test_cached_result_is_returned_for_the_same_workload_and_device(tmp_path):
    path = str(tmp_path / "cache.json")
    best, _, _ = AT.tune("w", "gpu", cands(), sample_ms, path=path)

    def never(c):
        raise AssertionError("a cached workload is not timed again")

    again, _, cached = AT.tune("w", "gpu", cands(), never, path=path)
    assert cached and again == best
    other, _, cached = AT.tune("w", "other gpu", cands(), sample_ms, path=path)
    assert not cached and other == best


def test_no_valid_candidate_raises(tmp_path):
    def broken(c):
        raise ValueError("does not fit")

    with pytest.raises(RuntimeError, match="does not fit"):
        AT.tune("w", "gpu", cands(), broken, path=str(tmp_path / "cache.json"))
