"""Host logic of the autotuner (no GPU): candidate generation and selection."""
from paper_1706_03024_gb300.autotune import Candidate, default_candidates, select


def test_default_candidates_cover_depth_block_and_cells():
    c = default_candidates(has_grid=True, max_cell=8)
    assert {x.regroup for x in c} >= {1, 2, 4, 8}
    assert {x.block_size for x in c} == {128, 256}
    assert {x.form for x in c} == {"wavefront", "wavefront_warp", "wavefront_pool"}
    assert all(x.block_size == 128 and x.macro_cell == 0 for x in c if x.form == "wavefront_pool")
    assert {x.skip_cell for x in c} == {0, 1, 2, 4, 8}
    assert any(x.macro_cell for x in c)
    h = default_candidates(has_grid=False)
    assert {x.skip_cell for x in h} == {0} and not any(x.macro_cell for x in h)


def test_select_keeps_the_fastest_after_retiming():
    cands = [Candidate(regroup=r) for r in (1, 2, 4, 8)]
    speed = {1: 10.0, 2: 30.0, 4: 29.0, 8: 5.0}
    calls = []

    def measure(c):
        calls.append(c.regroup)
        return speed[c.regroup]
    res = select(cands, measure)
    assert res.best.regroup == 2
    # finalists (within the pruning factor of the best) are timed twice
    assert calls.count(2) == 2 and calls.count(4) == 2 and calls.count(8) == 1


def test_select_is_robust_to_a_noisy_first_timing():
    seq = {2: iter([100.0, 20.0]), 4: iter([70.0, 60.0])}
    res = select([Candidate(regroup=2), Candidate(regroup=4)], lambda c: next(seq[c.regroup]))
    assert res.best.regroup == 4
