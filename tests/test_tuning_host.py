"""The autotuner's candidate set (host logic, no GPU): the knobs it spans and
where each applies."""
from paper_2203_02293_b300 import rt
from paper_2203_02293_b300.tuning import KNOBS, TALL_COLUMN_LAYERS, default_candidates


def _set(cands, key):
    return {c[key] for c in cands}


def test_candidates_span_every_knob():
    cands = default_candidates(20, 40)
    assert all(set(c) == set(KNOBS) for c in cands)
    assert _set(cands, "systems_per_lane") == {1, 2}
    assert _set(cands, "block_threads") == {128, 256}
    assert _set(cands, "ctas_per_sm") == {0, 2}
    # staging depth: both instances with two systems per lane, the default with one
    assert {c["staging_depth"] for c in cands if c["systems_per_lane"] == 2} == {
        rt.RT_STAGING_DEPTH_MIN, rt.RT_STAGING_DEPTH_MAX}
    assert {c["staging_depth"] for c in cands if c["systems_per_lane"] == 1} == {rt.RT_STAGING_DEPTH_MIN}
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)


def test_planck_staging_candidates_follow_g_points_and_column_height():
    assert _set(default_candidates(20, 40), "planck_staging") == {rt.RT_STAGE_SHARED}
    assert _set(default_candidates(20, TALL_COLUMN_LAYERS + 1), "planck_staging") == {
        rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT}
    assert _set(default_candidates(1, 40), "planck_staging") == {
        rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE}
