"""Host logic of the schedule autotuner (no GPU): the candidate set of a
context and the JSON cache of chosen tunings."""
from paper_2107_06635_gb300 import autotune, ntu


def test_candidates_cover_the_valid_schedules():
    # D = 8 split-BF16: t12 pairing on/off x 2 or 3 ALS CTAs x splits up to
    # the allocated 4 x both builds of the reduced metric
    c = autotune.candidates(8, ntu.NTU_MIXED_BF16X3, 4, (1, 2))
    assert len(c) == 2 * 2 * 3 * 2
    assert len({tuple(sorted(t.items())) for t in c}) == len(c)
    assert {t["als_split"] for t in c} == {1, 2, 4}
    # no pairing below D = 8, no split beyond what the context allocated
    c = autotune.candidates(4, ntu.NTU_MIXED_BF16X3, 2, (1,))
    assert all(t["t12_pair"] == -1 and t["als_split"] in (1, 2) for t in c)
    assert len(c) == 2 * 2
    # FP64 contexts do not split
    c = autotune.candidates(8, ntu.NTU_FP64, 4, (0,))
    assert all(t["als_split"] == 1 for t in c)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuning.json")
    work = {"D": 8, "r": 2, "batch": 912}
    assert autotune.lookup("GPU", work, path) is None
    rec = {"chosen": dict(autotune.AUTOMATIC, als_split=2), "chosen_ms": 1.0}
    autotune.remember("GPU", work, rec, path)
    autotune.remember("GPU", {"D": 4}, {"chosen": autotune.AUTOMATIC}, path)
    assert autotune.lookup("GPU", work, path) == rec
    assert autotune.lookup("other GPU", work, path) is None
    # the key does not depend on the order of the workload's fields
    assert autotune.lookup("GPU", {"batch": 912, "r": 2, "D": 8}, path) == rec
