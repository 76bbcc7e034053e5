"""The autotuner: stored choices per graph class, and (on the GPU) a search
whose every setting must give the same counts."""
import json

import pytest

from paper_1503_02368_gb300 import autotune


def test_save_and_load_roundtrip(tmp_path):
    p = str(tmp_path / "t.json")
    best = {"tau": 64, "cta_warps": 8, "light_max": 16, "seconds": 1.0}
    autotune.save("cls_a", best, [best], path=p)
    autotune.save("cls_b", dict(best, tau=8), [best], path=p)
    assert autotune.load("cls_a", path=p) == best
    assert autotune.load("cls_b", path=p)["tau"] == 8
    assert autotune.load("missing", path=p) is None
    assert set(json.load(open(p))) == {"cls_a", "cls_b"}


def test_committed_choices_are_valid():
    for cls in ("rmat_s22_triangle", "rmat_s20_ego4096"):
        b = autotune.load(cls)
        assert b is not None
        assert b["cta_warps"] in (4, 8, 16) and 1 <= b["light_max"] <= 32 and b["tau"] >= 0
        assert b.get("pair_warps", 1) in (1, 2, 4)


@pytest.mark.gpu
def test_tuning_search_keeps_counts():
    import synth
    from synth import workloads as W
    g = W.rmat_graph(12, 1503 + 12)
    best, trials = autotune.tune_whole(g, "triangle", taus=(0, 32), warps=(4, 8), light=(8, 32), reps=1,
                                       pair_warps=(1, 4))
    assert len(trials) == 16 and best in trials
    assert {t["pair_warps"] for t in trials} == {1, 4}
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(9, 9), 16, 0, 8, 512)
    best, trials = autotune.tune_batch(g, ["triangle", "clique4"] * 8, off, pool, taus=(8,), warps=(8,),
                                       light=(16, 32), reps=1)
    assert len(trials) == 2
