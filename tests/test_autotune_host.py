"""Host logic of the batch tuner (paper_2310_17790_gb300.autotune): the batch
signature, the candidate list and the JSON cache.  No GPU: fake batch entries
carry only what the signature reads."""

import json

import pytest

torch = pytest.importorskip("torch")

from paper_2310_17790_gb300 import autotune  # noqa: E402


class _F:
    def __init__(self, r, width, depth):
        self.r, self.width, self.depth = r, (width, width, width), (depth, depth, depth)


def _entries(specs):
    out = []
    for r, w, d, n_N, n_S in specs:
        X = torch.zeros(3, n_N)
        out.append((_F(r, w, d), X, n_S, 1.0, 1.0, None, 1e-3, torch.zeros(r), torch.zeros(r)))
    return out


def test_signature_groups_batches_of_the_same_shape():
    a = _entries([(6, 128, 5, 1000, 50), (12, 64, 4, 3000, 150)])
    b = _entries([(12, 64, 4, 2900, 151), (6, 128, 5, 1100, 49)])     # same mix, same magnitudes
    c = _entries([(6, 128, 5, 1000, 50), (16, 64, 4, 3000, 150)])     # another r
    d = _entries([(6, 128, 5, 9000, 50), (12, 64, 4, 30000, 150)])    # 10x the particles
    assert autotune.batch_signature(a) == autotune.batch_signature(b)
    assert autotune.batch_signature(a) != autotune.batch_signature(c)
    assert autotune.batch_signature(a) != autotune.batch_signature(d)


def test_candidates_cover_every_choice_of_the_library():
    c = autotune.default_candidates()
    assert {x["gn_columns"] for x in c} == {32, 64}
    assert {x["p2g_group"] for x in c} == {64, 128}
    assert 0.0 in {x["gn_split"] for x in c}
    assert len({json.dumps(x, sort_keys=True) for x in c}) == len(c)


def test_cache_round_trip_and_tuning_for_uses_the_cache(tmp_path, monkeypatch):
    path = str(tmp_path / "tuning.json")
    e = _entries([(6, 128, 5, 1000, 50)])
    cache = autotune.TuningCache(path)
    assert cache.get(e) is None
    best = {"gn_columns": 32, "gn_split": 1.5, "p2g_group": 128}
    cache.put(e, best, 1.25)
    again = autotune.TuningCache(path)
    assert again.get(e) == best
    assert json.load(open(path))[autotune.batch_signature(e)]["ms_per_step"] == 1.25

    calls = []
    monkeypatch.setattr(autotune, "tune_batch", lambda *a, **k: calls.append(1) or (best, 2.0, []))
    assert again.tuning_for(e) == best and not calls          # cached: no timing
    other = _entries([(16, 64, 4, 5000, 250)])
    assert again.tuning_for(other) == best and calls == [1]   # not cached: timed once
    assert autotune.TuningCache(path).get(other) == best
