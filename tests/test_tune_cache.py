"""Host logic of the batched-plan autotuning cache (JSON file keyed by GPU name
and a signature of the request); no GPU needed."""
import json
import os

from paper_1603_08081_gb300 import tune_cache as TC

SPECS = [dict(sigma_s=3.0, sigma_r=30.0), dict(sigma_s=6.5, sigma_r=12.0, eps=1e-2)]
SHAPES = [(300, 260), (70, 90)]


def test_signature_covers_what_the_schedules_depend_on():
    base = TC.signature("tc_fp16_single", "reflect", SHAPES, [True, True], SPECS)
    # dict order and explicit defaults do not matter
    again = TC.signature("tc_fp16_single", "reflect", SHAPES, [True, True],
                         [dict(sigma_r=30.0, sigma_s=3.0, W=0, T=255.0), dict(eps=1e-2, sigma_r=12.0, sigma_s=6.5)])
    assert base == again and len(base) == 64
    changed = [
        TC.signature("tc_fp16", "reflect", SHAPES, [True, True], SPECS),
        TC.signature("tc_fp16_single", "truncate", SHAPES, [True, True], SPECS),
        TC.signature("tc_fp16_single", "reflect", [(300, 261), (70, 90)], [True, True], SPECS),
        TC.signature("tc_fp16_single", "reflect", SHAPES, [True, False], SPECS),
        TC.signature("tc_fp16_single", "reflect", SHAPES, [True, True], [SPECS[0], dict(SPECS[1], sigma_r=12.5)]),
        TC.signature("tc_fp16_single", "reflect", SHAPES, [True, True], [SPECS[0], dict(SPECS[1], W=7)]),
        TC.signature("tc_fp16_single", "reflect", SHAPES[::-1], [True, True], SPECS[::-1]),
        TC.signature("tc_fp16_single", "reflect", SHAPES[:1], [True], SPECS[:1]),
    ]
    assert len(set(changed + [base])) == len(changed) + 1


def test_record_and_lookup_per_gpu(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert TC.lookup(path, "GPU A", "s1") is None  # no file yet
    TC.record(path, "GPU A", "s1", {"schedule": "persistent_tc", "ms": 6.4})
    TC.record(path, "GPU B", "s1", {"schedule": "per_image_form_streams", "ms": 7.0})
    TC.record(path, "GPU A", "s2", {"schedule": "per_image_form", "ms": 1.0})
    assert TC.lookup(path, "GPU A", "s1")["schedule"] == "persistent_tc"
    assert TC.lookup(path, "GPU B", "s1")["schedule"] == "per_image_form_streams"
    assert TC.lookup(path, "GPU B", "s2") is None
    TC.record(path, "GPU A", "s1", {"schedule": "per_image_form", "ms": 5.0})  # replaced
    assert TC.lookup(path, "GPU A", "s1")["ms"] == 5.0
    d = json.load(open(path))
    assert d["version"] == TC.VERSION and set(d["entries"]) == {"GPU A", "GPU B"}
    assert sorted(os.listdir(tmp_path / "sub")) == ["tune.json"]  # no temporary file left


def test_unreadable_or_foreign_files_are_treated_as_empty(tmp_path):
    path = str(tmp_path / "tune.json")
    for content in ("{not json", json.dumps({"version": TC.VERSION + 1, "entries": {"G": {"s": {"schedule": "x"}}}}),
                    json.dumps([1, 2]), json.dumps({"version": TC.VERSION, "entries": {"G": {"s": {"ms": 1}}}})):
        with open(path, "w") as fh:
            fh.write(content)
        assert TC.lookup(path, "G", "s") is None
    TC.record(path, "G", "s", {"schedule": "persistent"})
    assert TC.lookup(path, "G", "s")["schedule"] == "persistent"
