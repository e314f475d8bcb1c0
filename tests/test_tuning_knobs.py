"""Host logic of the autotuner's hand-off to the build: tuning.json -> compile definitions."""
import json

from paper_2307_06345_gb300 import _build


def test_tuned_knobs_mapping(tmp_path, monkeypatch):
    doc = {"choice": {"sort": {"threads": 256, "items": 14, "min_blocks": 3},
                      "leaves": {"items": 12}}}
    p = tmp_path / "tuning.json"
    p.write_text(json.dumps(doc))
    monkeypatch.setattr(_build, "TUNING", str(p))
    assert _build.tuned_knobs() == {"CSTONE_SORT_THREADS": 256, "CSTONE_SORT_ITEMS": 14, "CSTONE_SORT_MIN_BLOCKS": 3,
                                    "CSTONE_LEAVES_ITEMS": 12}
    flags = _build._flags(_build.tuned_knobs())
    assert "-DCSTONE_SORT_ITEMS=14" in flags and "-DCSTONE_LEAVES_ITEMS=12" in flags
    assert "arch=compute_103a,code=sm_103a" in flags


def test_no_tuning_file_means_source_defaults(tmp_path, monkeypatch):
    monkeypatch.setattr(_build, "TUNING", str(tmp_path / "absent.json"))
    assert _build.tuned_knobs() == {}


def test_partial_choice(tmp_path, monkeypatch):
    p = tmp_path / "tuning.json"
    p.write_text(json.dumps({"choice": {"leaves": {"items": 4}}}))
    monkeypatch.setattr(_build, "TUNING", str(p))
    assert _build.tuned_knobs() == {"CSTONE_LEAVES_ITEMS": 4}
