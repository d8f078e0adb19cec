"""Host logic of the tuned library variants (build.py, autotune.py): tags,
paths and the tuning table's choices, without compiling anything."""
import json
import os

from paper_1806_03761_gb300 import autotune, build as B


def test_variant_tags_name_the_changed_knobs():
    assert B.variant_tag(dict(B.DEFAULTS), "mixed") == "default"
    k = dict(B.DEFAULTS, PEPS_QR_NB=8)
    assert B.variant_tag(k, "mixed") == "mixed-PEPS_QR_NB8"
    k = dict(B.DEFAULTS, PEPS_MINB=1, PEPS_NT=512)
    assert B.variant_tag(k, "fp64") == "fp64-PEPS_MINB1-PEPS_NT512"
    assert B.variant_path(dict(B.DEFAULTS), "mixed") == B.LIB
    assert B.variant_path(k, "fp64").endswith(os.path.join("fp64-PEPS_MINB1-PEPS_NT512", "libpeps.so"))


def test_candidates_start_from_the_default_and_change_one_thing():
    cands = [autotune.knobs_of(d) for d in autotune.CANDIDATES]
    assert cands[0] == B.DEFAULTS
    tags = [B.variant_tag(k, "mixed") for k in cands]
    assert len(set(tags)) == len(tags)
    for k in cands:
        assert set(k) == set(B.DEFAULTS)


def test_tuning_table_choices(tmp_path, monkeypatch):
    table = {"16x16_D6_Dc24_mixed": {"precision": "mixed", "choice": dict(B.DEFAULTS, PEPS_QR_NB=2),
                                     "samples_per_s": {"default": 1.0}}}
    p = tmp_path / "tuning.json"
    p.write_text(json.dumps(table))
    monkeypatch.setattr(B, "TUNING", str(p))
    (knobs, prec), = B.tuned_variants()
    assert prec == "mixed" and knobs["PEPS_QR_NB"] == 2
