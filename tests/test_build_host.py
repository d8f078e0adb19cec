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


def test_committed_tuning_table_names_known_knobs():
    """Every choice in the committed tuning table sets only knobs build.py
    knows, within the values the kernels accept."""
    table = json.load(open(B.TUNING))
    assert table
    for key, entry in table.items():
        assert entry["precision"] in B.FORMS
        k = entry["choice"]
        assert set(k) <= set(B.DEFAULTS), key
        full = dict(B.DEFAULTS, **k)
        assert full["PEPS_NT"] % 64 == 0 and full["PEPS_MINB"] in (1, 2, 3, 4)
        assert full["PEPS_QR_NB"] in (2, 4, 8)
        # the tag reproduces the path build() makes for it
        assert B.variant_path(full, entry["precision"]).endswith("libpeps.so")


def test_build_makes_each_distinct_variant_once(monkeypatch):
    built = []
    monkeypatch.setattr(B, "build_default", lambda *a, **k: B.LIB)
    monkeypatch.setattr(B, "build_variant", lambda k, p, v=False: built.append(B.variant_tag(k, p)))
    monkeypatch.setattr(B, "tuned_variants",
                        lambda: [(dict(B.DEFAULTS, PEPS_MINB=3), "mixed")] * 2 +
                                [(dict(B.DEFAULTS, PEPS_QR_NB=8), "mixed")])
    assert B.build() == B.LIB
    assert sorted(built) == ["mixed-PEPS_MINB3", "mixed-PEPS_QR_NB8"]


def test_bench_library_tag():
    import bench

    class L:
        def __init__(self, name):
            self._name = name

    class C:
        def __init__(self, name):
            self.lib = L(name)

    assert bench.library_tag(C(B.LIB)) == "default"
    assert bench.library_tag(C(os.path.join(B.LIBDIR, "mixed-PEPS_MINB3", "libpeps.so"))) == "mixed-PEPS_MINB3"
