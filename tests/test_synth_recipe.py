"""The seeded input recipe against the shapes the paper prints (tests/golden)."""
import os

import numpy as np
import pytest

from paper_1903_01852_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ao_compare_shapes.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            out[k] = int(v)
    return out


def test_paper_scao_mvm_is_twice_the_valid_count():
    g = golden()
    assert g["scao_sh_mvm_cols"] == 2 * g["scao_sh_valid_subaps"]


def test_annulus_rule_reproduces_paper_count_within_half_percent():
    g = golden()
    n = int(synth.annulus_mask(g["scao_sh_subaps_across"], 0.28).sum())
    assert n == 4632 and abs(n - g["scao_sh_valid_subaps"]) / g["scao_sh_valid_subaps"] < 0.005


@pytest.mark.parametrize("name,nvalid", [("scao_small", [208]), ("elt_scao_sh", [4304]),
                                          ("elt_scao_pyramid", [6144])])
def test_valid_counts(name, nvalid):
    cfg = synth.make_config(name)
    assert [synth.num_valid(w) for w in cfg["wfs"]] == nvalid
    assert cfg["M"].shape == (cfg["na"], 2 * sum(nvalid))


def test_mcao_shapes_follow_table_ao_compare():
    g = golden()
    # build the geometry only (the 1.7 GB matrix is not needed here)
    rng = np.random.default_rng(0)
    lgs = synth.sh_wfs(rng, g["lgs_subaps_across"], g["lgs_pixels_per_subap"], g["lgs_image_side"],
                       g["lgs_image_side"], 0.28)
    ngs = synth.sh_wfs(rng, g["ngs_subaps_across"], g["ngs_pixels_per_subap"], g["ngs_image_side"],
                       g["ngs_image_side"], 0.28)
    ns = g["lgs_number"] * 2 * synth.num_valid(lgs) + g["ngs_number_mcao"] * 2 * synth.num_valid(ngs)
    assert ns == 55608
    assert lgs["nsubx"] * lgs["npx"] == g["lgs_image_side"]


def test_frames_are_seeded_uint16():
    cfg = synth.make_config("scao_small")
    f1 = synth.draw_frames(cfg, 2, seed=5)
    f2 = synth.draw_frames(cfg, 2, seed=5)
    assert f1[0][0].dtype == np.uint16 and f1[0][0].shape == (128, 128)
    assert all(np.array_equal(a[0], b[0]) for a, b in zip(f1, f2))
    assert not np.array_equal(f1[0][0], f1[1][0])


def test_chunk_plan_covers_frame_and_aligns_to_subaperture_rows():
    cfg = synth.make_config("elt_scao_sh")
    w = cfg["wfs"][0]
    plan = synth.chunk_plan(w, 8)
    assert len(plan) == 8 and plan[0][0] == 0 and plan[-1][1] == w["height"]
    assert all(a[1] == b[0] for a, b in zip(plan, plan[1:]))
    assert all((e - w["oy"]) % w["npx"] == 0 for _, e in plan[:-1])
