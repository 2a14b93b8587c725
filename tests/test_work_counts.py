"""The per-frame work counts of the render (tests/golden/work_counts.json,
the roofline's algorithmic units) are current: recounted here by the
oracle's counting build, which must also render exactly the image of the
plain oracle build (the counting type changes no arithmetic).  No GPU."""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2010_08735_gb300 import synth

GOLDEN = json.loads((Path(__file__).parent / "golden" / "work_counts.json").read_text())


def scene_for(orc, exact_tables, colour_tables, name):
    wk = synth.WORKLOADS[name]
    D, U = exact_tables
    Ct, dl = colour_tables
    dt = 1 if wk["cube_dtype"] == "f16" else 2
    rec = orc.build_cubemap(synth.stars(wk["n_stars"], wk["star_seed"]), wk["cube_n"], dt)
    return orc.SceneTables(D.astype(np.float32), U.astype(np.float32), Ct.astype(np.float32),
                           dl.astype(np.float32), rec, wk["cube_n"], dt)


@pytest.mark.parametrize("name", ["static_256", "orbit_1080p"])
def test_work_counts_are_current(orc, exact_tables, colour_tables, name):
    wk = synth.WORKLOADS[name]
    scene = scene_for(orc, exact_tables, colour_tables, name)
    img, counts = orc.count_render(wk["camera"], wk["disc"], scene, exposure_stars=0.01)
    for k, v in GOLDEN[name].items():
        if k != "seconds":
            assert counts[k] == v, (k, counts[k], v)
    # the counting build renders what the plain oracle renders, bit for bit
    if name == "static_256":
        ref, _, _ = orc.render(wk["camera"], wk["disc"], scene, exposure_stars=0.01)
        assert np.array_equal(img, ref)


def test_work_counts_are_plausible():
    """Sanity of the tallies: every visited texel is one cube record read; the
    occupied unique records are a subset of the unique ones; the per-pixel
    arithmetic sits in the hundreds of operations."""
    for name in ("static_256", "orbit_1080p", "infall_4k"):
        c = GOLDEN[name]
        px = c["pixels"]
        assert c["unique_cube_records_occupied"] <= c["unique_cube_records"] <= c["fetch_cube"]
        assert 100 < (c["add"] + c["mul"]) / px < 2000
        assert c["fetch_D"] % 4 == 0 and c["fetch_U"] % 4 == 0 and c["fetch_C"] % 8 == 0
