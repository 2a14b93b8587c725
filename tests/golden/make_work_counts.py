"""Write tests/golden/work_counts.json: the work the method does per frame on
each workload, tallied by the oracle's counting build (oracle/op_count.cpp --
the FP64 oracle compiled with counting doubles), not by the CUDA path.

Per frame: arithmetic by class (add/sub, mul, div, sqrt, elementary
functions, comparisons, other), table texels read (D, U, C, disc), cube-map
records read, and the unique cube-map records the frame touches (all and
occupied).  These are the algorithmic units of the render kernel's roofline.
Run from the repository root:  python tests/golden/make_work_counts.py
"""
from __future__ import annotations

import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2010_08735_gb300 import synth  # noqa: E402

EXPOSURE_STARS = 0.01


def counts_for(name: str, D, U, Ct, dl) -> dict:
    wk = synth.WORKLOADS[name]
    dt = 1 if wk["cube_dtype"] == "f16" else 2
    st = synth.stars(wk["n_stars"], wk["star_seed"])
    rec = oracle.build_cubemap(st, wk["cube_n"], dt)
    scene = oracle.SceneTables(D.astype(np.float32), U.astype(np.float32), Ct.astype(np.float32),
                               dl.astype(np.float32), rec, wk["cube_n"], dt)
    t = time.time()
    _, c = oracle.count_render(wk["camera"], wk["disc"], scene, exposure_stars=EXPOSURE_STARS)
    c["seconds"] = round(time.time() - t, 2)
    return c


def main(names=("static_256", "orbit_1080p", "infall_4k")) -> None:
    D, U = oracle.tables_exact(512, 64, 32, 1e-3)
    Ct, dl = oracle.colour_table(), oracle.disc_colour_table()
    out = {"_source": "oracle counting build (oracle/op_count.cpp) over the full frame of each workload; "
                      "written by tests/golden/make_work_counts.py",
           "_classes": list(oracle.COUNT_CLASSES)}
    for n in names:
        out[n] = counts_for(n, D, U, Ct, dl)
        print(n, {k: v for k, v in out[n].items()}, flush=True)
    path = Path(__file__).with_name("work_counts.json")
    path.write_text(json.dumps(out, indent=1) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ("static_256", "orbit_1080p", "infall_4k"))
