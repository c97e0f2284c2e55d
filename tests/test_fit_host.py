"""Host logic of the batched fitter's autotuner (no GPU): which tile map
the timings select."""
import os

import pytest

from paper_2203_06139_gb300 import _build, cg
from paper_2203_06139_gb300.fit import pick_map


def M(w, c, t, k):
    return {"warp_max_bins": w, "cta_max_bins": c, "cta_threads": t, "cluster_size": k}


def test_pick_map_prefers_smaller_clusters_among_near_ties():
    timings = [(50.91, M(512, 4096, 128, 8)), (50.93, M(1024, 16384, 256, 4)), (51.15, M(2048, 16383, 256, 2)),
               (60.0, M(2048, 1 << 30, 256, 1))]
    assert pick_map(timings) == M(2048, 16383, 256, 2)


def test_pick_map_keeps_a_clearly_faster_map():
    timings = [(45.0, M(512, 4096, 128, 8)), (50.0, M(2048, 16383, 256, 2)), (50.2, M(2048, 1 << 30, 256, 1))]
    assert pick_map(timings) == M(512, 4096, 128, 8)


def test_pick_map_ties_on_cluster_size_go_to_larger_ctas_then_time():
    timings = [(50.0, M(2048, 16383, 128, 2)), (50.5, M(2048, 32767, 256, 2)), (50.4, M(2048, 16383, 256, 2))]
    assert pick_map(timings) == M(2048, 16383, 256, 2)
    assert pick_map(timings[:1]) == timings[0][1]


def test_pick_map_without_timings_raises():
    with pytest.raises(cg.CgError):
        pick_map([])


def test_generated_kernels_get_the_fp64_header_verbatim(tmp_path, monkeypatch):
    """The text handed to NVRTC as cg_fp64.cuh is the file itself, as one C
    raw string (written into the build directory by the build)."""
    monkeypatch.setattr(_build, "BUILD", str(tmp_path))
    _build.write_fp64_text()
    inc = open(os.path.join(str(tmp_path), "cg_fp64_text.inc")).read()
    head = 'static const char kCgFp64Text[] = R"CGFP64TEXT('
    body = inc[inc.index(head) + len(head):inc.rindex(')CGFP64TEXT";')]
    assert body == open(os.path.join(_build.CSRC, "cg_fp64.cuh")).read()
