"""The benchmark's byte accounting and the summary it prints early in its line, on CPU.

The roofline fractions are algorithmic bytes over event-timed durations, so the byte counts are
checked here against their stated definitions: a tracking step's nominal per-access bytes are 40 B
per pixel (4 B depth, 20 B payload, 16 B hash slot; FP16 30 B, dense 24 B), its usable-pixel count
4 B per pixel plus key and payload per usable pixel, and fusion 4 B per pixel plus 48 B per
ray-voxel update.  The summary must carry every fraction the forms report.
"""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_nominal_tracking_bytes_per_pixel():
    assert bench.track_bytes_nominal("f32", 307200) == 40 * 307200
    assert bench.track_bytes_nominal("f16", 1000) == 30 * 1000
    assert bench.track_bytes_nominal("dense", 1000) == 24 * 1000


def test_usable_pixel_and_compulsory_bytes():
    # per access: 4 B per pixel + (8 B key + 20 B payload) per usable pixel
    assert bench.track_bytes("f32", 100, 60) == 4 * 100 + 28 * 60
    assert bench.track_bytes("dense", 100, 60) == 4 * 100 + 20 * 60
    # compulsory: each distinct voxel's payload and block's key once
    assert bench.track_bytes("f32", 100, 0, 10, 2) == 4 * 100 + 20 * 10 + 8 * 2
    # fusion per access: 48 B per visit; compulsory: payload read and written once per voxel
    assert bench.fuse_bytes("f32", 100, 7) == 4 * 100 + 48 * 7
    assert bench.fuse_bytes("f32", 100, 0, 10, 2) == 4 * 100 + 40 * 10 + 8 * 2


def test_roof_fraction():
    r = bench.roof(6.0e9, 1e-3, 6000.0)
    assert math.isclose(r["GBs"], 6000.0) and math.isclose(r["frac"], 1.0)


def _split(track_frac, fusion_frac):
    rf = lambda f: {"GBs": f * 6772.9, "frac": f}  # noqa: E731
    return {"track": {"per_access": rf(track_frac), "per_access_usable": rf(track_frac * 0.8),
                      "compulsory": rf(0.08)},
            "fusion": {"per_access": rf(fusion_frac), "compulsory": rf(0.03)}}


def test_forms_summary_carries_every_fraction():
    acc = {"max_in_voxels": 1.8}
    batch = {"value": 4.4e10, "fp16_value": 3.8e10, "plain_value": 1.05e10, "ms_per_frame": 2.1,
             "speedup_vs_plain": 4.2, "fp16_speedup_vs_plain": 3.6,
             "pose_accuracy": {"batched": acc, "batched_fp16": acc, "plain": acc,
                               "gate_all_scenes_within_2_voxels": True},
             "split": {"batched": _split(0.62, 0.70), "batched_fp16": _split(0.45, 0.55)}}
    out = bench.forms_summary({"batched_64_scenes": batch})["batched_64_scenes"]
    assert out["accuracy_gate"] is True
    t = out["hbm_frac"]["batched"]["track"]
    assert t["per_access"] == 0.62 and math.isclose(t["per_access_usable"], 0.496) and t["compulsory"] == 0.08
    f = out["hbm_frac"]["batched_fp16"]["fusion"]
    assert f == {"per_access": 0.55, "compulsory": 0.03}
