"""Host-side pieces of the benchmark contract (no GPU): defaults, mode numbering, the
algorithmic byte and operation models the rooflines divide by, and the DRAM-traffic lookup keyed
by kernel sources."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2504_05562_gb300 import stf  # noqa: E402


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_defaults_are_one_gpu_with_enough_warmup_and_steps():
    a = _args()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 100
    assert (a.width, a.height, a.tex, a.fmt, a.mode, a.filter) == (3840, 2160, 2048, "fp16", "wave3", "bilinear")


def test_mode_numbers_match_the_library():
    assert bench.MODES == {"full": stf.MODE_FULL, "one_tap": stf.MODE_ONE_TAP, "quad2": stf.MODE_QUAD2,
                           "wave2": stf.MODE_WAVE2, "wave3": stf.MODE_WAVE3, "wave4": stf.MODE_WAVE4}
    for name, m in bench.EXACT_MODES.items():
        assert m == bench.MODES[name[:-len("_exact")]] | stf.MODE_FLAG_EXACT


def test_algorithmic_bytes_of_the_4k_frame():
    # float4 output per pixel + (960 + 1) x (540 + 1) FP16 8-channel texels under the supports
    a = _args()
    assert bench.algorithmic_bytes(a) == 3840 * 2160 * 16 + 961 * 541 * 16 == 141028816


def test_operation_model_grows_with_the_footprint():
    one = bench.alg_ops_per_pixel("bilinear", "one_tap")
    counts = [bench.alg_ops_per_pixel("bilinear", m) for m in ("quad2", "wave3", "wave4")]
    assert one < counts[0] < counts[1] < counts[2]
    assert bench.alg_ops_per_pixel("bilinear", "wave3") == 342
    assert bench.alg_ops_per_pixel("bspline", "wave3") > 342
    # the issue peak: SMs x 4 sub-partitions x 32 lanes at the sampled clock
    assert abs(bench.alu_peak_ops(2070.0, 152) - 152 * 4 * 32 * 2070e6) < 1.0
    assert abs(bench.alu_peak_ops(1500.0, 148) - 148 * 4 * 32 * 1500e6) < 1.0


def test_traffic_entries_are_keyed_by_current_sources():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, e in t.items():
        kernel = key.split("/")[0]
        assert e["dram_bytes_per_launch"] > 0
        if e["src_hash"] == bench.src_hash(kernel):
            assert bench.load_traffic(key) == e["dram_bytes_per_launch"]
        else:
            assert bench.load_traffic(key) is None
