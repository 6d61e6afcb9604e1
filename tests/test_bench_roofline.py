"""The benchmark's roofline arithmetic, reproduced by hand from its inputs: the
per-unit FP32 work (per radial neighbour entry 12 + 4 K_r forward and 20 + 6 K_r
backward, per unordered angular pair 10 + 4 K_a and 40 + 6 K_a, per atom
2 sum n_l n_{l-1} per network pass), the unit counts of the launch, the
event-timed launch duration and the FP32 FMA peak."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2107_11311_gb300 import inputs  # noqa: E402


def test_fused_roofline_by_hand():
    m = inputs.make_model("water", hidden=(32, 32))
    n = 331776
    entries, pairs = 28_000_000, 110_000_000
    form = {"stats": (entries, 9_000_000, pairs), "fused": True, "precision": "fp32",
            "stage_ms": {"forces": 2.0, "descriptor": None}}
    props = SimpleNamespace(multi_processor_count=152)
    rl = bench.roofline_of(form, m, n, props, 2070.0, "measured", "water_331776")
    Kr, Ka = 17, 9
    by_hand = (entries * ((12 + 4 * Kr) + (20 + 6 * Kr)) + pairs * ((10 + 4 * Ka) + (40 + 6 * Ka))
               + n * 2 * 2 * (52 * 32 + 32 * 32 + 32 * 1))
    assert rl["flops_per_launch"] == by_hand
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert abs(rl["peak"] - peak) < 1e-9
    assert abs(rl["achieved"] - by_hand / 2.0e-3 / 1e12) < 1e-9
    assert abs(rl["frac"] - by_hand / 2.0e-3 / 1e12 / peak) < 1e-12
    assert rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["kernel"].startswith("k_potential ")
    # the list form: the same algorithmic flops, charged to the list-driven kernel
    rl2 = bench.roofline_of(dict(form, list=True), m, n, props, 2070.0, "measured", "water_331776")
    assert rl2["flops_per_launch"] == by_hand and rl2["kernel"].startswith("k_potential_list ")


def test_split_form_roofline_takes_the_slower_kernel():
    m = inputs.make_model("water")
    form = {"stats": (1000, 300, 4000), "fused": False, "precision": "bf16x3",
            "stage_ms": {"descriptor": 0.5, "network": 0.1, "forces": 0.8}}
    rl = bench.roofline_of(form, m, 100, SimpleNamespace(multi_processor_count=152), 2070.0, "measured", "x")
    assert rl["flops_per_launch"] == 1000 * (20 + 6 * 17) + 4000 * (40 + 6 * 9)
    assert rl["launch_ms"] == 0.8 and rl["traffic"] is None
