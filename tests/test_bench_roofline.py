"""The roofline entry bench.py reports for the headline step, on CPU from
synthetic kernel times: the algorithmic flops of the FP64 fine-solve
kernels (5 per row-step over the intervals still iterating), those of the
refined FP32 kernel (5 + 60 R per row-step), the peak each is held to, and
the per-launch DRAM traffic scaled from the captured per-system figure."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2508_08873_gb300 import workloads as W  # noqa: E402


def _kern(ms_f64, ms_f32, launches_f64=35):
    return {"propagate_f64": (launches_f64 * 2, ms_f64 * 2),
            "propagate_f32": (4, ms_f32 * 2)}


@pytest.mark.parametrize("rounds", [0, 1, 2])
def test_fine_roofline_accounting(rounds):
    P = W.adr1d()
    k = 29                                     # iterations of the solve
    kern = _kern(22.5 if rounds == 0 else 13.6, 1.3)
    roof = bench.fine_roofline(P, kern, [k, k], 27.4, 2, rounds)
    systems = P.N * k - k * (k - 1) / 2        # intervals still iterating, summed over the solve
    per_row = 5.0 if rounds == 0 else 5.0 + 60.0 * rounds
    flops = per_row * P.n * P.M * systems
    ms = (22.5 if rounds == 0 else 13.6)
    assert roof["achieved"] == pytest.approx(flops / (ms * 1e-3) / 1e12)
    peak = (bench.FP64_PEAK_GFLOPS if rounds == 0 else bench.FP32_PEAK_GFLOPS) / 1e3
    assert roof["peak"] == pytest.approx(peak)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak)
    assert roof["flops_per_row_step"] == per_row
    # one propagating launch per iteration; the rest return at once
    assert roof["systems_per_launch"] == pytest.approx(systems / k)
    assert roof["noop_launches_per_step"] == pytest.approx(35 - k)
    per_sys = bench.F64_DRAM_BYTES_PER_SYSTEM if rounds == 0 else bench.IRT_DRAM_BYTES_PER_SYSTEM
    assert roof["traffic"] == pytest.approx(per_sys * systems / k)
    assert roof["share_of_step"] == pytest.approx(ms / 27.4)


def test_fine_roofline_picks_the_dominant_family():
    """When the FP32 sketches dominate (a build-heavy step), the entry is the
    FP32 family's, against the FP32 peak, with no traffic figure."""
    P = W.adr1d()
    roof = bench.fine_roofline(P, _kern(0.5, 9.0), [3, 3], 12.0, 2, 0)
    assert roof["kernel"] == "propagate_f32"
    assert roof["peak"] == pytest.approx(bench.FP32_PEAK_GFLOPS / 1e3)
    assert roof["traffic"] is None
    assert roof["systems_per_launch"] == pytest.approx(2 * P.N * (P.R + P.p) / 2)
