"""CPU checks of the benchmark's measurement helpers: the clock-sample parser
that reports throttle reasons beside the number, and the FP32-local error
summary.  The GPU work of the benchmark itself runs only on a GPU."""
import importlib.util
import os

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_max_and_reasons(tmp_path):
    B = _bench()
    path = tmp_path / "clocks.csv"
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    path.write_text("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    s = B.ClockSampler(0)
    s.proc, s.path = _Done(), str(path)
    out = s.stop()
    assert out["sm_mhz"] == 2040.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not path.exists()


def test_clock_samples_report_thermal_and_hw_slowdown(tmp_path):
    B = _bench()
    path = tmp_path / "clocks.csv"
    path.write_text("0, 1500, 2070, 800.0, 0x48, Active, Not Active, Active, Not Active\n")
    s = B.ClockSampler(0)
    s.proc, s.path = _Done(), str(path)
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    B = _bench()
    s = B.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_tally_error_summary():
    B = _bench()
    t64 = torch.tensor([100, 200, 0, 400], dtype=torch.int64)
    t32 = torch.tensor([101, 198, 3, 400], dtype=torch.int64)
    c64 = np.zeros(16, np.uint64)
    c32 = np.zeros(16, np.uint64)
    c64[0], c32[0], c32[10] = 1000, 1002, 50
    e = B.tally_error(t32, t64, c32, c64)
    assert abs(e["tally_l1_rel"] - 6.0 / 700.0) < 1e-15
    assert abs(e["tally_linf_rel"] - 0.01) < 1e-15
    assert e["bins"] == 4 and e["bins_only_fp32"] == 1
    assert abs(e["segments_rel_diff"] - 0.002) < 1e-15 and abs(e["close_call_fraction"] - 50 / 1002) < 1e-15
    # a list of per-geometry tallies is summarised as one concatenated tally
    assert B.tally_error([t32, t32], [t64, t64])["tally_l1_rel"] == e["tally_l1_rel"]
    assert B._guarded(lambda: 1 / 0) == {"error": "ZeroDivisionError: division by zero"}


def test_cpu_baseline_compares_traced_rows_under_the_near_surface_rule():
    # rows equal to the oracle's own traces all match; a planted length
    # error in one row is reported as a failure, not hidden
    import oracle as O
    from paper_2406_13849_gb300 import inputs as I
    B = _bench()
    desc = I.to_json(I.small_core())
    o = O.Geometry(desc, O.MODE_CSG)
    ids, cap = np.arange(5, 25), 64
    rows_i = np.full((len(ids), cap), -1, np.int32)
    rows_l = np.zeros((len(ids), cap))
    for r, pid in enumerate(ids):
        inst, ln, kind, st = o.trace(int(pid), B.SEED, B.P_ABSORB, cap=cap)
        rows_i[r, :len(inst)] = inst
        rows_l[r, :len(ln)] = ln
    out = B.cpu_baseline(desc, 2000, 500, traced=(ids, rows_i, rows_l, cap))
    rule = out["near_surface_rule"]
    assert rule["compared"] == len(ids) and rule["matched"] == len(ids) and rule["failed"] == 0
    rows_l[3, 2] += 1e-6
    rule = B.cpu_baseline(desc, 2000, 500, traced=(ids, rows_i, rows_l, cap))["near_surface_rule"]
    assert rule["failed"] == 1 and rule["findings"][0]["pid"] == int(ids[3])


def test_roofline_numerators_match_the_counting_oracle():
    # the operation counts bench.py states are what oracle.flop_counts
    # computes (same samples), so a change of the oracle's arithmetic or of
    # the workloads shows up here
    bench = _bench()
    from oracle import flop_counts as F
    from paper_2406_13849_gb300 import inputs as I
    c2, _ = F.per_segment(I.config2(), 2000)
    assert c2 == bench.OPS_PER_SEGMENT
    assert F.batch_per_segment(200)["rect"] == bench.OPS_PER_SEGMENT_BATCH
    assert F.transmission_per_ray(512) == bench.OPS_PER_RAY_TRANSMISSION
