"""Host logic of bench.py on CPU: whole-job throughput, the roofline object of the dominant kernel
class, the version gate on stored ncu traffic, and the parsing of the nvidia-smi clock record
that decides whether a run was throttled."""
import json

import pytest

import bench


def test_whole_job_throughput():
    assert bench.aggregate(2000.0, 3, 2) == pytest.approx(3.0)      # 6 solves in 2 s
    assert bench.aggregate(500.0, 1, 1) == pytest.approx(2.0)


def test_peak_ratio_is_the_nominal_tf32_over_bf16():
    assert bench.TF32_OVER_BF16 == pytest.approx(1.1 / 2.25)


def test_roofline_of_a_tensor_bound_factorisation():
    """The update runs inside a seconds-long step: its peak is the sustained bf16 rate times the
    nominal tf32/bf16 ratio.  Every class with a work model gets its own object."""
    timings = {"lu_update": (800.0, 400), "apply": (300.0, 17), "spmv": (2.0, 17), "orth": (0.0, 0)}
    flops = 4.0e14
    dom, rs = bench.roofline(timings, flops, 8.0e10, 2, 6779.4, 1714.6, spmv=1.0e10)
    r = rs[dom]
    assert dom == "lu_update" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops * 2 / 0.8 / 1e12)
    assert r["peak"] == pytest.approx(1714.6 * 1.1 / 2.25)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert rs["apply"]["achieved"] == pytest.approx(8.0e10 * 17 / 0.3 / 1e9)
    assert rs["spmv"]["achieved"] == pytest.approx(1.0e10 / 0.002 / 1e9)
    assert rs["spmv"]["frac"] == pytest.approx(rs["spmv"]["achieved"] / 6779.4)


def test_roofline_of_an_hbm_bound_apply():
    timings = {"lu_update": (100.0, 50), "apply": (300.0, 20)}
    dom, rs = bench.roofline(timings, 1e13, 5.0e10, 1, 6779.4, 1714.6)
    r = rs[dom]
    assert dom == "apply" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(5.0e10 * 20 / 0.3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6779.4)
    assert "spmv" not in rs                   # no work model given


def test_roofline_of_fp64_factors_is_alu_bound():
    dom, rs = bench.roofline({"lu_update": (1000.0, 10)}, 1e12, 1.0, 1, 6779.4, 1714.6, factor_bits=64)
    r = rs[dom]
    assert dom == "lu_update" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(1.0) and r["peak"] == bench.FP64_NOMINAL_TFLOPS


def test_spmv_and_apply_byte_models():
    """SpMV: 20 B per stored entry (16 B values + 4 B column), 8 B row pointer per row, input
    8 B (FP32) or 16 B (FP64) and output 16 B per row and right-hand side.  Apply passes: groups
    of up to 4 right-hand sides with FP32 factors (2 with FP64); the sizes are the live columns."""
    assert bench.spmv_bytes(10, 100, 1, True) == 20 * 100 + 8 * 11 + 24 * 10
    assert bench.spmv_bytes(10, 100, 3, False) == 20 * 100 + 8 * 11 + 32 * 30
    assert bench.apply_group_sizes(32, 32) == [4] * 8
    assert bench.apply_group_sizes(7, 32) == [4, 3]         # the last pass: 3 live columns of 4
    assert bench.apply_group_sizes(3, 64) == [2, 1]
    assert bench.rhs_groups(20, 8) == [8, 8, 4]
    assert bench.apply_group_sizes(32, 32, True) == [32]
    assert bench.apply_group_sizes(40, 32, True) == [32, 8]
    assert bench.apply_group_sizes(12, 32, True) == [12]
    assert bench.apply_group_sizes(4, 32, True) == [4]          # below 8 columns: CUDA-core groups


def test_stored_traffic_needs_the_current_kernel_version(tmp_path, monkeypatch):
    path = tmp_path / "traffic.json"
    entry = {"workload": "w", "lu_panel": 24, "bytes_per_launch": 123.0, "source_version": "old"}
    path.write_text(json.dumps({"k_lu_update_tc": entry}))
    monkeypatch.setattr(bench, "TRAFFIC", str(path))
    assert bench.measured_traffic("k_lu_update_tc", "w", 24) is None
    entry["source_version"] = bench.UPDATE_VERSION
    path.write_text(json.dumps({"k_lu_update_tc": entry}))
    assert bench.measured_traffic("k_lu_update_tc", "w", 24) == 123.0
    assert bench.measured_traffic("k_lu_update_tc", "w", 16) is None
    assert bench.measured_traffic("k_lu_update_tc", "other", 24) is None


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clock_summary(tmp_path, lines):
    s = bench.ClockSampler(0, str(tmp_path))
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = _DoneProcess()
    s.f = open(s.path)
    return s.stop()


def test_clock_record_without_throttling(tmp_path):
    rows = [f"0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
            for mhz in (2070, 2055, 2070, 1980, 2070)]
    c = _clock_summary(tmp_path, rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_clock_record_flags_every_throttle_reason(tmp_path):
    rows = ["0, 1800, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active",
            "garbage line",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = _clock_summary(tmp_path, rows)
    assert c["samples"] == 2 and c["sm_mhz"] == 1650.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


class _FakeLib:
    """Subdomain sizes only: (n_s, tets, padded order)."""

    def __init__(self, sizes):
        self.sizes = sizes

    def oras_subdomain_size(self, h, s):
        n = self.sizes[s]
        return n, 0, -(-n // bench.TB) * bench.TB


def test_work_model_closed_forms():
    sizes = [12749, 1000, 64, 8370]
    upd, apply_bytes = bench.work_model(_FakeLib(sizes), None, len(sizes), 3)
    tb = bench.TB
    closed = 0.0
    for n in sizes:
        nts = -(-n // tb)
        closed += 8.0 * tb ** 3 * (nts - 1) * nts * (2 * nts - 1) / 6.0   # 8 TB^3 sum_j j^2
    assert upd == pytest.approx(closed, rel=1e-12)
    # the trailing updates of a dense LU are (8/3) n^3 real flops to leading order
    big = bench.work_model(_FakeLib([12749]), None, 1, 1)[0]
    assert big == pytest.approx(8.0 / 3.0 * 12749 ** 3, rel=0.01)
    assert apply_bytes == pytest.approx(8.0 * sum(n * n for n in sizes) + 3 * 36.0 * sum(sizes))


def test_roofline_sums_panel_and_trailing_updates():
    """The panel updates (class lu_panel) and the trailing updates share one kernel and one flop
    model: their times add up for the update's achieved rate and for the dominant class."""
    timings = {"lu_update": (500.0, 20), "lu_panel": (300.0, 400), "apply": (700.0, 17)}
    dom, rs = bench.roofline(timings, 4e14, 1e9, 1, 6761.6, 1718.2)
    assert dom == "lu_update"
    assert abs(rs["lu_update"]["achieved"] - 4e14 / 0.8 / 1e12) < 1e-9
    assert "lu_panel" not in rs
