"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic summary
written from an ncu CSV, the source hash it is keyed to, and the summary of the
clock samples taken during the timed region."""
import csv
import io
import json
import os
import shutil

import bench


def _ncu_csv(path, name, launches):
    """One kernel's capture in the shape ncu --csv writes (one row per metric):
    `launches` is a list of (read MB, write MB)."""
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
           "Metric Unit", "Metric Value"]
    rows = [hdr]
    for i, (rd, wr) in enumerate(launches):
        for metric, unit, val in (("dram__bytes_read.sum", "Mbyte", rd),
                                  ("dram__bytes_write.sum", "Mbyte", wr),
                                  ("gpu__time_duration.sum", "usecond", 10.0)):
            rows.append([str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(1, 1, 1)",
                         "0", "10.3", "Command line profiler metrics", metric, unit, f"{val:,.2f}"])
    with open(path, "w", newline="") as f:
        f.write('==PROF== Connected to process 1\n')
        csv.writer(f).writerows(rows)


def test_write_traffic_sums_kernels_per_search_and_broad_phase(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    shutil.copytree(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                 "paper_2109_14814_gb300", "csrc"),
                    tmp_path / "paper_2109_14814_gb300" / "csrc")
    caps = tmp_path / "caps"
    caps.mkdir()
    idx = {rx: i for i, (rx, _, _, _) in enumerate(bench.TRAFFIC_KERNELS)}
    _ncu_csv(caps / f"traffic_{idx['k_bounds_pass']:02d}.csv", "void tms::k_bounds_pass<1, 1, 4>(x)",
             [(134.4, 205.8)])
    _ncu_csv(caps / f"traffic_{idx['k_cell_pass']:02d}.csv", "void tms::k_cell_pass<1, 1>(x)",
             [(1.0, 0.0), (2.0, 0.5), (3.0, 0.5)])
    _ncu_csv(caps / f"traffic_{idx['k_patch_quads']:02d}.csv", "void tms::k_patch_quads<1, 0>(x)",
             [(60.0, 13.6)])
    _ncu_csv(caps / f"traffic_{idx['k_narrow_filter']:02d}.csv", "void tms::k_narrow_filter<1>(x)",
             [(80.0, 1.0)])
    out = bench.write_traffic(str(caps))
    saved = json.load(open(prof / "traffic.json"))
    assert saved == json.loads(json.dumps(out))
    assert out["source_hash"] == bench.source_hash()
    assert abs(out["kernels"]["k_bounds_pass"]["dram_bytes_per_search"] - 340.2e6) < 1.0
    # a kernel launched three times per search: its launches summed
    assert out["kernels"]["k_cell_pass"]["launches"] == 3
    assert abs(out["kernels"]["k_cell_pass"]["dram_bytes_per_search"] - 7.0e6) < 1.0
    # the narrow phase is not in the broad phase's total
    assert abs(out["broad_dram_bytes_per_search"] - (340.2e6 + 7.0e6 + 73.6e6)) < 1.0
    assert bench.broad_traffic() == out["broad_dram_bytes_per_search"]
    assert bench.committed_traffic("tms::k_bounds_pass") == out["kernels"]["k_bounds_pass"][
        "dram_bytes_per_search"]
    # commands: one kernel, one to three launches, clocks left alone
    for c in bench.traffic_commands("d", "w.pt"):
        assert "--clock-control none" in c and " -k regex:^" in c
        assert int(c.split(" -c ")[1].split()[0]) in (1, 2, 3)


def test_source_hash_covers_only_the_search_sources():
    assert len(bench.SEARCH_SOURCES) == 7
    assert "tms_refine.cu" not in bench.SEARCH_SOURCES and "tms_faces.cu" in bench.SEARCH_SOURCES
    assert len(bench.source_hash()) == 16


def test_clock_summary_median_max_and_throttle_reasons(tmp_path):
    """The clock line the bench attaches: median SM clock under load, the
    maximum, and every throttle reason seen active at least once ("Not Active"
    is not active); malformed lines are skipped and the sample file removed."""
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "truncated line",
        "0, 1410, 2070, 700.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    ]
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    out = cs.summary()
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2025.0          # median of 2070, 1980, 2070, 1410
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not path.exists()
    # no sampler output at all (nvidia-smi missing): no clock figures, no reasons
    cs2 = bench.ClockSampler(0)
    cs2.path = str(tmp_path / "absent.csv")
    assert cs2.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
