"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic summary
written from an ncu CSV, the source hash it is keyed to, and the summary of the
clock samples taken during the timed region."""
import csv
import io
import json
import os
import shutil

import bench


def _ncu_csv(path):
    # two searches' worth of launches in the shape ncu --csv writes (one row per metric)
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
           "Metric Unit", "Metric Value"]
    seq = [("tms::k_search_init(tms::Bounds *)", 0.0, 0.0),
           ("void tms::k_bounds_pass<1, 1, 4>(tms::FacePassArgs)", 134.4, 205.8),
           ("tms::k_grid_params(tms::GridArgs)", 0.0, 0.0),
           ("void tms::k_cell_pass<1, 1>(tms::FacePassArgs, int)", 69.1, 0.0),
           ("void tms::k_cell_pass<1, 2>(tms::FacePassArgs, int)", 81.4, 9.6),
           ("void tms::k_cell_pass<1, 3>(tms::FacePassArgs, int)", 82.0, 13.3),
           ("tms::k_group_count(tms::GroupArgs)", 70.8, 18.6),
           ("tms::k_cells_reduce(tms::GroupArgs)", 8.4, 0.0),
           ("tms::k_cells_partials(tms::GroupArgs, int)", 0.0, 0.0),
           ("tms::k_cells_down(tms::GroupArgs)", 16.1, 0.0),
           ("tms::k_group_scatter(tms::GroupArgs)", 95.8, 7.1),
           ("void tms::k_emit<1, 0>(tms::EmitArgs, int)", 232.0, 17.4),
           ("void tms::k_narrow_filter<1>(tms::NarrowArgs)", 82.3, 0.2),
           ("tms::k_narrow_fp64(tms::NarrowArgs)", 25.1, 0.0),
           ("tms::k_radix_pass(tms::RadixArgs)", 0.2, 0.0)]
    rows, i = [hdr], 0
    for _ in range(2):
        for name, rd, wr in seq + [("void at::vectorized_elementwise_kernel<4>(int)", 0.0, 268.4)]:
            for metric, unit, val in (("dram__bytes_read.sum", "Mbyte", rd),
                                      ("dram__bytes_write.sum", "Mbyte", wr),
                                      ("gpu__time_duration.sum", "usecond", 10.0)):
                rows.append([str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(1, 1, 1)",
                             "0", "10.3", "Command line profiler metrics", metric, unit, f"{val:,.2f}"])
            i += 1
    rows.append([str(i), "1", "python", "h", "tms::k_search_init(tms::Bounds *)", "1", "7", "", "",
                 "0", "10.3", "", "dram__bytes_read.sum", "byte", "0"])
    with open(path, "w", newline="") as f:
        f.write('==PROF== Connected to process 1\n')
        csv.writer(f).writerows(rows)


def test_write_traffic_takes_the_last_complete_search(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    shutil.copytree(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                 "paper_2109_14814_gb300", "csrc"),
                    tmp_path / "paper_2109_14814_gb300" / "csrc")
    _ncu_csv(tmp_path / "t.csv")
    out = bench.write_traffic(str(tmp_path / "t.csv"))
    saved = json.load(open(prof / "traffic.json"))
    assert saved == json.loads(json.dumps(out))
    assert abs(out["tms::k_bounds_pass"]["dram_bytes_per_launch"] - 340.2e6) < 1.0
    # two launches in the probe stage: per-launch average
    assert abs(out["tms::k_cell_pass<PROBE_MARK, PROBE>"]["dram_bytes_per_launch"] - 93.15e6) < 1.0
    # four launches in the cells + scatter stage
    assert abs(out["tms::k_cells_* + k_group_scatter"]["dram_bytes_per_launch"] - 127.4e6 / 4) < 1.0
    assert set(out["tms::k_narrow_filter + k_narrow_fp64"]["kernels"]) == {"k_narrow_filter<1>",
                                                                           "k_narrow_fp64"}
    # torch's L2-flush fill is not a stage; every entry carries the source hash
    assert all(v["source_hash"] == bench.source_hash() for v in out.values())
    assert bench.committed_traffic("tms::k_emit") == out["tms::k_emit"]["dram_bytes_per_launch"]


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
