"""Benchmark of the mesh-vs-mesh intersection search on GB300.

One step = one full search (every broad- and narrow-phase stage, merged and
sorted output, hit count read back) of the 4096 x 512 vs 4096 x 512 vertex
meshes (4,186,112 triangles each, 256 planted hits, 1e4 planted near-misses),
with the inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tms|reference]

For N > 1 (launched by torch.distributed.run) every rank searches its own
replica of the workload: the searches are independent units (weak scaling).
The reference arm times the CPU oracle (test infrastructure, exact pruning by a
bounding-volume hierarchy, OpenMP) on the host cores for the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "ms per full manifold-mesh search (4M×4M tris), HBM GB/s & FP64 util vs peak"
UNIT = "ms/search"
WORKLOAD = dict(workload="mesh-vs-mesh search, 4096x512 vs 4096x512 vertex grids "
                         "(4,186,112 triangles per mesh), lambda=4 stretch, 3 folds, "
                         "256 planted hits + 1e4 planted near-misses (1e-9..1e-3)",
                N=4096, M=512, triangles_per_mesh=4186112)
ENTRY_BYTES = 8 + 4                   # face-cell entry: u64 key, u32 face id
NOMINAL_SM_MAX_MHZ = 2070              # GB300 maximum SM clock
REF_MAX_STEPS = 10                     # timed oracle searches of the reference arm
# FP32 operations of one verified FP32 solve (an FMA counts 2): 20 system
# entries with error bounds (12 each), elimination on [A | I | r] (98), back
# substitution for five right-hand sides (80), the bound matrix W (32),
# alpha = |I - C A| + |C| W (337), the residual bound (112), the error bound
# (35) and the margin tests (22)
FP32_SOLVE_FLOPS = 956
# FP32 operations of the separating-axis prefilter with all four axes: five
# split difference vectors with bounds (80), two offset vectors (16), two sets
# of Plucker coordinates (56), the FP64 solve's reach (12), the two dual
# choices (28), four interval tests (260)
SAT_FLOPS = 452
# FP32 operations of the quad-level test every quad candidate takes: seven split
# difference vectors (112), the FP64 solve's reach (20), two mixed directions
# (4D cross products, 56 each) and their interval tests over eight vertices (90
# each).  The second stage, on the tenth or so of the candidates these leave
# (two more mixed directions and the dual axes), is not counted.
QUAD_SAT_FLOPS = 424
# FP32 lane operations per second of one GB300 (152 SMs x 128 lanes x 2070 MHz,
# an FMA counted 2)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64 operations of one narrow-phase solve of Eq. (precise) (an FMA counts 2):
# the 16 matrix entries and 4 right-hand-side entries (20), the squared column
# norms (28), elimination with partial pivoting (46) and back substitution
# (16); the 4 pivot reciprocals, the margin, the point, rho and the (theta, s)
# estimates are not counted
FP64_SOLVE_FLOPS = 110


# the broad phase's stages (tms_last_stage_ms labels), and per reported stage the
# labels it sums and its kernels (the keys of profiles/traffic.json)
BROAD_STAGES = ("init", "face_bounds", "grid_params", "bitmap_clear", "face_mark_A", "face_probe_B",
                "face_probe_A", "group_count", "group_cells", "emit", "patch_quads")
STAGE_PARTS = {
    "face_bounds": ("face_bounds",),
    "face_mark": ("face_mark_A",),
    "face_probe": ("face_probe_B", "face_probe_A"),
    "group_count": ("group_count",),
    "group_cells": ("group_cells",),
    "emit": ("emit", "patch_quads"),
    "narrow": ("narrow",),
    "sort_merge": ("sort_hits", "merge_output"),
}
STAGE_KERNELS = {
    "face_bounds": "tms::k_bounds_pass",
    "face_mark": "tms::k_cell_pass<MARK>",
    "face_probe": "tms::k_cell_pass<EMIT_ALL>",
    "group_count": "tms::k_group_count",
    "group_cells": "tms::k_cells_* + k_group_scatter",
    "emit": "tms::k_emit + k_patch_quarters + k_patch_quads",
    "narrow": "tms::k_quad_filter + k_narrow_filter + k_narrow_fp64",
    "sort_merge": "tms::k_radix_* + k_dedup_*",
}
BROAD_KERNELS = ("k_search_init", "k_bounds_pass", "k_grid_params", "k_cell_pass", "k_group_count",
                 "k_cells_reduce", "k_cells_partials", "k_cells_down", "k_group_scatter", "k_emit",
                 "k_patch_quarters", "k_patch_quads")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest `value` over all ranks of the process group (the job's time
    is its slowest rank's); `value` itself when there is no group."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_times(total_ms: float, steps: int, ws: int):
    """(ms per search over the whole job, ms per step) from the slowest rank's
    time for `steps` steps; each rank searches one replica per step, so the job
    completes steps * ws searches in total_ms."""
    return total_ms / (steps * ws), total_ms / steps


def _traffic_table():
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        return t if t.get("source_hash") == source_hash() else None
    except (OSError, ValueError):
        return None


def committed_traffic(label: str):
    """DRAM bytes per search of a reported stage (STAGE_KERNELS label) from the
    committed ncu summary (profiles/traffic.json), or None when absent or taken
    on other sources."""
    t = _traffic_table()
    if not t:
        return None
    st = t.get("stages", {}).get(label)
    return st.get("dram_bytes_per_search") if st else None


def broad_traffic():
    """ncu DRAM bytes of the broad phase's kernels per search, or None."""
    t = _traffic_table()
    return t.get("broad_dram_bytes_per_search") if t else None


# One ncu capture per kernel (the pool's rule for counters beyond the launch
# list: one kernel, one to three launches), on the bench workload (about 1 GB on
# the device, inputs larger than L2), after three warm-up searches.  Per kernel:
# (regex, launches per search, stage label, in the broad phase).
TRAFFIC_KERNELS = [
    ("k_search_init", 1, None, True),
    ("k_bounds_pass", 1, "face_bounds", True),
    ("k_grid_params", 1, None, True),
    ("k_cell_pass", 1, "face_probe", True),
    ("k_group_count", 1, "group_count", True),
    ("k_cells_reduce", 1, "group_cells", True),
    ("k_cells_partials", 1, "group_cells", True),
    ("k_cells_down", 1, "group_cells", True),
    ("k_group_scatter", 1, "group_cells", True),
    ("k_emit", 1, "emit", True),
    ("k_patch_quarters", 1, "emit", True),
    ("k_patch_quads", 1, "emit", True),
    ("k_quad_filter", 1, "narrow", False),
    ("k_narrow_filter", 1, "narrow", False),
    ("k_narrow_fp64", 1, "narrow", False),
]
TRAFFIC_METRICS = "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum"
TRAFFIC_BENCH = "python bench.py --steps 1 --warmup 3 --no-e2e --no-cpu --workload-cache {cache}"


def traffic_commands(out_dir: str, cache: str):
    """The ncu command of each TRAFFIC_KERNELS entry (CSV into out_dir)."""
    cmds = []
    for i, (rx, per, _, _) in enumerate(TRAFFIC_KERNELS):
        cmds.append(f"ncu --metrics {TRAFFIC_METRICS} --clock-control none -k regex:^{rx} "
                    f"-s {2 * per} -c {per} --csv --log-file {out_dir}/traffic_{i:02d}.csv "
                    + TRAFFIC_BENCH.format(cache=cache))
    return cmds


def _ncu_rows(path: str):
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1024.0, "MB": 1048576.0,
             "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "ns": 1e-9, "us": 1e-6, "ms": 1e-3}
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    h = rows[hi]
    ci = {k: h.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    launches = {}
    for r in rows[hi + 1:]:
        if len(r) < len(h):
            continue
        L = launches.setdefault(int(r[ci["ID"]]), {"name": r[ci["Kernel Name"]], "bytes": 0.0, "s": 0.0})
        v = float(r[ci["Metric Value"]].replace(",", "")) * scale.get(r[ci["Metric Unit"]], 1.0)
        if r[ci["Metric Name"]] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            L["bytes"] += v
        elif r[ci["Metric Name"]] == "gpu__time_duration.sum":
            L["s"] += v
    return [launches[k] for k in sorted(launches)]


def write_traffic(csv_dir: str) -> dict:
    """profiles/traffic.json from the per-kernel CSVs of traffic_commands(): DRAM
    bytes per search of every kernel, per reported stage, and over the broad
    phase's kernels."""
    out = {"source_hash": source_hash(), "kernels": {}, "stages": {},
           "workload": "4096x512 vs 4096x512 vertex meshes, quad faces, patch level, mixed "
                       "precision (the bench workload)",
           "commands": traffic_commands("<dir>", "<cache>")}
    broad = 0.0
    for i, (rx, per, label, is_broad) in enumerate(TRAFFIC_KERNELS):
        path = os.path.join(csv_dir, f"traffic_{i:02d}.csv")
        if not os.path.exists(path):
            continue
        ls = _ncu_rows(path)
        if not ls:
            continue
        b = sum(L["bytes"] for L in ls)       # one search's launches of this kernel
        out["kernels"][rx] = {"dram_bytes_per_search": b, "launches": len(ls),
                              "duration_us_serialised": sum(L["s"] for L in ls) * 1e6}
        if label:
            key = STAGE_KERNELS[label]
            st = out["stages"].setdefault(key, {"dram_bytes_per_search": 0.0, "kernels": []})
            st["dram_bytes_per_search"] += b
            st["kernels"].append(rx)
        if is_broad:
            broad += b
    out["broad_dram_bytes_per_search"] = broad
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


# the files that hold the search's kernels and their launch sequence
SEARCH_SOURCES = ("tms_common.cuh", "tms_faces.cu", "tms_group.cu", "tms_pairs.cu",
                  "tms_narrow.cu", "tms_sort.cu", "tms_api.cu")


def source_hash() -> str:
    """Hash of the search's kernel sources: committed DRAM counters taken on other
    sources are not reported."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2109_14814_gb300", "csrc")
    for name in SEARCH_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# the smaller workload offered for profiler captures (the pool's rule: counters
# beyond the launch list on a case of a few GB at most, inputs larger than L2)
WORKLOAD_1024 = dict(workload="mesh-vs-mesh search, 1024x256 vs 1024x256 vertex grids "
                              "(522,240 triangles per mesh), lambda=4 stretch, 3 folds, 64 planted hits",
                     N=1024, M=256, triangles_per_mesh=522240)


def build_workload(device, cache: str = "", config: int = 3):
    """The 4096 x 512 pair (config 3), or the 1024 x 256 pair (config 2); with
    `cache`, read from that file when it exists (else generated and written
    there), so that repeated runs of the bench in one session (profiler
    captures) skip the generator."""
    import synth
    if cache and os.path.exists(cache):
        return torch.load(cache, weights_only=False)
    pair = synth.config2() if config == 2 else synth.config3()
    if cache:
        torch.save(pair, cache)
    return pair


def fp64_peak(device) -> float:
    """FP64 FMA throughput of this GPU (TFLOP/s), from a dependent-chain kernel
    with enough independent chains to fill every SM (torch-free: libtms)."""
    import paper_2109_14814_gb300 as tms
    return tms.probe_fp64_tflops()


def run_tms(args, ws, rank, local):
    import paper_2109_14814_gb300 as tms

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    peaks, peaks_kind = measured_peaks()
    pair = build_workload(device, args.workload_cache, args.config)
    XA = pair.A.X.to(device).contiguous()
    XB = pair.B.X.to(device).contiguous()
    A = tms.Mesh(XA, pair.A.s, True)
    B = tms.Mesh(XB, pair.B.s, True)
    stream = torch.cuda.Stream(device)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)
    out = torch.empty((1 << 17, tms.HIT_BYTES), dtype=torch.uint8, device=device)
    kw = dict(timing=0)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            h = tms.search(A, B, out=out, stream=stream, **kw)
        n_hits = len(h)
        stats = tms.last_stats(stream)
        # per-stage device times from a separate plan whose graph records an event
        # between stages (the events cost time, so the timed steps run without them)
        stage_sum = {}
        n_stage_runs = 10
        for i in range(3 + n_stage_runs):
            flush.fill_(i & 0xFF)
            tms.search(A, B, out=out, stream=stream, timing=1)
            if i >= 3:
                for k, v in tms.last_stage_ms(stream).items():
                    stage_sum[k] = stage_sum.get(k, 0.0) + v
        stage_ms = {k: v / n_stage_runs for k, v in stage_sum.items()}

    if args.only_extras:
        # just the named secondary measurements (for profiling them on their own)
        fp64_tf = tms.probe_fp64_tflops()
        runs = {"plain_fp64": lambda: plain_fp64(tms, A, B, out, stream, flush, h, fp64_tf),
                "batched": lambda: batched_search(tms, device, stream, flush),
                "adjoint": lambda: adjoint_timing(tms, device, stream),
                "refine": lambda: refine_timing(tms, pair, h, stream, flush, fp64_tf),
                "continuation": lambda: continue_timing(tms, pair, h, stream, fp64_tf),
                "layers": lambda: layer_timing(tms, device, stream, flush),
                "theta": lambda: theta_timing(tms, device, stream, flush),
                "e2e_pipelined": lambda: pipelined_e2e(tms, pair, device)}
        names = [x for x in args.only_extras.split(",") if x]
        unknown = [x for x in names if x not in runs]
        if unknown:
            raise SystemExit(f"unknown extras {unknown}; choose from {sorted(runs)}")
        if rank == 0:
            print(json.dumps({"extras": {x: runs[x]() for x in names}}), flush=True)
        return

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(i & 0xFF)          # L2 flush, outside the step's events
                starts[i].record(stream)
                h = tms.search(A, B, out=out, stream=stream, **kw)
                ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), device)
    if ws > 1:
        torch.distributed.barrier()
    value, ms_per_step = job_times(total_ms, args.steps, ws)

    # Roofline of the broad phase (A2-A7: bounds pass through candidate emission),
    # the search's HBM-bound part, as one unit: its algorithmic bytes
    #   B_broad = V * 32 (each mesh's FP64 vertices read once, both meshes)
    #           + E * 16 (one 8-byte (key, id) entry written and read per
    #                     face-cell incidence the grid registers)
    #           + K * 8  (one 8-byte candidate pair written)
    # with E and K this search's counts (at the patch level E counts patch-cell
    # incidences and K quad pairs), divided by the summed device time of the
    # broad stages; and the ncu DRAM bytes of the same kernels (profiles/
    # traffic.json, taken on the same sources) over the same time.  Both
    # against the measured copy bandwidth.  Per stage, the share of B_broad that
    # stage moves: the vertex read (bounds pass), the entry writes (cell passes),
    # the entry reads (cell table), the candidate writes (emission).
    V2 = pair.A.N * pair.A.M + pair.B.N * pair.B.M
    E, K = stats["entries"], stats["candidates"]
    hbm = peaks.get("hbm_gbs")
    broad_stages = BROAD_STAGES
    broad_ms = sum(stage_ms.get(k, 0.0) for k in broad_stages)
    b_broad = 32 * V2 + 16 * E + 8 * K
    share = {"face_bounds": 32 * V2, "face_probe": 8 * E, "group_count": 8 * E,
             "emit": 8 * K}
    kernels = {}
    for st_name, kname in STAGE_KERNELS.items():
        t = sum(stage_ms.get(x, 0.0) for x in STAGE_PARTS[st_name])
        byt = share.get(st_name, 0)
        ach = (byt / 1e9) / (t / 1e3) if (t > 0 and byt) else None
        kernels[st_name] = {"kernel": kname, "ms": t, "algorithmic_bytes": byt, "achieved_gbs": ach,
                            "frac": ach / hbm if (ach and hbm) else None,
                            "traffic": committed_traffic(kname)}
    traffic = broad_traffic()
    ach = (b_broad / 1e9) / (broad_ms / 1e3) if broad_ms > 0 else None
    roofline = {"kernel": "broad phase: " + ", ".join(BROAD_KERNELS), "stage": "broad (A2-A7)",
                "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm if (ach and hbm) else None, "traffic": traffic,
                "peak_kind": f"{peaks_kind} copy bandwidth",
                "algorithmic_bytes": b_broad,
                "algorithmic_formula": "32 V + 16 E + 8 K (V vertices of both meshes, E face-cell "
                                       "entries, K candidate pairs)",
                "V": V2, "E": E, "K": K, "ms": broad_ms,
                "share_of_step": broad_ms / ms_per_step if ms_per_step else None,
                "ncu_achieved": (traffic / 1e9) / (broad_ms / 1e3) if (traffic and broad_ms) else None,
                "ncu_frac": ((traffic / 1e9) / (broad_ms / 1e3) / hbm) if (traffic and broad_ms and hbm)
                else None,
                "largest_stage": max(stage_ms, key=stage_ms.get)}
    # FP64 utilisation of the narrow phase
    fp64 = None
    try:
        peak64 = tms.probe_fp64_tflops()
        flops = float(FP64_SOLVE_FLOPS) * stats["fp64_solves"]
        t_narrow = stage_ms.get("narrow", 0.0)
        ach = flops / (t_narrow / 1e3) / 1e12 if t_narrow > 0 else None
        fp64 = {"kernel": "tms::k_narrow", "solves_fp64": stats["fp64_solves"],
                "candidates": stats["candidates"], "flops_per_solve": FP64_SOLVE_FLOPS,
                "achieved_tflops": ach, "peak_tflops": peak64,
                "frac": (ach / peak64) if (ach and peak64) else None,
                "peak_kind": "measured FP64 FMA-chain probe on this GPU"}
    except Exception as e:  # the probe is optional diagnostics
        fp64 = {"error": str(e)}
    # FP32 arithmetic of the narrow phase's filters (quad-level and triangle-level
    # separating axes, verified solves) over the narrow stage's time, against the
    # FP32 lane rate at the maximum clock
    t_narrow = stage_ms.get("narrow", 0.0)
    f32 = (QUAD_SAT_FLOPS * stats["quad_tests"] + SAT_FLOPS * stats["sat_tests"]
           + FP32_SOLVE_FLOPS * stats["fp32_solves"])
    ach32 = f32 / (t_narrow / 1e3) / 1e12 if t_narrow > 0 else None
    narrow_fp32 = {"bound": "alu", "flops": f32, "ms": t_narrow, "achieved_tflops": ach32,
                   "peak_tflops": FP32_PEAK_TFLOPS,
                   "frac": ach32 / FP32_PEAK_TFLOPS if ach32 else None,
                   "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz, FMA = 2",
                   "counts": {"quad_tests": stats["quad_tests"], "sat_tests": stats["sat_tests"],
                              "fp32_solves": stats["fp32_solves"]}}

    # end to end through the C ABI with host buffers (tms_search_host: the
    # vertices copied from pinned host memory, the search, the hits copied back)
    e2e = None
    if not args.no_e2e:
        hA = pair.A.X.contiguous().pin_memory()
        hB = pair.B.X.contiguous().pin_memory()
        hout = torch.empty((1 << 17, tms.HIT_BYTES), dtype=torch.uint8).pin_memory()
        e_times = []
        d2h = 0
        with torch.cuda.stream(stream):
            for i in range(max(3, args.steps // 2) + 2):
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                he = tms.search_host(A, B, hA, hB, out=hout, stream=stream)
                n = len(he)
                ev1.record(stream)
                stream.synchronize()
                if i >= 2:
                    e_times.append(ev0.elapsed_time(ev1))
                d2h = n * tms.HIT_BYTES
        e_ms = sum(e_times) / len(e_times)
        e2e = {"value": e_ms / 1.0, "unit": UNIT,
               "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(pair)

    extras = None
    if args.extras:
        extras = {"plain_fp64": plain_fp64(tms, A, B, out, stream, flush, h,
                                           (fp64 or {}).get("peak_tflops")),
                  "batched": batched_search(tms, device, stream, flush),
                  "adjoint": adjoint_timing(tms, device, stream),
                  "refine": refine_timing(tms, pair, h, stream, flush,
                                          (fp64 or {}).get("peak_tflops") or tms.probe_fp64_tflops()),
                  "continuation": continue_timing(tms, pair, h, stream,
                                                  (fp64 or {}).get("peak_tflops") or tms.probe_fp64_tflops()),
                  "layers": layer_timing(tms, device, stream, flush),
                  "theta": theta_timing(tms, device, stream, flush),
                  "e2e_pipelined": pipelined_e2e(tms, pair, device)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded manifold-like meshes)",
        "config": dict(WORKLOAD if args.config == 3 else WORKLOAD_1024, precision="FP32 outward boxes and certified FP32 pre-solve, FP64 narrow phase",
                       l2="256 MiB buffer written between steps, outside the step events",
                       parallelism=f"replicas x{ws}" if ws > 1 else "1 GPU",
                       hits=n_hits, candidates=stats["candidates"], entries=stats["entries"],
                       cells=stats["cells"], pair_slots=stats["pair_slots"],
                       patch_pairs=stats["patch_pairs"], patch_tests=stats["patch_tests"],
                       quad_tests=stats["quad_tests"], quad_kept=stats["quad_kept"],
                       sat_tests=stats["sat_tests"],
                       fp32_solves=stats["fp32_solves"], fp64_solves=stats["fp64_solves"]),
        "roofline": roofline, "kernels": kernels, "fp64": fp64, "narrow_fp32": narrow_fp32,
        "cpu_baseline": cpu, "e2e": e2e,
        "clocks": clk.summary(), "gpu_launches": stats["kernels"] * args.steps,
        "source_hash": source_hash(),
        "stage_ms": stage_ms, "wall_s": wall,
    }
    if extras is not None:
        line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)


def _timed(fn, stream, flush, steps):
    """Median CUDA-event time (ms) of fn() over `steps` runs, L2 flushed before each."""
    ts = []
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def plain_fp64(tms, A, B, out, stream, flush, mixed_hits, fp64_tf=None):
    """The same search with FP64 boxes and cell keys and no FP32 filters (the
    plain path): its time, whether it finds the identical hit set, and the FP64
    rate of its narrow stage (every triangle pair of every candidate solved,
    FP64_SOLVE_FLOPS each) against the measured FP64 peak."""
    kw = dict(precision=0, narrow_filter=0)
    with torch.cuda.stream(stream):
        for _ in range(3):
            h = tms.search(A, B, out=out, stream=stream, **kw)
        same = (torch.equal(h.triA, mixed_hits.triA) and torch.equal(h.triB, mixed_hits.triB))
    ms = _timed(lambda: tms.search(A, B, out=out, stream=stream, **kw), stream, flush, 20)
    with torch.cuda.stream(stream):
        tms.search(A, B, out=out, stream=stream, timing=1, **kw)
    st = tms.last_stats(stream)
    stage = tms.last_stage_ms(stream)
    t_n = stage.get("narrow", 0.0)
    ach = FP64_SOLVE_FLOPS * st["fp64_solves"] / (t_n * 1e-3) / 1e12 if t_n > 0 else None
    return {"ms_per_search": ms, "hits": len(h), "identical_hit_set_to_mixed": bool(same),
            "fp64_solves": st["fp64_solves"], "narrow_ms": t_n,
            "fp64": {"kernel": "tms::k_narrow_fp64", "flops_per_solve": FP64_SOLVE_FLOPS,
                     "achieved_tflops": ach, "peak_tflops": fp64_tf,
                     "frac": (ach / fp64_tf) if (ach and fp64_tf) else None,
                     "peak_kind": "measured FP64 FMA-chain probe on this GPU"},
            "params": "precision=0 (FP64 boxes and keys), narrow_filter=0 (every pair to FP64)"}


def batched_search(tms, device, stream, flush, n_pairs=256):
    """The batched search of the 256 uneven mesh pairs of the alpha sweep (one
    CUDA graph replay per batch): total and per-pair time; beside it the same
    sweep as a loop of one search per pair, in the plain FP64 form and in the
    mixed form, and the batched plain form, each with the identical hit set."""
    import synth
    sizes = synth.config4_sizes(n_pairs=n_pairs)
    pairs = [synth.config4_pair(p, n_pairs=n_pairs, sizes=sizes) for p in range(n_pairs)]
    XA = [p.A.X.to(device).contiguous() for p in pairs]
    XB = [p.B.X.to(device).contiguous() for p in pairs]
    As = [tms.Mesh(x, p.A.s, True) for x, p in zip(XA, pairs)]
    Bs = [tms.Mesh(x, p.B.s, True) for x, p in zip(XB, pairs)]
    tris = sum(2 * p.A.N * (p.A.M - 1) + 2 * p.B.N * (p.B.M - 1) for p in pairs)
    out = torch.empty((1 << 18, tms.HIT_BYTES), dtype=torch.uint8, device=device)
    offs = torch.empty(n_pairs + 1, dtype=torch.int64, device=device)

    def keys(h):
        return list(zip(h.pair.tolist(), h.triA.tolist(), h.triB.tolist()))

    def batched(**kw):
        with torch.cuda.stream(stream):
            for _ in range(3):
                h = tms.search_batched(As, Bs, out=out, offsets=offs, stream=stream, **kw)
        k = keys(h)
        st = tms.last_stats(stream)
        ms = _timed(lambda: tms.search_batched(As, Bs, out=out, offsets=offs, stream=stream, **kw),
                    stream, flush, 10)
        return ms, k, st

    one = torch.empty((1 << 14, tms.HIT_BYTES), dtype=torch.uint8, device=device)

    def loop(**kw):
        found = []

        def run():
            found.clear()
            for p in range(n_pairs):
                h = tms.search(As[p], Bs[p], out=one, stream=stream, **kw)
                found.extend((p, a, b) for a, b in zip(h.triA.tolist(), h.triB.tolist()))
        with torch.cuda.stream(stream):
            run()
        ms = _timed(run, stream, flush, 2)
        return ms, sorted(found)

    ms, k, stats = batched()
    # the autotuner's per-size-class choice, read back through the cache file
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    t0 = time.perf_counter()
    best, _ = tms.autotune(As, Bs, cache_path=cache, stream=stream)
    tune_s = time.perf_counter() - t0
    ms_tuned, k_tuned, _ = batched(autotune_cache=cache)
    classes = [l.split() for l in open(cache).read().splitlines() if l.startswith("C|")]
    ms_plain_b, k_plain_b, _ = batched(precision=0, narrow_filter=0)
    ms_loop_plain, k_loop_plain = loop(precision=0, narrow_filter=0)
    ms_loop_mixed, k_loop_mixed = loop()
    return {"pairs": n_pairs, "triangles_total": tris, "ms_per_batch": ms,
            "ms_per_pair": ms / n_pairs, "hits": len(k), "launches_per_batch": stats["kernels"],
            "entries": stats["entries"], "candidates": stats["candidates"],
            "tuned_ms_per_batch": ms_tuned, "tuning_s": tune_s,
            "tuned": {"face_level": best["face_level"], "patch": best["patch"],
                      "block_faces": best["block_faces"], "tile_rows": best["tile_rows"],
                      "cell_mult_by_size_class": {c[0].split("class=")[1].split("|")[0]: float(c[1])
                                                  for c in classes}},
            "plain_fp64_batched_ms": ms_plain_b,
            "plain_fp64_loop_ms": ms_loop_plain,
            "mixed_loop_ms": ms_loop_mixed,
            "speedup_batched_vs_plain_loop": ms_loop_plain / ms if ms > 0 else None,
            "identical_hit_set": {"plain_batched": k_plain_b == k, "plain_loop": k_loop_plain == k,
                                  "mixed_loop": k_loop_mixed == k, "tuned": k_tuned == k},
            "loop_note": "one tms_search per pair on the same stream (each synchronises to read "
                         "its count), host time included"}


def adjoint_timing(tms, device, stream):
    """tms_backward on the 512-hit differentiation workload (config 5): time per
    call and FP64 rate at ~150 FLOPs per hit."""
    import synth
    pair = synth.config5()
    XA = pair.A.X.to(device).contiguous()
    XB = pair.B.X.to(device).contiguous()
    A = tms.Mesh(XA, pair.A.s, True)
    B = tms.Mesh(XB, pair.B.s, True)
    hits = tms.search(A, B, stream=stream)
    n = len(hits)
    g = torch.Generator(device="cpu").manual_seed(5)
    gP = torch.randn(n, 4, generator=g, dtype=torch.float64).to(device)
    gZ = torch.randn(n, 4, generator=g, dtype=torch.float64).to(device)
    gA = torch.zeros_like(XA)
    gB = torch.zeros_like(XB)
    dA = pair.A.dXdalpha.to(device).contiguous()
    dB = pair.B.dXdalpha.to(device).contiguous()
    ga = torch.zeros(n, dtype=torch.float64, device=device)
    call = lambda: tms.backward(A, B, hits, gP=gP, gZ=gZ, gradA=gA, gradB=gB, dA_dalpha=dA,
                                dB_dalpha=dB, galpha=ga, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(3):
            call()
    ts = []
    with torch.cuda.stream(stream):
        for _ in range(20):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    return {"hits": n, "ms_per_backward": ms, "fp64_gflops": 150.0 * n / (ms / 1e3) / 1e9,
            "note": "latency-bound: a few hundred hits, one thread each"}


def refine_flops_per_eval(K: int, n_folds: int) -> int:
    """Algorithmic FP64 flops of one evaluation of f, Df and the damped-Newton
    update for one seed (FMA = 2), counted from the closed-form sheets:
    128 per harmonic (three harmonic sums over 4 coordinates plus two
    angle-addition steps), 66 per fold (two cubics and five 4-vector
    accumulations), 695 for the rest (sheet assembly 68, 19 dot products 133,
    normal frame and its partials 270, crossing term and row of Df 92, norms 42,
    4x4 elimination 70, arguments 12, update 8).  Sines, cosines, exponentials,
    square roots and divisions are not counted."""
    return 695 + 128 * K + 66 * n_folds


def refine_timing(tms, pair, hits, stream, flush, fp64_tf):
    """tms_refine on the search's own hits, seeds read in place from the hit
    records (default schedule: alpha 0.5, tol 1e-10): time per call, seeds/s,
    iterations and FP64 rate against the measured FP64 peak; plus the oracle
    on a bounded sample of generator seeds (the planted records' estimates)."""
    from oracle import refine as oref
    sp = tms.surface_pair(pair.surface)
    n = len(hits)
    dev = hits.raw.device
    res = tms.Refined(torch.empty((n, 4), dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.int32, device=dev),
                      torch.empty(n, dtype=torch.int32, device=dev))
    call = lambda: tms.refine(sp, hits, stream=stream, out=res)
    with torch.cuda.stream(stream):
        for _ in range(3):
            call()
    ms = _timed(call, stream, flush, 20)
    st = res.status.cpu().numpy()
    it = res.iters.cpu().numpy().astype(np.int64)
    evals = int(it.sum() + np.isin(st, (0, 1, 2)).sum())
    fpe = refine_flops_per_eval(sp.n_harmonics, sp.n_folds)
    achieved = fpe * evals / (ms * 1e-3) / 1e12
    seeds = pair.planted.params.numpy()
    t0 = time.perf_counter()
    o = oref.damped_newton(pair.surface, seeds)
    cpu_s = time.perf_counter() - t0
    o_evals = int(o["iters"].sum() + np.isin(o["status"], (0, 1, 2)).sum())
    return {"seeds": n, "ms_per_call": ms, "seeds_per_s": n / (ms * 1e-3),
            "iterations_total": int(it.sum()), "evaluations": evals,
            "iterations_median": float(np.median(it)) if n else 0.0,
            "status_counts": {tms.REFINE_STATUS[k]: int((st == k).sum()) for k in range(5)},
            "roofline": {"kernel": "tms::k_refine", "bound": "alu (fp64)", "achieved": achieved,
                         "peak": fp64_tf, "unit": "TFLOP/s", "frac": achieved / fp64_tf,
                         "flops_per_evaluation": fpe,
                         "peak_kind": "measured FP64 FMA-chain probe on this GPU"},
            "cpu_baseline": {"value": cpu_s * 1e3 / max(o_evals, 1), "unit": "ms/evaluation",
                             "gpu_value": ms / max(evals, 1), "cores": 1, "kind": "oracle",
                             "sample": f"{len(seeds)} planted-record seeds of the same meshes, "
                                       "numpy FP64 vectorised over seeds"}}


def continue_timing(tms, pair, hits, stream, fp64_tf, n_steps=50, dalpha=1e-3, max_iter=60):
    """tms_continue from the search's own hits (seeds read in place) through
    n_steps values of alpha_u (step 0 refines the hits at the meshes' alpha):
    time per call, branch-steps/s and FP64 rate; plus the oracle on a bounded
    sample of generator seeds (the planted records' estimates)."""
    from oracle import refine as oref
    sp = tms.surface_pair(pair.surface)
    alphas = torch.tensor([pair.surface.alpha + dalpha * (j + 1) for j in range(n_steps)],
                          dtype=torch.float64)
    call = lambda: tms.continue_branches(sp, hits, alphas, stream=stream, max_jump=0.05,
                                         max_iter=max_iter)
    with torch.cuda.stream(stream):
        for _ in range(2):
            out = call()
        ts = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = call()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    st = out.status.cpu().numpy()
    it = out.iters.cpu().numpy().astype(np.int64)
    evals = int(it.sum() + np.isin(st, (0, 1, 2, 5, 6)).sum())
    fpe = refine_flops_per_eval(sp.n_harmonics, sp.n_folds)
    achieved = fpe * evals / (ms * 1e-3) / 1e12
    n = len(hits)
    seeds = pair.planted.params.numpy()[:256]
    t0 = time.perf_counter()
    o = oref.continuation(pair.surface, seeds, alphas.numpy(), param="u", max_jump=0.05,
                          max_iter=max_iter)
    cpu_s = time.perf_counter() - t0
    o_evals = int(o["iters"].sum() + np.isin(o["status"], (0, 1, 2, 5, 6)).sum())
    final = st[:, -1] if n else st
    return {"branches": n, "steps": n_steps + 1, "dalpha": dalpha, "ms_per_call": ms,
            "corrector": f"alpha 0.5, tol 1e-10, max_iter {max_iter} per step; max_jump 0.05",
            "branch_steps_per_s": n * (n_steps + 1) / (ms * 1e-3), "evaluations": evals,
            "branches_alive_at_end": int((final == 0).sum()),
            "status_at_end": {tms.CONTINUE_STATUS[k]: int((final == k).sum()) for k in range(8)},
            "roofline": {"kernel": "tms::k_continue", "bound": "alu (fp64)", "achieved": achieved,
                         "peak": fp64_tf, "unit": "TFLOP/s", "frac": achieved / fp64_tf,
                         "flops_per_evaluation": fpe,
                         "peak_kind": "measured FP64 FMA-chain probe on this GPU"},
            "cpu_baseline": {"value": cpu_s * 1e3 / max(o_evals, 1), "unit": "ms/evaluation",
                             "gpu_value": ms / max(evals, 1), "cores": 1, "kind": "oracle",
                             "sample": f"{len(seeds)} planted-record branches of the same meshes "
                                       "over the same steps, numpy FP64 vectorised over branches"}}


def layer_timing(tms, device, stream, flush):
    """The method-of-layers sweep at the paper's benchmark shapes (1024 x 957 and
    2048 x 1025 globalized meshes, 14 layers, 112 half-layer pairs of
    2,424,307,712 quad pairs each): one batched search per sweep (graph replay)
    against the paper's loop of one search per pair."""
    import synth
    p = synth.layered_pair(device="cpu")
    lay = p.meta["layers"]
    XA = p.A.X.to(device).contiguous()
    XB = p.B.X.to(device).contiguous()
    A = tms.Mesh(XA, p.A.s, True)
    B = tms.Mesh(XB, p.B.s, True)
    pairs = tms.layer_pairs(p.A.s, lay["D_u"], lay["lam_u"], p.B.s, lay["D_s"], lay["lam_s"],
                            lay["n_max"])
    sweep = tms.LayerSweep(A, B, pairs)
    out = torch.empty((1 << 16, tms.HIT_BYTES), dtype=torch.uint8, device=device)
    offs = torch.empty(len(pairs) + 1, dtype=torch.int64, device=device)
    with torch.cuda.stream(stream):
        for _ in range(3):
            h = sweep.search(out=out, offsets=offs, stream=stream)
    stats = tms.last_stats(stream)
    ms = _timed(lambda: sweep.search(out=out, offsets=offs, stream=stream), stream, flush, 10)
    views = [(tms.Mesh(XA, p.A.s, True, k0=q["a"][0], k1=q["a"][1]),
              tms.Mesh(XB, p.B.s, True, k0=q["b"][0], k1=q["b"][1])) for q in pairs]
    one = torch.empty((1 << 14, tms.HIT_BYTES), dtype=torch.uint8, device=device)

    def loop():
        for va, vb in views:
            tms.search(va, vb, out=one, stream=stream)
    with torch.cuda.stream(stream):
        loop()
    ms_loop = _timed(loop, stream, flush, 3)
    quad_pairs = sum((p.A.N * (q["a"][1] - q["a"][0] - 1)) * (p.B.N * (q["b"][1] - q["b"][0] - 1))
                     for q in pairs)
    return {"pairs": len(pairs), "quad_pairs_total": quad_pairs, "hits": len(h),
            "ms_per_sweep": ms, "ms_per_pair": ms / len(pairs),
            "quad_pairs_per_s": quad_pairs / (ms * 1e-3),
            "ms_per_sweep_one_search_per_pair": ms_loop, "launches_per_sweep": stats["kernels"],
            "meshes": f"{p.A.N}x{p.A.M} and {p.B.N}x{p.B.M}, {lay['n_max']} layers, "
                      f"{lay['per_layer'] + 1} columns per half-layer",
            "paper_context": "the paper's mean kernel time per half-layer pair: 0.14278 / 0.02964 / "
                             "0.04160 s on its three GPUs (broad phase only, narrow phase on the CPU)"}


def theta_timing(tms, device, stream, flush):
    """Globalization-style translation of every s column of a 2048 x 1025 x 4
    coordinate array by its own shift (Eq. translate), the theta-derivative of
    the same array (Eq. translate2), and 16 phase alignments of 4 x 4096
    circles (Eq. rhoEquationDiscrete); with the numpy oracle on the same data."""
    from oracle import theta as oth
    g = torch.Generator().manual_seed(11)
    C, M, N = 4, 1025, 2048
    X = torch.randn(C, M, N, generator=g, dtype=torch.float64)
    rho = torch.rand(M, generator=g, dtype=torch.float64) * 6.0 - 3.0
    Xd, rd, out = X.to(device), rho.to(device), torch.empty(C, M, N, dtype=torch.float64, device=device)
    with torch.cuda.stream(stream):
        for _ in range(3):
            tms.theta_translate(Xd, rd, out=out, stream=stream)
    ms_t = _timed(lambda: tms.theta_translate(Xd, rd, out=out, stream=stream), stream, flush, 10)
    ms_d = _timed(lambda: tms.theta_translate(Xd, rd, derivative=True, out=out, stream=stream),
                  stream, flush, 10)
    logn = int(round(math.log2(N)))
    # two complex transforms of N points per pair of real rows, 10 flops per butterfly,
    # plus the per-frequency multiply (6 flops)
    flops = (C // 2) * M * (2 * 10 * (N // 2) * logn + 6 * N)
    nbytes = 2 * C * M * N * 8
    t0 = time.perf_counter()
    oth.translate(X.numpy(), rho.numpy()[None, :])
    cpu_t = time.perf_counter() - t0
    A, Np = 16, 4096
    Wp = torch.randn(A, 4, Np, generator=g, dtype=torch.float64)
    Wr = torch.roll(Wp, 100, dims=-1) + 1e-3 * torch.randn(A, 4, Np, generator=g, dtype=torch.float64)
    Wpd, Wrd = Wp.to(device), Wr.to(device)
    with torch.cuda.stream(stream):
        tms.phase_align(Wrd, Wpd, stream=stream)
    ms_p = _timed(lambda: tms.phase_align(Wrd, Wpd, stream=stream), stream, flush, 5)
    t0 = time.perf_counter()
    oth.phase_align(Wr[0].numpy(), Wp[0].numpy())
    cpu_p = (time.perf_counter() - t0) * A
    fp64 = tms.probe_fp64_tflops()
    return {"translate": {"array": f"{C} x {M} x {N} (one shift per s column)", "ms": ms_t,
                          "derivative_ms": ms_d, "fp64_tflops": flops / (ms_t * 1e-3) / 1e12,
                          "fp64_frac": flops / (ms_t * 1e-3) / 1e12 / fp64,
                          "hbm_gbs": nbytes / (ms_t * 1e-3) / 1e9,
                          "flops_counted": "per pair of real rows: two N-point complex radix-2 "
                                           "transforms (10 flops per butterfly) + 6 per frequency",
                          "cpu_baseline_ms": cpu_t * 1e3, "cpu_kind": "oracle (numpy FFT, 1 core)"},
            "phase_align": {"alignments": A, "N": Np, "coords": 4, "ms": ms_p,
                            "norms_per_s": A * Np * Np / (ms_p * 1e-3),
                            "cpu_baseline_ms": cpu_p * 1e3,
                            "cpu_kind": "oracle (numpy, one roll per shift), one alignment timed x 16"}}


def pipelined_e2e(tms, pair, device, steps: int = 50):
    """End to end through tms_search with host buffers, as a job of many steps
    would run it: two device buffer sets, the host-to-device copy of step i+1 on
    a copy stream while step i searches, each step's hits copied back to pinned
    host memory.  The bench line's own e2e keeps every copy on the critical path."""
    hA = pair.A.X.contiguous().pin_memory()
    hB = pair.B.X.contiguous().pin_memory()
    XA = [torch.empty_like(hA, device=device) for _ in range(2)]
    XB = [torch.empty_like(hB, device=device) for _ in range(2)]
    As = [tms.Mesh(x, pair.A.s, True) for x in XA]
    Bs = [tms.Mesh(x, pair.B.s, True) for x in XB]
    outs = [torch.empty((1 << 17, tms.HIT_BYTES), dtype=torch.uint8, device=device) for _ in range(2)]
    hout = torch.empty((1 << 17, tms.HIT_BYTES), dtype=torch.uint8).pin_memory()
    s_copy, s_comp = torch.cuda.Stream(device), torch.cuda.Stream(device)
    copied = [torch.cuda.Event() for _ in range(2)]

    def copy_into(b):
        with torch.cuda.stream(s_copy):
            XA[b].copy_(hA, non_blocking=True)
            XB[b].copy_(hB, non_blocking=True)
            copied[b].record(s_copy)

    def run(n):
        copy_into(0)
        n_hits = 0
        for i in range(n):
            b = i % 2
            s_comp.wait_event(copied[b])
            if i + 1 < n:
                copy_into(1 - b)          # overlaps this step's search
            h = tms.search(As[b], Bs[b], out=outs[b], stream=s_comp)
            n_hits = len(h)
            with torch.cuda.stream(s_comp):
                hout[:n_hits].copy_(h.raw, non_blocking=True)
        return n_hits

    run(4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_copy)
    n_hits = run(steps)
    e1.record(s_comp)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"ms_per_step": ms, "steps": steps, "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8),
            "d2h_bytes_per_step": int(n_hits * tms.HIT_BYTES),
            "scheme": "two device buffer sets; the H2D copy of step i+1 on a copy stream during "
                      "the search of step i; hits of every step copied to pinned host memory"}


def cpu_baseline(pair):
    import oracle
    OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
    t0 = time.perf_counter()
    r = oracle.search(OA, OB)
    dt = time.perf_counter() - t0
    return {"value": dt * 1e3, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "the full workload (one complete search): FP64 C oracle, exact box "
                      "pruning by a bounding-volume hierarchy, OpenMP over A triangles",
            "hits": int(r.size)}


def run_reference(args, ws, rank, local):
    """The oracle (CPU, FP64) on the same workload and metric.  Its cost is
    dominated by the bounding-volume hierarchy over mesh B, so a step cannot be
    a smaller sample of the search: every step is one complete search, and the
    steps are capped (REF_MAX_STEPS timed, one warm-up) so that the run ends in
    well under a minute on the host cores."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pair = build_workload("cpu")
    OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
    steps, warmup = max(1, min(args.steps, REF_MAX_STEPS)), min(args.warmup, 1)
    for _ in range(warmup):
        oracle.search(OA, OB)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.search(OA, OB)
        times.append((time.perf_counter() - t0) * 1e3)
    v = sum(times) / len(times)
    sample = (f"the full workload per step (one complete search); {steps} timed steps and "
              f"{warmup} warm-up of the {args.steps} + {args.warmup} requested")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded manifold-like meshes)", "config": dict(WORKLOAD),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tms", choices=["tms", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--extras", action="store_true",
                    help="also time the plain FP64 path, the batched 256-pair search, the adjoint, "
                         "the refinement of the hits, their continuation, the layer sweep and "
                         "the theta-grid operations")
    ap.add_argument("--write-traffic", default="", metavar="DIR",
                    help="write profiles/traffic.json from the per-kernel ncu CSVs in DIR "
                         "(made by the --traffic-commands lines) and exit; needs no GPU")
    ap.add_argument("--traffic-commands", default="", metavar="DIR",
                    help="print the per-kernel ncu commands (CSV into DIR) and exit")
    ap.add_argument("--config", type=int, default=3, choices=[2, 3],
                    help="3: the 4096 x 512 benchmark workload (default); 2: the 1024 x 256 "
                         "workload, for profiler captures of a small case")
    ap.add_argument("--workload-cache", default="", metavar="PATH",
                    help="read the workload from PATH if it exists, else generate and write it")
    ap.add_argument("--only-extras", default="",
                    help="comma-separated extras to run alone (no main timing): plain_fp64, batched, "
                         "adjoint, refine, continuation, layers, theta, e2e_pipelined")
    args = ap.parse_args()
    if args.write_traffic:
        t = write_traffic(args.write_traffic)
        for k, v in t["kernels"].items():
            print(f"{k}: {v['dram_bytes_per_search'] / 1e6:.1f} MB per search ({v['launches']} launches)")
        print(f"broad phase: {t['broad_dram_bytes_per_search'] / 1e6:.1f} MB per search")
        return
    if args.traffic_commands:
        for c in traffic_commands(args.traffic_commands, args.workload_cache or "/tmp/tms_c3.pt"):
            print(c)
        return
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank, local)
        return
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        run_tms(args, ws, rank, local)
    finally:
        if ws > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
