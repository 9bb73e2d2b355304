"""Benchmark: Floquet steps/s of the kicked-Ising BP-TNS evolution, 127-qubit
heavy-hex (Eagle layout), chi = 64, on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--chi 64] [--prec fp32] [--theta 0.8] [--presteps 7]

One timed step = one application of U(theta_h) (RX on 127 qubits, 144 ZZ gates
by BP-gauged simple update with the refined FP64 truncation solve, BP regauge
to the tolerance).  The state is evolved `presteps` untimed steps first so that every
bond has reached chi (steps >= log2(chi) + 1), then W warm-up steps, then K
timed steps bracketed by CUDA events on the library's stream.

Multi-GPU (torchrun): the theta sweep shards with no collective on the data
path: rank r evolves its own instance at theta_r from 16 uniform values in
[0, pi/2]; a barrier and an all-reduce of the elapsed time give max-over-ranks
timing ("scaling": "weak").

--impl reference times the CPU FP64 oracle (test infrastructure) on bounded
samples of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Floquet steps/s (127q heavy-hex, chi=64)"
UNIT = "steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join(ROOT, "paper_2306_14887_gb300", "csrc")

# nominal figures (GB300), used only when a measurement is missing
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_TFLOPS = 1.25
TF32_OVER_BF16 = 1.1 / 2.25

# the source files holding the kernels of each profile class (a committed
# traffic figure is used only while these files are unchanged)
_CONTRACT = ("tc_stream.cu", "tc_gemm.cu", "tc_common.cuh", "kernels.cu")
CLASS_SOURCE = {"bp_contract": _CONTRACT, "gate_env": _CONTRACT, "gate_rebuild": _CONTRACT,
                "bp_normalise": ("kernels.cu",), "copyback": ("kernels.cu",),
                "phys_gate": ("kernels.cu",), "rho": ("kernels.cu",),
                "trunc_solve": ("solve32.cu", "solve.cu", "solve_refine.cu"),
                "trunc_refine": ("solve_refine.cu",)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--chi", type=int, default=64)
    p.add_argument("--prec", default="tf32")
    p.add_argument("--fp32-steps", type=int, default=3,
                   help="timed steps of the plain FP32 path measured beside the main line (0: skip)")
    p.add_argument("--solve", default="auto", choices=["auto", "refined", "shared", "fp64"])
    p.add_argument("--kernels", default="auto", choices=["auto", "tile"])
    p.add_argument("--theta", type=float, default=None)
    p.add_argument("--presteps", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serve-jobs", type=int, default=16,
                   help="jobs of the serving leg (0: skip)")
    p.add_argument("--serve-mix", type=int, default=0,
                   help="jobs of the full-mix serving leg (all sizes and chi; 0: skip)")
    p.add_argument("--serve-policy", default="shortest", choices=["fifo", "shortest"],
                   help="admission order of the full-mix serving leg")
    p.add_argument("--solve-bench", default="",
                   help="only time the standalone truncation solves named here (comma-separated, "
                        "e.g. refined,shared) on one layer-sized batch, and exit")
    p.add_argument("--no-peaks", action="store_true",
                   help="skip the torch.matmul rate measurements (the roofline then takes the "
                        "peaks file and the nominal ratios), e.g. under a profiler")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the heuristic split-K counts of the sweep launches")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched 64-instance leg")
    p.add_argument("--batch-prec", default="tf32,tf32x3",
                   help="comma-separated precisions of the batched leg")
    p.add_argument("--config4", action="store_true",
                   help="also run the large-chi periodic-cell leg (chi 128 and 256, 50 steps, "
                        "theta 0.4 / 0.7 / 1.0, BF16X3 against FP32) and print its own line")
    p.add_argument("--config4-steps", type=int, default=50)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def theta_for(rank, args):
    if args.theta is not None:
        return args.theta
    grid = np.linspace(0.0, np.pi / 2, 16)
    # interior values: the endpoints are the trivial Clifford points
    return float(grid[(9 + rank) % 15 or 9])


def max_over_ranks(ms, device):
    """The slowest rank's elapsed time, on every rank (the only collective of
    the timing; the data path has none)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


SOLVE_NAMES = {
    "refined": "refined FP64 (FP64 Cholesky, FP32 Jacobi start, FP64 Newton refinement and legs)",
    "shared": "shared FP32 (FP32 Cholesky, Jacobi and legs)",
    "fp64": "FP64 Jacobi eigen-solves",
}


def solve_kind(solve, chi):
    """The truncation solve the library runs for --solve at this chi."""
    if solve == "auto":
        solve = "refined"
    if solve in ("refined", "shared") and chi > 64:
        return "fp64"
    return solve


def workload_config(args, world):
    """The workload both arms report (the reference arm times the oracle on it)."""
    chi = args.chi
    presteps = args.presteps if args.presteps is not None else int(np.log2(max(chi, 1))) + 1
    theta = theta_for(0, args)
    solve = SOLVE_NAMES[solve_kind(args.solve, chi)]
    return {"workload": f"eagle127 heavy-hex, chi={chi}, prec={args.prec}, solve={solve}, "
                        f"theta_h={theta:.4f}, saturated after {presteps} steps",
            "qubits": 127, "edges": 144, "chi": chi,
            "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (
                (36 * 4 * chi ** 3 + 89 * 4 * chi ** 2 + 2 * 4 * chi) * 4 / 1e6),
            "parallelism": f"theta-sharded x{world}" if world > 1 else "single GPU"}


def serve_leg(tn, args):
    """p50 / p99 latency of a bounded sample of the serving workload: the first
    jobs of the seeded Poisson stream (200 jobs/s) whose graph has at most 127
    qubits and chi at most 64, submitted at their arrival times to a server with
    4 slots; latency is arrival to result."""
    from workloads import serving_jobs
    n, edges, cols = eagle()
    keep = np.all(edges < 27, axis=1)  # the 27-qubit patch: qubits 0..26 of the layout
    graphs = {27: (27, edges[keep], cols[keep]), 127: (n, edges, cols)}
    stream = [j for j in serving_jobs(n=2000) if j[1] in graphs and j[2] <= 64][:args.serve_jobs]
    lat, steps_done = [], 0
    with tn.Server(slots=4) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (arr, size, chi, theta, steps) in stream:
            while time.perf_counter() - t0 < arr - stream[0][0]:
                time.sleep(0.0005)
            gn, ge, gc = graphs[size]
            tickets.append(srv.submit(gn, ge, gc, chi, theta, steps, prec=args.prec))
        for t in tickets:
            z, info = srv.wait(t)
            lat.append(info["latency_s"])
            steps_done += info["steps_done"]
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array(lat)
    return {"jobs": len(lat), "slots": 4, "arrival_rate_per_s": 200.0,
            "p50_s": round(float(np.percentile(lat, 50)), 4),
            "p99_s": round(float(np.percentile(lat, 99)), 4),
            "steps_per_s": round(steps_done / wall, 3), "peak_resident": st["peak_resident"],
            "sample": "first %d jobs of the seeded stream with <= 127 qubits and chi <= 64 "
                      "(27- and 127-qubit graphs, chi 16/32/64, 5-20 steps), prec %s"
                      % (len(lat), args.prec)}


def read_serving_golden():
    """{job index: (min_gap, z)} of the FP64 oracle's seeded serving sample
    (tests/golden/serving_sample_oracle.txt, written by a script that calls
    only oracle/)."""
    path = os.path.join(ROOT, "tests", "golden", "serving_sample_oracle.txt")
    out, gap = {}, {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "job":
            kv = dict(zip(f[2::2], f[3::2]))
            gap[int(f[1])] = float(kv["min_gap"])
        elif f[0] == "Z":
            i = int(f[1])
            out[i] = (gap[i], np.array([float(x) for x in f[2:]]))
    return out


def serve_mix_leg(tn, args):
    """The serving workload at its stated mix: the first --serve-mix jobs of the
    seeded Poisson stream (200 jobs/s; 27, 127, 433 and 1121 qubits; chi 16,
    32, 64 and 128; 5-20 steps) submitted at their arrival times to a server
    with 8 slots admitting by HBM footprint in the --serve-policy order.
    Latency is arrival to result; the <Z> error against the FP64 oracle on the seeded 2% sample of the jobs
    with at most 127 qubits and chi at most 64."""
    from workloads import serving_jobs
    n, edges, cols = eagle()
    keep = np.all(edges < 27, axis=1)
    graphs = {27: (27, edges[keep], cols[keep]), 127: (n, edges, cols),
              433: tn.heavy_hex(13, 27), 1121: tn.heavy_hex(21, 43)}
    stream = serving_jobs(n=2000)[:args.serve_mix]
    gold = read_serving_golden()
    lat, steps_done, dz = [], 0, {}
    by_kind = {}
    with tn.Server(slots=8, policy=args.serve_policy) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (arr, size, chi, theta, steps) in stream:
            while time.perf_counter() - t0 < arr - stream[0][0]:
                time.sleep(0.0005)
            gn, ge, gc = graphs[size]
            tickets.append(srv.submit(gn, ge, gc, chi, theta, steps, prec=args.prec))
        for i, t in enumerate(tickets):
            # the server records each job's latency itself, so the order of the
            # waits does not matter; a large job may finish last under the
            # least-work-first policy
            res = srv.wait(t, timeout=None)
            if res is None:
                raise RuntimeError("serving job %d did not finish" % i)
            z, info = res
            lat.append(info["latency_s"])
            steps_done += info["steps_done"]
            by_kind.setdefault("%dq" % stream[i][1], []).append(info["latency_s"])
            if i in gold:
                dz[i] = float(np.abs(np.asarray(z) - gold[i][1]).max())
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array(lat)
    return {"jobs": len(lat), "slots": 8, "arrival_rate_per_s": 200.0,
            "policy": args.serve_policy,
            "p50_s": round(float(np.percentile(lat, 50)), 3),
            "p99_s": round(float(np.percentile(lat, 99)), 3),
            "p50_s_by_size": {k: round(float(np.percentile(v, 50)), 3) for k, v in by_kind.items()},
            "steps_per_s": round(steps_done / wall, 3), "wall_s": round(wall, 2),
            "peak_resident": st["peak_resident"], "prec": args.prec,
            "oracle_dz": {str(k): float("%.3g" % v) for k, v in dz.items()},
            "oracle_min_gap": {str(k): float("%.3g" % gold[k][0]) for k in dz},
            "sample": "first %d jobs of the seeded stream, every size and chi; oracle on the "
                      "seeded 2%% sample of jobs with <= 127 qubits and chi <= 64 "
                      "(tests/golden/serving_sample_oracle.txt)" % len(lat)}


def read_batched_golden():
    """The FP64 oracle's <Z_v> for the covered instances of the batched
    workload (tests/golden/batched64_oracle.txt, written by a script that calls
    only oracle/): {index: (min_gap, z)}."""
    path = os.path.join(ROOT, "tests", "golden", "batched64_oracle.txt")
    out = {}
    if not os.path.exists(path):
        return out
    gap = {}
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "inst":
            kv = dict(zip(f[2::2], f[3::2]))
            gap[int(f[1])] = float(kv["min_gap"])
        elif f[0] == "Z":
            i = int(f[1])
            out[i] = (gap[i], np.array([float(x) for x in f[2:]]))
    return out


def batch_leg(tn, args):
    """The batched workload in each precision of --batch-prec (see batch_run)."""
    return {prec: batch_run(tn, args, prec) for prec in args.batch_prec.split(",") if prec}


def batch_run(tn, args, prec):
    """The batched workload: 64 seeded instances (27/65/127/433 qubits, chi from
    {8, 16, 32, 64}, theta_h ~ U[0, pi/2], 10 steps) as one union handle per chi,
    the four handles driven concurrently (tn.Batch).  Reports instance-steps/s
    of the batch and of the same instances run one by one, and per instance
    the <Z> error against its alone run and against the FP64 oracle (where the
    golden file covers it)."""
    import torch
    from workloads import batched_jobs
    graphs = {27: None, 65: tn.heavy_hex(5, 11), 127: eagle(), 433: tn.heavy_hex(13, 27)}
    n, edges, cols = graphs[127]
    keep = np.all(edges < 27, axis=1)
    graphs[27] = (27, edges[keep], cols[keep])
    jobs = batched_jobs(n=64)
    steps = jobs[0][3]
    insts = [graphs[size] + (chi, theta) for (size, chi, theta, _st) in jobs]
    # warm-up: the same batch for one step (module loading, graph capture paths)
    with tn.Batch(insts, prec=prec, solve=args.solve) as b:
        b.evolve(1)
    torch.cuda.synchronize()
    with tn.Batch(insts, prec=prec, solve=args.solve) as b:
        tuned = None
        if not args.no_autotune:
            # split-K counts per (chi, degree) launch shape, on the initial states (untimed)
            tables = b.autotune(reps=3)
            tuned = {str(chi): sum(1 for ln in t.splitlines() if ln.strip())
                     for chi, t in tables.items()}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.evolve(steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        zb = b.expect_z()
        sweeps = b.bp_sweeps()
    alone_s, d_alone = 0.0, []
    for (gn, ge, gc, chi, theta), z in zip(insts, zb):
        stream = torch.cuda.Stream()
        with tn.TNState(gn, ge, gc, chi=chi, prec=prec, stream=stream, solve=args.solve) as a:
            stream.synchronize()
            t0 = time.perf_counter()
            a.apply_floquet(theta, steps)
            stream.synchronize()
            alone_s += time.perf_counter() - t0
            d_alone.append(float(np.abs(a.expect_z_all() - z).max()))
    gold = read_batched_golden()
    d_oracle = [None] * len(jobs)
    near_tie = []
    for i, (gap, zo) in gold.items():
        d_oracle[i] = float(np.abs(zb[i] - zo).max())
        if gap <= 1e-6:
            near_tie.append(i)
    cov = [d for d in d_oracle if d is not None]
    return {"instances": len(jobs), "steps": steps,
            "instance_steps_per_s": round(len(jobs) * steps / wall, 3),
            "wall_s": round(wall, 3),
            "alone_instance_steps_per_s": round(len(jobs) * steps / alone_s, 3),
            "groups": "one union handle per chi (8, 16, 32, 64), driven concurrently",
            "max_dz_vs_alone": max(d_alone),
            "dz_vs_alone": [float("%.3g" % d) for d in d_alone],
            "oracle_covered": len(cov),
            "max_dz_vs_oracle": max(cov) if cov else None,
            "dz_vs_oracle": [None if d is None else float("%.3g" % d) for d in d_oracle],
            "oracle_near_ties": near_tie,
            "bp_sweeps_last": [int(x) for x in sweeps],
            "autotuned_rows_by_chi": tuned,
            "prec": prec,
            "note": "oracle values from tests/golden/batched64_oracle.txt (FP64 oracle on every "
                    "instance with chi <= 16, chi = 32 up to 127 qubits, chi = 64 at 27 qubits)"}


def config4_leg(tn, args):
    """The large-chi leg (the infinite heavy-hex lattice through its periodic
    5-site cell, reading r14): for chi in {128, 256} and theta_h in {0.4, 0.7,
    1.0}, `steps` Floquet steps with split-BF16 contractions and with the plain
    FP32 path, both with the refined FP64 truncation solve; per run the steps/s,
    the largest |<Z>| difference between the two precisions, and the mean over
    the cell's six bonds of the entanglement entropy s = -sum l^2 log2 l^2
    (reading r16)."""
    import torch
    # the 5-site cell: corners A = 0, B = 1, bond midpoints 2, 3, 4; A-m_k has
    # colour k - 1 and B-m_k colour k mod 3
    cell_edges = np.array([(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4)], dtype=np.int32)
    cell_cols = np.array([0, 1, 2, 1, 2, 0], dtype=np.uint8)

    class _Cell:
        n, edges, colours = 5, cell_edges, cell_cols
    g = _Cell()
    rows = []
    for chi in (128, 256):
        for theta in (0.4, 0.7, 1.0):
            res = {}
            for prec in ("bf16x3", "fp32"):
                stream = torch.cuda.Stream()
                with tn.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec, stream=stream) as s:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.apply_floquet(theta, args.config4_steps)
                    e1.record(stream)
                    stream.synchronize()
                    ms = e0.elapsed_time(e1)
                    res[prec] = {"z": s.expect_z_all(),
                                 "s": float(np.mean([s.entanglement_entropy(e)
                                                     for e in range(len(g.edges))])),
                                 "steps_per_s": args.config4_steps / (ms * 1e-3)}
            rows.append({"chi": chi, "theta_h": theta, "steps": args.config4_steps,
                         "bf16x3_steps_per_s": round(res["bf16x3"]["steps_per_s"], 3),
                         "fp32_steps_per_s": round(res["fp32"]["steps_per_s"], 3),
                         "max_dz_bf16x3_vs_fp32": float(np.abs(res["bf16x3"]["z"] -
                                                               res["fp32"]["z"]).max()),
                         "entropy_bf16x3": round(res["bf16x3"]["s"], 6),
                         "entropy_fp32": round(res["fp32"]["s"], 6),
                         "z_mean_fp32": float(np.mean(res["fp32"]["z"]))})
    return {"leg": "config4: periodic 5-site cell (infinite heavy-hex lattice), refined FP64 "
                   "truncation solve", "runs": rows}


def eagle():
    import paper_2306_14887_gb300 as tn
    return tn.heavy_hex(7, 15)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- roofline
def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


def src_hash(names):
    h = hashlib.sha256()
    for name in names:
        h.update(open(os.path.join(CSRC, name), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(cls):
    """DRAM bytes per launch of the class from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except Exception:
        return None
    ent = t.get(cls)
    if not ent or ent.get("source_sha") != src_hash(CLASS_SOURCE[cls]):
        return None
    return ent.get("dram_bytes_per_launch")


def bp_sweep_flops(chi, n_by_deg):
    """Algorithmic real flops of one BP sweep: 16 chi^4 complex multiply-adds per
    degree-3 site, 8 chi^3 per degree-2 site, 2 chi^2 per degree-1 site, 8 real
    flops per complex multiply-add."""
    return 8.0 * (16 * chi ** 4 * n_by_deg[3] + 8 * chi ** 3 * n_by_deg[2] + 2 * chi ** 2 * n_by_deg[1])


def measure_peaks():
    """TF32, FP32 (no TF32) and FP64 dense matmul rates of this GPU, measured the
    way the BF16 figure of the peaks file was: torch.matmul on square matrices,
    best of 5 after warm-up, CUDA events (TFLOP/s)."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, n, tf32 in (("tf32", torch.float32, 8192, True),
                              ("fp32", torch.float32, 4096, False),
                              ("fp64", torch.float64, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = 1e30
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(5):
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        out[name + "_tflops"] = round(2.0 * n ** 3 / best / 1e12, 2)
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "torch.matmul n^3 (tf32 8192, fp32 4096 without TF32, fp64 4096), best of 5"
    return out


def roofline(prof, prec, chi, sweeps, n_by_deg, solve, mp):
    """The roofline of the dominant profile class of the timed region."""
    cls = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[cls]
    n = max(1, p["launches"])
    ms_per = p["ms"] / n
    pk = peaks()
    bf16_sus = pk.get("bf16_tflops_sustained", 1715.0)
    sus_ratio = bf16_sus / pk.get("bf16_tflops", bf16_sus)
    if cls == "bp_contract":
        # algorithmic work of the sweeps, not the executed (padded, re-ordered) work
        p = dict(p)
        p["flops"] = bp_sweep_flops(chi, n_by_deg) * sweeps
    if cls == "trunc_refine":
        # FP64 Newton step and leg matrices (the library's algorithmic count)
        bound, unit = "alu", "TFLOP/s"
        peak = mp.get("fp64_tflops", FP64_TFLOPS)
        achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
        note = "FP64: measured torch.matmul float64"
    elif cls == "trunc_solve":
        bound, unit = "alu", "TFLOP/s"
        if solve == "fp64":
            peak, note = mp.get("fp64_tflops", FP64_TFLOPS), "FP64: measured torch.matmul float64"
        else:
            peak, note = mp.get("fp32_tflops", FP32_SIMT_TFLOPS), "FP32: measured torch.matmul without TF32"
        achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
    elif cls in ("bp_contract", "gate_env", "gate_rebuild"):
        if prec == "fp32":
            bound, unit = "alu", "TFLOP/s"
            peak, note = mp.get("fp32_tflops", FP32_SIMT_TFLOPS), "FP32: measured torch.matmul without TF32"
        elif prec in ("bf16", "bf16x3"):
            bound, unit = "tensor", "TFLOP/s"
            peak, note = bf16_sus, "bf16 sustained (peaks file)"
        else:
            bound, unit = "tensor", "TFLOP/s"
            peak = mp.get("tf32_tflops", pk.get("bf16_tflops", 1945.0) * TF32_OVER_BF16) * sus_ratio
            note = ("tf32: measured torch.matmul TF32 burst x the peaks file's bf16 "
                    "sustained/burst ratio (%.3f)" % sus_ratio)
        achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
    else:
        bound, unit, peak = "hbm", "GB/s", pk.get("hbm_gbs", 6792.1)
        achieved = p["bytes"] / (p["ms"] * 1e-3) / 1e9
        note = "measured HBM copy (peaks file)"
    tr = traffic_for(cls)
    return {"bound": bound, "kernel": cls, "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": unit, "frac": round(achieved / peak, 4),
            "traffic": tr, "launches": p["launches"], "ms_per_launch": round(ms_per, 4),
            "share_of_timed": None, "peak_source": note + " (of measured)"}


# ------------------------------------------------------------ CPU oracle leg
def oracle_step_estimate(chi, bp_iters, n_gate_sample=6, seed=3):
    """Time the FP64 oracle on a bounded sample of the 127-qubit chi workload:
    one synchronous BP sweep and `n_gate_sample` simple-update gates on a random
    state with every bond at chi; returns (seconds per Floquet step, detail)."""
    from oracle import bptn as OB
    from oracle import graph as OG
    from workloads import random_state
    g = OG.eagle127()
    tensors, msgs = random_state([g.degree(v) for v in range(g.n)], g.edges, chi, seed)
    st = OB.BPState(g, chi)
    st.T, st.M = tensors, msgs
    t0 = time.perf_counter()
    st.bp_sweep()
    t_sweep = time.perf_counter() - t0
    order = [e for layer in g.layers() for e in layer]
    pick = [order[i] for i in np.linspace(0, len(order) - 1, n_gate_sample).astype(int)]
    t0 = time.perf_counter()
    for e in pick:
        st.apply_zz(e)
    t_gate = (time.perf_counter() - t0) / len(pick)
    per_step = t_gate * len(g.edges) + bp_iters * t_sweep
    return per_step, {"t_sweep_s": t_sweep, "t_gate_s": t_gate, "gates_sampled": len(pick)}


def oracle_single_thread(chi, bp_iters, n_gate_sample=2):
    """The same bounded oracle sample in a fresh process with every BLAS and
    OpenMP pool at one thread; returns (seconds per Floquet step, detail) or
    None if the child fails."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    code = ("import json, bench; sec, det = bench.oracle_step_estimate(%d, %r, n_gate_sample=%d); "
            "print(json.dumps([sec, det]))" % (chi, float(bp_iters), n_gate_sample))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        sec, det = json.loads(r.stdout.strip().splitlines()[-1])
        return sec, det
    except Exception:
        return None


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


# --------------------------------------------------------------------- ours
def run_ours(args, rank, world, local):
    import torch
    import paper_2306_14887_gb300 as tn
    from paper_2306_14887_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        build.build()
    else:
        torch.cuda.set_device(local)
    chi = args.chi
    presteps = args.presteps if args.presteps is not None else int(np.log2(max(chi, 1))) + 1
    theta = theta_for(rank, args)
    n, edges, cols = eagle()
    mp = {} if args.no_peaks else measure_peaks()
    stream = torch.cuda.Stream()
    s = tn.TNState(n, edges, cols, chi=chi, prec=args.prec, stream=stream, solve=args.solve,
                     kernels=args.kernels)
    s.apply_floquet(theta, presteps)
    tune = None
    if not args.no_autotune:
        # split-K counts of the sweep launches timed on this state (untimed setup)
        table = s.autotune(reps=5)
        rows = [ln.split() for ln in table.strip().splitlines() if ln.strip()]
        tune = {"rows": len(rows),
                "split_counts": {k: sum(1 for r in rows if r[7] == k)
                                 for k in sorted({r[7] for r in rows}, key=int)},
                "note": "tn_autotune on the bench state after the untimed steps: per sweep "
                        "launch with a split-K count, the fastest power of two (kept only "
                        "when 3% faster than the heuristic's)"}
    for _ in range(args.warmup):
        s.apply_floquet(theta, 1)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    s.profile_enable(True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    tma_launches = 0
    bp_iters = 0
    disc = 0.0
    jac_sweeps = jac_edges = jac_max = 0
    for _ in range(args.steps):
        s.apply_floquet(theta, 1)
        st = s.stats()
        launches += st["kernel_launches"]
        tma_launches += st["tma_launches"]
        bp_iters += st["bp_iters_total"]
        disc = max(disc, st["discarded_max"])
        jac_sweeps += st["solve_sweeps"]
        jac_edges += st["solve_edges"]
        jac_max = max(jac_max, st["solve_sweeps_max"])
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.profile_enable(False)
    clocks = clk.stop()
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
    z = s.expect_z_all()
    s.close()
    value = world * args.steps / (ms * 1e-3)

    # end to end through the C ABI: a fresh job built from the host graph and
    # brought to the same saturated state (untimed), then the same K steps,
    # each followed by the device->host read of <Z_v> for all 127 qubits
    e2e = None
    if not args.no_e2e:
        s2 = tn.TNState(n, edges, cols, chi=chi, prec=args.prec, stream=stream, solve=args.solve,
                     kernels=args.kernels)
        s2.apply_floquet(theta, presteps + args.warmup)
        stream.synchronize()
        t0 = time.perf_counter()
        zs = []
        for _ in range(args.steps):
            s2.apply_floquet(theta, 1)
            zs.append(s2.expect_z_all())
        el = time.perf_counter() - t0
        s2.close()
        e2e = {"value": round(world * args.steps / el, 4), "unit": UNIT,
               "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8 * n,
               "note": "host wall clock over K steps of a fresh job (built with tn_create from "
                       "the host graph, brought to the same step count untimed): per step "
                       "tn_apply_floquet (theta, 8 bytes, passed by value) and tn_expect_z_all "
                       "into host memory"}
    nbd = {d: int(sum(1 for v in range(n) if int(np.sum(edges == v)) == d)) for d in (1, 2, 3)}
    rl = roofline(prof, args.prec, chi, bp_iters, nbd, solve_kind(args.solve, chi), mp)
    rl["share_of_timed"] = round(prof[rl["kernel"]]["ms"] / ms, 4)
    if not mp:
        rl["peak_source"] = ("not measured in this run (--no-peaks): the peaks file or the "
                             "nominal figure in its place")
    serving = None
    if args.serve_jobs > 0 and rank == 0:
        serving = serve_leg(tn, args)
    batched = None
    if not args.no_batch and rank == 0:
        batched = batch_leg(tn, args)
    serving_mix = None
    if args.serve_mix > 0 and rank == 0:
        serving_mix = serve_mix_leg(tn, args)
    fp32_line = None
    if args.fp32_steps > 0 and args.prec != "fp32":
        s3 = tn.TNState(n, edges, cols, chi=chi, prec="fp32", stream=stream, solve=args.solve)
        s3.apply_floquet(theta, presteps + 1)
        stream.synchronize()
        s3.profile_enable(True)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp32_steps):
            s3.apply_floquet(theta, 1)
        f1.record(stream)
        stream.synchronize()
        fms = f0.elapsed_time(f1)
        fprof = s3.profile()
        s3.profile_enable(False)
        zf = s3.expect_z_all()
        s3.close()
        fp32_line = {"value": round(args.fp32_steps / (fms * 1e-3), 4), "unit": UNIT,
                     "steps": args.fp32_steps, "ms_per_step": round(fms / args.fp32_steps, 3),
                     "kernel_ms": {k: round(v["ms"], 3) for k, v in fprof.items()},
                     "note": "plain FP32 path: CUDA-core FP32 contractions with the same "
                             "truncation solve (%s), same workload and theta, so that "
                             "mixed_over_fp32 compares the contraction precision alone"
                             % SOLVE_NAMES[solve_kind(args.solve, chi)],
                     "mixed_over_fp32": None}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}.get(args.prec, args.prec),
        "data": "synthetic (initial state |0..0>, theta_h from the uniform [0, pi/2] grid)",
        "config": workload_config(args, world),
        "gpu_launches": int(launches),
        "autotune": tune,
        "tma_stream_launches": int(tma_launches),
        "bp_sweeps_per_step": round(bp_iters / args.steps, 2),
        "jacobi_sweeps_per_edge": {"mean": round(jac_sweeps / max(1, jac_edges), 2),
                                   "max": int(jac_max)},
        "discarded_weight_max": disc,
        "roofline": rl,
        "peaks_measured": mp,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
        "clocks": clocks,
        "e2e": e2e,
        "z_mean": float(np.mean(z)),
        "fp32_path": fp32_line,
        "serving": serving, "batched": batched, "serving_mix": serving_mix,
    }
    if fp32_line:
        fp32_line["mixed_over_fp32"] = round(value / world / fp32_line["value"], 3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, det = oracle_step_estimate(chi, bp_iters / args.steps)
        out["cpu_baseline"] = {"value": round(1.0 / sec, 6), "unit": UNIT, "cores": blas_threads(),
                               "kind": "oracle", "estimate": True,
                               "sample": "FP64 NumPy oracle on the 127-qubit chi=%d workload: one BP "
                                         "sweep and %d simple-update gates on a random full-chi "
                                         "state timed, the step estimated as 144 gates + %.1f "
                                         "sweeps (the GPU path's measured count) (sweep %.2f s, "
                                         "gate %.2f s)" % (
                                             chi, det["gates_sampled"], bp_iters / args.steps,
                                             det["t_sweep_s"], det["t_gate_s"])}
        one = oracle_single_thread(chi, bp_iters / args.steps)
        if one is not None:
            sec1, det1 = one
            out["cpu_baseline"]["single_thread"] = {
                "value": round(1.0 / sec1, 6), "unit": UNIT, "cores": 1, "estimate": True,
                "sample": "the same sample with every BLAS/OpenMP pool at one thread (sweep %.2f s, "
                          "gate %.2f s)" % (det1["t_sweep_s"], det1["t_gate_s"])}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if args.config4 and rank == 0:
        print(json.dumps(config4_leg(tn, args)), flush=True)


# ---------------------------------------------------------------- reference
def run_reference(args, rank, world):
    """The FP64 oracle on bounded samples of the workload: each sample times one
    synchronous BP sweep and two simple-update gates on a random full-chi
    127-qubit state; a Floquet step is estimated as 144 gates + 16 sweeps (the
    GPU path's measured count at this workload).  The line is labelled an
    estimate, and `steps` counts the Floquet steps of work actually timed (the
    samples' total time over the per-step estimate), so that steps x
    ms_per_step is the timed work."""
    if rank != 0:
        return
    chi = args.chi
    bp = 16.0
    times, sample_s = [], 0.0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        sec, det = oracle_step_estimate(chi, bp, n_gate_sample=2, seed=100 + i)
        if i >= args.warmup:
            times.append(sec)
            sample_s += time.perf_counter() - t0
    per = float(np.mean(times))
    val = 1.0 / per
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": UNIT,
           "n_gpus": world, "steps": round(sample_s / per, 4), "warmup": args.warmup,
           "ms_per_step": round(per * 1e3, 2), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, world),
           "estimate": True, "samples": args.steps,
           "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": blas_threads(),
                            "kind": "oracle", "estimate": True,
                            "sample": "each of %d samples: one BP sweep + 2 simple-update gates on "
                                      "a random full-chi 127-qubit state; step estimated as 144 "
                                      "gates + %.0f sweeps; steps = equivalent Floquet steps of "
                                      "work timed" % (args.steps, bp)},
           "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def solve_bench(args):
    """The standalone truncation solve on one layer-sized batch: 51 edges at
    chi = 64 (degree-3-like rows: 256 per open environment), seeded complex
    Gaussian environment-weighted site matrices X with spectra decaying as
    exp(-0.05 k), their open-p Gram matrices N_p = X_p^T conj(X_p) as the
    inputs.  Prints one JSON line with the time per call of each solve."""
    import torch
    import paper_2306_14887_gb300 as tn
    from paper_2306_14887_gb300 import build
    build.build()
    chi, ne, rows = 64, 51, 256
    r = np.random.default_rng(5)
    gram = np.zeros((ne, 2, 2, 2, chi, chi), dtype=np.float32)
    for k in range(ne):
        for side in range(2):
            x = r.standard_normal((2, rows, chi)) + 1j * r.standard_normal((2, rows, chi))
            x *= np.exp(-0.05 * np.arange(chi))[None, None, :]
            for p in range(2):
                n_p = x[p].T @ x[p].conj()
                gram[k, side, p, 0], gram[k, side, p, 1] = n_p.real, n_p.imag
    g = torch.from_numpy(gram.reshape(-1)).cuda()
    d = torch.zeros_like(g)
    sv = torch.zeros(ne * chi, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    out = {"leg": "standalone truncation solve, %d edges, chi %d" % (ne, chi)}
    for solve in args.solve_bench.split(","):
        for _ in range(max(args.warmup, 1)):
            tn.truncation_solve(g.data_ptr(), d.data_ptr(), sv.data_ptr(), ne, chi, 1,
                                stream=st.cuda_stream, solve=solve)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            tn.truncation_solve(g.data_ptr(), d.data_ptr(), sv.data_ptr(), ne, chi, 1,
                                stream=st.cuda_stream, solve=solve)
        e1.record(st)
        torch.cuda.synchronize()
        out[solve + "_ms_per_call"] = round(e0.elapsed_time(e1) / args.steps, 4)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.solve_bench:
        if rank == 0:
            solve_bench(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
