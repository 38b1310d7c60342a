"""Throughput of the Q4C real-space integration hot path on GB300.

One step = one pass of the whole hot path over the 64-atom cluster workload
(~1.24M grid points, 800 basis functions): q4c_integrate (V, W0, SO_x,y,z and
the SS spinor blocks), q4c_density with a random P and
q4c_integrate_backward with random G, all in the requested precision.

value = algorithmic FLOPs of the step / device time, where the algorithmic
FLOPs are 14 n_p n_b^2 (integration) + 2 n_p n_b^2 (density) + 14 n_p n_b^2
(adjoint) summed over batches (the useful n_b x n_p x n_b products).

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|fp64]
                       [--impl ours|reference]
Under torchrun with N > 1 every rank runs an independent replica of the
workload (the path is single-GPU by design); value sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Q4C grid integration TFLOP/s (% peak), split-prec vs FP64 at <=1e-9 rel err"
L2_FLUSH_BYTES = 512 << 20


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# DRAM traffic per launch of a kernel group, from the committed ncu summary
# of that kernel; trusted only while the sources it was captured from are
# unchanged (the summary records their sha256).
TRAFFIC_PROFILES = {
    "split_products": ("k_split_products_cluster64.md", ["split.cu", "tc.cuh", "df.cuh", "internal.h"]),
    "split_backward": ("k_split_rowdot_cluster64.md", ["rowdot.cu", "tc.cuh", "df.cuh", "internal.h"]),
    "split_density": ("k_split_rowdot_cluster64.md", ["rowdot.cu", "tc.cuh", "df.cuh", "internal.h"]),
    "split_gslice": ("k_gslice_cluster64.md", ["rowdot.cu", "tc.cuh", "df.cuh", "internal.h"]),
    "basis_df": ("k_basis_df_cluster64.md", ["basis_df.cu", "df.cuh", "internal.h"]),
}


def kernel_source_hash(name: str):
    import hashlib
    ent = TRAFFIC_PROFILES.get(name)
    if ent is None:
        return None
    h = hashlib.sha256()
    for f in ent[1]:
        with open(os.path.join(ROOT, "paper_2608_00773_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(name: str):
    """(bytes per launch, summary file) if the summary matches the current sources, else (None, why)."""
    ent = TRAFFIC_PROFILES.get(name)
    if ent is None:
        return None, "no ncu summary for this kernel"
    path = os.path.join(ROOT, "profiles", ent[0])
    if not os.path.exists(path):
        return None, f"profiles/{ent[0]} missing"
    want, val = None, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith(f"source_sha256[{name}]:"):
                want = line.split(":", 1)[1].strip()
            elif line.startswith(f"traffic_bytes_per_launch[{name}]:"):
                val = float(line.split(":", 1)[1].strip())
    if val is None or want is None:
        return None, f"profiles/{ent[0]} has no traffic line for {name}"
    if want != kernel_source_hash(name):
        return None, f"sources changed since profiles/{ent[0]} was captured"
    return val, f"profiles/{ent[0]}"


# FP64 FMA rate of GB300: 2 DFMA per SM per clock -> 4 flop/clk/SM
def fp64_peak_tflops(sm_mhz: float) -> float:
    return 152 * sm_mhz * 1e6 * 4 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)  # sampling runs before the timed region starts
        except (FileNotFoundError, OSError):
            self.proc = None
        self.t_start = time.perf_counter()
        self.t_end = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop_window(self):
        """End of the timed region: later samples are not counted."""
        self.t_end = time.perf_counter()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t_end = self.t_end if self.t_end is not None else float("inf")
        for t, line in self.lines:
            if not (self.t_start <= t <= t_end):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = float(f[2])
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_molecules_sample(wl, stride: int, threads: int = 1):
    """Batched molecules are independent: one oracle step for every stride-th
    molecule, each on its own grid, pattern and v, the molecules dealt to
    `threads` concurrent parts; returns (wall seconds, fraction of the
    workload's algorithmic FLOPs those molecules carry)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from workloads import ADJOINT_KINDS, fill_pattern, potential
    mols = list(range(0, wl.n_molecules, stride))
    jobs = []
    for m in mols:
        wm = wl.molecule(m)
        xyz, w, ids = O.grid(wm)
        ob = O.OracleBasis(wm)
        pat = ob.pattern()
        P = fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wm.nf_of_atom, 11, "P")
        G = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wm.nf_of_atom, 12, k, a) for k, a in ADJOINT_KINDS]
        jobs.append((ob, pat, xyz, w, potential(xyz, wm), P, G))

    def one(job):
        ob, pat, xyz, w, v, P, G = job
        ob.matrix_blocks(xyz, w, v, pat)
        ob.density(xyz, P, pat)
        ob.adjoint(xyz, w, G, pat)

    t0 = time.perf_counter()
    if threads == 1:
        for j in jobs:
            one(j)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, jobs))
    t = time.perf_counter() - t0
    # the sampled molecules' share of the work: their atoms' functions squared, weighted by atoms
    nf = wl.nf_of_atom.astype(np.float64)
    cost = np.array([float(nf[wl.mol_atom_ptr[m]:wl.mol_atom_ptr[m + 1]].sum()) ** 2 *
                     (wl.mol_atom_ptr[m + 1] - wl.mol_atom_ptr[m]) for m in range(wl.n_molecules)])
    return t, float(cost[mols].sum() / cost.sum())


def oracle_step_sample(wl, stride: int, threads: int = 1):
    """One oracle step (matrices, density, adjoint) on the raw grid points with
    id % stride == 0, the points dealt round-robin to `threads` parts that run
    concurrently (the oracle's C calls release the GIL; each part's sums are
    its own, as in a split of the grid); returns (wall seconds, fraction of
    the workload)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from workloads import ADJOINT_KINDS, fill_pattern, potential
    if getattr(wl, "mol_atom_ptr", None) is not None:
        return oracle_molecules_sample(wl, stride, threads)
    xyz, w, ids = O.grid(wl, stride=stride)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    v = potential(xyz, wl)
    P = fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 11, "P", blk_T=pat.blk_T)
    G = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 12, k, a, blk_T=pat.blk_T)
         for k, a in ADJOINT_KINDS]
    parts = [np.arange(k, len(w), threads) for k in range(threads)]  # interleaved: even cost per thread

    def chunk(k):
        i = parts[k]
        ob.matrix_blocks(xyz[i], w[i], v[i], pat)
        ob.density(xyz[i], P, pat)
        ob.adjoint(xyz[i], w[i], G, pat)

    t0 = time.perf_counter()
    if threads == 1:
        chunk(0)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(chunk, range(threads)))
    return time.perf_counter() - t0, 1.0 / stride


def step_flops(info) -> dict:
    s2 = info.flops_alg / 14.0  # sum over batches of n_p n_b^2
    return {"integrate": 14.0 * s2, "density": 2.0 * s2, "backward": 14.0 * s2}


# ---------------------------------------------------------------------------

def run_reference(args, wl):
    rank, world, _ = dist_init()
    if rank != 0:
        return
    cores = host_cores()
    batched = getattr(wl, "mol_atom_ptr", None) is not None
    if batched:  # independent molecules: the FLOPs of the sampled molecules, each on its own grid
        flops = sum(workload_flops(wl.molecule(m)) for m in range(0, wl.n_molecules, args.ref_stride))
    else:
        flops = workload_flops(wl)
    times, fracs = [], []
    for _ in range(args.warmup):
        oracle_step_sample(wl, args.ref_stride, cores)
    for _ in range(args.steps):
        t, frac = oracle_step_sample(wl, args.ref_stride, cores)
        times.append(t)
        fracs.append(frac)
    t_sample = statistics.mean(times)
    t_step = t_sample / fracs[0]
    val = (flops / t_sample if batched else flops / t_step) / 1e12
    sample = (f"every {args.ref_stride}-th molecule on its own grid" if batched else
              f"raw grid ids divisible by {args.ref_stride}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "note": f"oracle (plain FP64 C, {cores} host threads) on a uniform "
                       f"sample ({sample}), time scaled to the full workload"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample}, split over {cores} threads"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_flops(wl) -> float:
    """Algorithmic FLOPs of one step (30 sum_b n_p n_b^2) counted on the
    oracle's own grid with the batching rule of the method (recursive median
    bisection along the longest bounding-box axis, ties by raw id, until a
    batch holds <= batch_max points; n_b = functions of the atoms strictly
    within r_c of some point of the batch)."""
    import oracle as O
    xyz, w, ids = O.grid(wl)
    nf = wl.nf_of_atom.astype(np.float64)
    total = 0.0
    stack = [np.arange(len(ids))]
    while stack:
        idx = stack.pop()
        if len(idx) <= wl.batch_max:
            P = xyz[idx]
            d2 = ((P[:, None, :] - wl.xyz[None]) ** 2).sum(-1)
            nb = float(nf[(d2 < wl.r_c ** 2).any(axis=0)].sum())
            total += len(idx) * nb * nb
            continue
        P = xyz[idx]
        ax = int(np.argmax(P.max(0) - P.min(0)))
        order = np.lexsort((ids[idx], P[:, ax]))
        mid = len(idx) // 2
        stack.append(idx[order[mid:]])
        stack.append(idx[order[:mid]])
    return 30.0 * total


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="FP64-path steps timed after the split run for the speedup (0: skip)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cluster64",
                    choices=["cluster64", "water", "molecules", "cluster512", "slab", "small_slab"],
                    help="cluster64: the 64-atom cluster (default); molecules: 2,000 independent molecules "
                         "in one grid; cluster512: the 512-atom cluster of the adjoint configuration; slab: "
                         "the 3,383-atom periodic slab; small_slab: its density and batch sizes in a 304-atom "
                         "cell (a profiling case of a few GB)")
    ap.add_argument("--cpu-stride", type=int, default=16, help="one-core sample of the cpu baseline")
    ap.add_argument("--cpu-stride-all", type=int, default=2, help="all-core sample of the cpu baseline")
    ap.add_argument("--ref-stride", type=int, default=7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tile shapes (skip q4c_autotune)")
    ap.add_argument("--separate", action="store_true",
                    help="time the three separate calls instead of the one-pass q4c_scf_pass")
    ap.add_argument("--print-source-hash", action="store_true",
                    help="print the sha256 of each profiled kernel's sources and exit")
    args = ap.parse_args()
    if args.print_source_hash:
        for name in TRAFFIC_PROFILES:
            print(f"source_sha256[{name}]: {kernel_source_hash(name)}")
        return

    from workloads import cluster512, cluster64, molecule_batch, slab, small_slab, water
    wl = {"cluster64": cluster64, "water": water, "molecules": molecule_batch, "cluster512": cluster512,
          "slab": slab, "small_slab": small_slab}[args.workload]()
    big = args.workload in ("molecules", "cluster512", "slab", "small_slab")
    if args.workload == "slab" and args.steps == 60:
        args.steps = 3  # a step of the slab takes seconds
    # sample strides that keep the oracle's share of a run to seconds
    if big:
        default_strides = {"molecules": (200, 20), "cluster512": (4000, 400), "slab": (40000, 0),
                           "small_slab": (4000, 0)}[args.workload]
        if args.cpu_stride == 16:
            args.cpu_stride = default_strides[0]
        if args.cpu_stride_all == 2:
            args.cpu_stride_all = default_strides[1]
    if args.impl == "reference":
        if args.workload in ("cluster512", "slab", "small_slab"):
            print(json.dumps({"impl": "reference", "unavailable": f"the oracle's FLOP count of the {wl.name} workload "
                              "needs its full grid (8 min of host time for the 512-atom cluster, hours for the "
                              "slab), beyond this arm's few-minute bound"}))
            return
        if args.workload == "molecules" and args.ref_stride == 7:
            args.ref_stride = 100
        return run_reference(args, wl)

    import torch

    import paper_2608_00773_gb300 as q
    from workloads import ADJOINT_KINDS, column_operator, fill_pattern, potential

    rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # ---- setup (untimed): tables, grid, inputs
    tables, grid = q.setup(wl)
    ex = grid.export()
    info = grid.info
    pat = (ex["blk_ptr"], ex["blk_col"], ex["blk_off"])
    if getattr(wl, "mol_atom_ptr", None) is not None:  # each point's potential from its own molecule
        from workloads import molecule_potential
        ppa = wl.n_rad * wl.n_theta * wl.n_phi
        v_h = molecule_potential(ex["xyz"], ex["point_id"] // ppa, wl, device=dev)
    else:
        v_h = potential(ex["xyz"], wl, device=dev if grid.n_points > 4_000_000 else None)
    P_h = fill_pattern(*pat, wl.nf_of_atom, 11, "P", blk_T=ex["blk_T"])
    G_h = [fill_pattern(*pat, wl.nf_of_atom, 12, k, a, blk_T=ex["blk_T"]) for k, a in ADJOINT_KINDS]
    v = torch.tensor(v_h, device=dev)
    P = torch.tensor(P_h, device=dev)
    G = [torch.tensor(g, device=dev) for g in G_h]
    nnz, npts = grid.nnz, grid.n_points
    mats = [torch.empty(nnz, dtype=torch.float64, device=dev) for _ in range(5)]
    mats.append(torch.empty(8 * nnz, dtype=torch.float64, device=dev))
    n_out = torch.empty(npts, dtype=torch.float64, device=dev)
    g_out = torch.empty(npts, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    fl = step_flops(info)
    F_step = sum(fl.values())
    stream = torch.cuda.current_stream()

    # tile shapes of the split path, per batch-size bucket, by the library's tuner (setup, untimed)
    tiling = q.q4c_autotune(tables, grid, v) if args.prec == "split" and not args.no_tune else q.q4c_grid_tiling(grid)

    # precision per phase: the requested one where the library provides it
    phase_prec = {}
    for name, fn in (("integrate", lambda p: q.q4c_integrate(tables, grid, v, p, out=mats, stream=stream)),
                     ("density", lambda p: q.q4c_density(tables, grid, P, p, out=n_out, stream=stream)),
                     ("backward", lambda p: q.q4c_integrate_backward(tables, grid, G, p, out=g_out, stream=stream))):
        try:
            fn(args.prec)
            phase_prec[name] = args.prec
        except q.Q4CError as e:
            if e.status != 5:
                raise
            phase_prec[name] = "fp64"
    torch.cuda.synchronize()

    def separate_step():
        q.q4c_integrate(tables, grid, v, phase_prec["integrate"], out=mats, stream=stream)
        q.q4c_density(tables, grid, P, phase_prec["density"], out=n_out, stream=stream)
        q.q4c_integrate_backward(tables, grid, G, phase_prec["backward"], out=g_out, stream=stream)

    # one pass per step (q4c_scf_pass: one basis evaluation per wave for the
    # three parts) where all phases run in one precision
    fused = len(set(phase_prec.values())) == 1 and not args.separate

    def step(_prec=None):
        if not fused:
            return separate_step()
        q.q4c_scf_pass(tables, grid, v, [P, None, None, None, None], G, phase_prec["integrate"], H_out=mats,
                       n_out=n_out, dLdv_out=g_out, stream=stream)

    prec = args.prec
    for _ in range(args.warmup):
        step(prec)
    torch.cuda.synchronize()

    # ---- timed region: device time per step, L2 flushed between steps
    q.profile(True)
    q.profile_read("")  # drop records of earlier calls
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(prec)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clocks.stop_window()
    barrier(world)
    q.profile(False)
    grid.status()  # raises if a bounded wait of a tensor kernel ran out (incomplete outputs)
    per_step = [a.elapsed_time(b) for a, b in ev]
    t_ms = max_over_ranks(statistics.mean(per_step), world)
    kern = {}
    for name in ("split_products", "split_prep", "split_backward", "split_density", "split_gslice", "fill_idx", "basis_df",
                 "products_fp64",
                 "density_fp64", "backward_fp64", "basis", "mirror", "spinor", ""):
        ms, n = q.profile_read(name)
        if n:
            kern[name or "other"] = (ms, n)
    launches_total = sum(n for _, n in kern.values())
    value = world * F_step / (t_ms * 1e-3) / 1e12

    # ---- dominant kernel roofline (algorithmic work of that kernel / its time)
    peaks, peak_src = load_peaks()
    clk = clocks.summary()
    dom_name, (dom_ms, dom_n) = max(kern.items(), key=lambda kv: kv[1][0])
    S_PAIRS = 21  # slice-pair products (s + t <= 5 of 6 BF16 slices per operand)
    if dom_name in ("split_products", "split_backward", "split_density"):
        work = {"split_products": "integrate", "split_backward": "backward", "split_density": "density"}[dom_name]
        achieved = fl[work] * S_PAIRS * args.steps / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16 burst (of {peak_src})",
                "work": f"algorithmic FLOPs of {work} x {S_PAIRS} slice pairs"}
    elif dom_name in ("products_fp64", "density_fp64", "backward_fp64"):
        work = {"products_fp64": "integrate", "density_fp64": "density", "backward_fp64": "backward"}[dom_name]
        calls = sum(1 for ph, pr in phase_prec.items() if ph == work and pr == "fp64") or 1
        achieved = fl[work] * args.steps * calls / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak_tflops(peaks.get("sm_max_mhz", 2070.0)),
                "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 2 DFMA/clk x sm_max_mhz (FP64 ALU)",
                "work": f"algorithmic FLOPs of {work}"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s"}
    roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("achieved") and roof.get("peak") else None
    roof["traffic"], roof["traffic_source"] = measured_traffic(dom_name)
    roof["kernel"] = dom_name
    roof["kernel_ms_per_launch"] = dom_ms / dom_n
    roof["share_of_step"] = dom_ms / (t_ms * args.steps)

    # ---- end to end through the public API: pinned host in, host out
    h_v = torch.from_numpy(v_h).pin_memory()
    h_P = torch.from_numpy(P_h).pin_memory()
    h_G = [torch.from_numpy(g).pin_memory() for g in G_h]
    h_out = [torch.empty(nnz, dtype=torch.float64).pin_memory() for _ in range(5)]
    h_ss = torch.empty(8 * nnz, dtype=torch.float64).pin_memory()
    h_n = torch.empty(npts, dtype=torch.float64).pin_memory()
    h_g = torch.empty(npts, dtype=torch.float64).pin_memory()
    bi = 8 * (h_v.numel() + h_P.numel() + sum(x.numel() for x in h_G))
    bo = 8 * (5 * nnz + 8 * nnz + 2 * npts)

    def e2e_step():
        v.copy_(h_v, non_blocking=True)
        P.copy_(h_P, non_blocking=True)
        for d_, h_ in zip(G, h_G):
            d_.copy_(h_, non_blocking=True)
        step(prec)
        for h_, d_ in zip(h_out, mats[:5]):
            h_.copy_(d_, non_blocking=True)
        h_ss.copy_(mats[5], non_blocking=True)
        h_n.copy_(n_out, non_blocking=True)
        h_g.copy_(g_out, non_blocking=True)
        stream.synchronize()

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    grid.status()
    e2e = {"value": world * F_step / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": bo}

    # ---- the integration alone (q4c_integrate, device time, L2 flushed)
    extra = {}
    if fused:  # the same step as three separate calls, for comparison
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(min(5, args.steps))]
        for a_, b_ in evs:
            flush.zero_()
            a_.record(stream)
            separate_step()
            b_.record(stream)
        torch.cuda.synchronize()
        grid.status()
        extra["separate_calls"] = {"ms_per_step": max_over_ranks(statistics.mean(a_.elapsed_time(b_) for a_, b_ in evs),
                                                                 world), "steps": len(evs)}
    evi = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in evi:
        flush.zero_()
        a_.record(stream)
        q.q4c_integrate(tables, grid, v, phase_prec["integrate"], out=mats, stream=stream)
        b_.record(stream)
    torch.cuda.synchronize()
    grid.status()
    t_int = max_over_ranks(statistics.mean(a_.elapsed_time(b_) for a_, b_ in evi), world)
    tf_int = world * fl["integrate"] / (t_int * 1e-3) / 1e12
    extra["integration_only"] = {
        "what": "q4c_integrate alone (V, W0, SO x,y,z and the SS spinor blocks), algorithmic 14 sum n_p n_b^2",
        "ms_per_call": t_int, "tflops": tf_int,
        "tensor_frac": tf_int * S_PAIRS / peaks["bf16_tflops"] if phase_prec["integrate"] == "split" else None,
        "tensor_frac_note": f"x {S_PAIRS} slice pairs / {peak_src} bf16 burst, whole call incl. basis and scatter"}

    # ---- FP64 comparison path and split error (reported beside the value)
    if big and args.fp64_steps == 3:
        # the FP64 path takes tens of seconds per step there (minutes on the slab)
        args.fp64_steps = 0 if args.workload == "slab" else 1
    if prec == "split" and (args.fp64_steps > 0 or args.workload == "slab"):
        ref = [torch.empty_like(m) for m in mats[:5]]
        q.q4c_integrate(tables, grid, v, "fp64", out=ref + [None], stream=stream)
        q.q4c_integrate(tables, grid, v, "split", out=mats, stream=stream)
        torch.cuda.synchronize()
        extra["split_rel_err_vs_fp64"] = {n: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
                                          for n, a, b in zip(["V", "W0", "SOx", "SOy", "SOz"], mats[:5], ref)}
        if getattr(wl, "mol_atom_ptr", None) is not None:
            # every molecule on its own: the largest relative error over the molecules, per matrix
            offs = ex["blk_off"][ex["blk_ptr"][wl.mol_atom_ptr]]
            worst = {}
            for nme, a, b in zip(["V", "W0", "SOx", "SOy", "SOz"], mats[:5], ref):
                d = (a - b).double() ** 2
                r = b.double() ** 2
                cd = torch.cat([torch.zeros(1, dtype=torch.float64, device=dev), torch.cumsum(d, 0)])
                cr = torch.cat([torch.zeros(1, dtype=torch.float64, device=dev), torch.cumsum(r, 0)])
                o = torch.tensor(offs, device=dev)
                num, den = cd[o[1:]] - cd[o[:-1]], cr[o[1:]] - cr[o[:-1]]
                worst[nme] = float(torch.sqrt(num / torch.clamp(den, min=1e-300)).max())
            extra["split_rel_err_vs_fp64_worst_molecule"] = worst
            extra["molecules"] = int(wl.n_molecules)
        del ref
    if prec == "split" and args.fp64_steps > 0:
        # the same step on the FP64 path (device time, L2 flushed), for the split/FP64 speedup
        fp64_phase = {"integrate": "fp64", "density": "fp64", "backward": "fp64"}

        def step64():
            q.q4c_integrate(tables, grid, v, "fp64", out=mats, stream=stream)
            q.q4c_density(tables, grid, P, "fp64", out=n_out, stream=stream)
            q.q4c_integrate_backward(tables, grid, G, "fp64", out=g_out, stream=stream)
        step64()
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.fp64_steps)]
        for a_, b_ in ev64:
            flush.zero_()
            a_.record(stream)
            step64()
            b_.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev64), world)
        p64 = fp64_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        extra["fp64_path"] = {"ms_per_step": t64, "tflops": world * F_step / (t64 * 1e-3) / 1e12,
                              "peak": p64, "peak_source": "derived: 152 SM x 2 DFMA/clk x sm_max_mhz",
                              "frac": world * F_step / (t64 * 1e-3) / 1e12 / p64,
                              "speedup_split_vs_fp64": t64 / t_ms, "steps": args.fp64_steps,
                              "phase_precision": fp64_phase}
        # the per-column operator of Eq. 19 (one non-symmetric product per
        # batch: 2 n_p n_b^2 algorithmic FLOPs) on both paths, same workload
        eps_c, knots_c = column_operator(wl, 1201)
        q.q4c_tables_set_columns(tables, eps_c, knots_c)
        F_split = torch.empty(nnz, dtype=torch.float64, device=dev)
        F_64 = torch.empty(nnz, dtype=torch.float64, device=dev)
        q.q4c_integrate_columns(tables, grid, v, "split", out=F_split, stream=stream)
        evc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a_, b_ in evc:
            flush.zero_()
            a_.record(stream)
            q.q4c_integrate_columns(tables, grid, v, "split", out=F_split, stream=stream)
            b_.record(stream)
        e64 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        flush.zero_()
        e64[0].record(stream)
        q.q4c_integrate_columns(tables, grid, v, "fp64", out=F_64, stream=stream)
        e64[1].record(stream)
        torch.cuda.synchronize()
        tc = statistics.mean(a_.elapsed_time(b_) for a_, b_ in evc)
        Fc = fl["integrate"] / 7.0
        extra["columns_operator"] = {
            "what": "F_ij = sum_p w phi_i (eps_j - V_j + v) phi_j (Eq. 19), q4c_integrate_columns",
            "split_ms": tc, "split_tflops": Fc / (tc * 1e-3) / 1e12, "fp64_ms": e64[0].elapsed_time(e64[1]),
            "rel_err_split_vs_fp64": float(torch.linalg.norm(F_split - F_64) / torch.linalg.norm(F_64)),
            "steps": len(evc)}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = host_cores()
        t1, f1 = oracle_step_sample(wl, args.cpu_stride, 1)
        single = {"value": F_step * f1 / t1 / 1e12, "cores": 1,
                  "sample": f"raw grid ids divisible by {args.cpu_stride} ({f1:.6f} of the workload), "
                            f"{t1:.1f} s of one core"}
        if args.cpu_stride_all > 0:
            tn, fn_ = oracle_step_sample(wl, args.cpu_stride_all, cores)
            cpu = {"value": F_step * fn_ / tn / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                   "sample": f"raw grid ids divisible by {args.cpu_stride_all} ({fn_:.4f} of the workload) split "
                             f"over {cores} threads, {tn:.1f} s wall", "single_core": single}
        else:  # one part only: each concurrent part would hold its own full-pattern accumulators
            cpu = {"value": single["value"], "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                   "sample": single["sample"] + "; one thread only (the oracle's matrices hold 5 x nnz compensated "
                                                "accumulators per concurrent part, 17 GB here)"}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-split/f32-acc/f64" if prec == "split" else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "atoms": wl.n_atoms, "n_basis": int(info.n_basis),
                   "points": int(info.n_points), "batches": int(info.n_batches), "max_nb": int(info.max_nb),
                   "precision": prec, "phase_precision": phase_prec,
                   "step": ("q4c_scf_pass (integration + density + adjoint, one basis evaluation per wave)"
                            if fused else "q4c_integrate + q4c_density + q4c_integrate_backward"),
                   "l2": "512 MB buffer written between timed steps", "replicas": world},
        "flops_per_step": fl,
        "tiling": [{"kernel": "products" if k < len(tiling) - 1 else "density/adjoint",
                    "nb_max": t["nb_max"] if t["nb_max"] < (1 << 29) else None, "k_steps_per_stage": t["k_steps"],
                    "batches": t["batches"], "tuner_ms": [t["ms_one"], t["ms_two"]]} for k, t in enumerate(tiling)],
        "phase_ms": {k: v_[0] / args.steps for k, v_ in kern.items()},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches_total,
        **extra,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
