#!/usr/bin/env python3
"""Benchmark: k-point eigensolves per second for a photonic-crystal band path (kernel-compensated MFD + LOBPCG).

Workload (one "step" = one pc_solve call over every k-point of the path, all hot-path kernels, from random blocks to
a relative residual of 1e-6), selected by ``--workload``:
- ``diamond-air-N64`` (default): the diamond conventional cell, 8 air spheres r = 0.3 a in eps = 13, N = 64^3, the
  lowest 12 bands at 60 Bloch vectors on Gamma-X-W-K-Gamma-L; the mixed-precision solve against the plain FP64
  solve of the same workload (a stated subset of its k-points, ``--fp64-stride``);
- ``fcc-spheres-N32``: the FCC conventional cell, 4 spheres eps = 13 r = 0.25 a in air, N = 32^3, 10 bands, 40
  k-points on the same path;
- ``fcc-spheres-N128``: the same FCC structure at N = 128^3, 16 bands, 64 k-points, solved in k-point chunks sized
  against the free device memory (``opts.kchunk`` caps them).
Synthetic, seeded input; every working set (search blocks of several GB) is larger than L2, so no flush is needed
between steps.

Prints ONE JSON line (rank 0). Multi-GPU: one process per GPU, each rank solves its own copy of the path
(independent problems, no collective on the data path; weak scaling).

``--impl reference`` times the FP64 CPU oracle (oracle/) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "k-point eigensolves/sec at 1e-6 residual (chosen vs plain FP64); stencil GB/s vs HBM"
UNIT = "k-points/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Double-float arithmetic (mixed_df.cu): one complex multiply-add (8 FP64-equivalent flops) is 4 products
# (mul + 3 fma + 3 for the renormalisation = 7 FP32 operations each) and 4 sums (11 each) = 72 FP32 operations,
# i.e. 9 FP32 operations per FP64-equivalent flop; its ALU peak in FP64-equivalent flops is the FP32 peak / 9.
DF_OPS_PER_FLOP = 9.0


# DRAM traffic per algorithmic byte of a stage's kernel, from an ncu capture of it on a smaller case (committed
# summary named beside it); the bench scales it by the bytes of its own launches. Only for kernels unchanged since.
MEASURED_TRAFFIC = {
    "gram": (1.4211 / 1.4093, "profiles/gram_tc_kernel_coupled48x16_16k_N32.md: dram__bytes_read + "
                              "dram__bytes_write = 1.4211 GB for 1.4093 GB algorithmic (16 k-points x (48 + 48 + 16) "
                              "columns), scaled to the launch"),
}


def stage_roofline(stage, d, precision, peaks, src):
    """Roofline entry for one stage: algorithmic work per launch / average event time of a launch."""
    calls = max(d["calls"], 1)
    t = d["ms"] / calls / 1e3
    if precision == "fp64" or stage in ("rr", "recompute"):
        achieved = d["flops"] / calls / t / 1e12
        line = {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (FP64 CUDA cores)"}
        if stage == "rr":
            line["note"] = ("one CTA per pencil: a launch for a k-point group occupies one SM per active k-point of "
                            "the group, so the fraction of the occupied SMs' FP64 peak is 152 / (active k-points) x "
                            "frac; the stage time is the interval on the group's stream while the other groups "
                            "share the GPU")
        return line
    if stage == "dfloat":
        achieved = d["flops"] / calls / t / 1e12
        peak = FP32_PEAK_TFLOPS / DF_OPS_PER_FLOP
        return {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "derived: FP32 peak (152 SMs x 128 lanes x 2 x 2.07 GHz) / 9 FP32 ops per "
                               "double-float flop"}
    achieved = d["bytes"] / calls / t / 1e9
    peak = float(peaks["hbm_gbs"])
    line = {"bound": "hbm", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"}
    if stage in MEASURED_TRAFFIC:
        ratio, how = MEASURED_TRAFFIC[stage]
        line["traffic"] = ratio * d["bytes"] / calls
        line["traffic_source"] = how
    return line


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(x, dist):
    """Max of a host float over ranks (timing only; never on the solve's data path)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(nk: int, rank: int, ws: int) -> list:
    """Contiguous share of nk independent k-points for one rank (strong scaling); every k-point on exactly one rank."""
    base, extra = divmod(nk, ws)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The benchmark's workloads: (constructor, description for config.workload, default FP64-comparison stride, the
# solve's options). The FP64 comparison solves every stride-th k-point of the path (all of them at stride 1).
WORKLOADS = {
    "diamond-air-N64": (wl.workload_diamond_64,
                        "diamond-air-N64: diamond conventional cell, 8 air spheres r=0.3a (FCC sites and the same "
                        "shifted by (1/4,1/4,1/4)) in eps=13, N=64, 12 bands, 60 k-points Gamma-X-W-K-Gamma-L, "
                        "tol 1e-6, all k-points in one batched solve", 3),
    "fcc-spheres-N32": (wl.workload_fcc_32,
                        "fcc-spheres-N32: FCC conventional cell, 4 spheres eps=13 r=0.25a in air, N=32, 10 bands, 40 "
                        "k-points Gamma-X-W-K-Gamma-L, tol 1e-6, all k-points in one batched solve", 1),
    "fcc-spheres-N128": (wl.workload_fcc_128,
                         "fcc-spheres-N128: FCC conventional cell, 4 spheres eps=13 r=0.25a in air, N=128, 16 bands, "
                         "64 k-points Gamma-X-W-K-Gamma-L, tol 1e-6, k-point chunks sized against the free device "
                         "memory", 16),
}


def make_workload(name: str):
    w = WORKLOADS[name][0]()
    w.kpts = np.ascontiguousarray(w.kpts)
    return w


def oracle_iters_per_kpoint(name: str):
    """The oracle's own LOBPCG iterations per k-point to the workload's tolerance: the mean over the k-points sampled
    in tests/golden/oracle_evals_<workload>.json (written by tests/golden/make_oracle_evals.py, which runs the oracle
    alone). Returns (mean, [(k-index, iterations)])."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_evals_{name}.json")
    rows = []
    if os.path.exists(path):
        with open(path) as f:
            doc = json.load(f)
        rows = [(r["kidx"], r["iters_at_workload_tol"]) for r in doc["kpoints"] if "iters_at_workload_tol" in r]
    if not rows:
        return None, []
    return float(np.mean([r[1] for r in rows])), rows


class OracleStepper:
    """The oracle's LOBPCG (oracle/eigs.py, as it stands) on one k-point of a workload, advanced one call at a time:
    each step is eigs.lobpcg(..., maxiter=1) from the block the previous step returned (a Rayleigh-Ritz on the block,
    one LOBPCG iteration on [X W], the residual): four block applications of the operator and one of the
    preconditioner, the work of one steady-state oracle iteration. Setup (operator, preconditioner symbols, initial
    block) happens in the constructor, outside the timed steps."""

    def __init__(self, w, kidx: int = 3):
        from oracle import eigs, geometry, mfd, precond, rng
        self.w, self.kidx = w, kidx
        N = w.N
        h = 1.0 / N
        m0 = 1.0 / geometry.eps_edges(N, w.structure.as_array(), w.structure.eps_bg)
        k = eigs.reduce_to_first_zone(w.kpts[kidx])
        g = mfd.penalty_gamma(h, k)
        Op = mfd.compensated_operator(N, k, h, m0, g)
        self.apply_A = lambda Y: Op @ Y
        self.apply_T = lambda Y: precond.apply_preconditioner_block(Y, N, h, k, g)
        self.project = eigs.constant_projector(N) if not np.any(k) else None
        m = w.nbands + min(w.nbands // 2 + 1, 21 - w.nbands)  # the block size of the CUDA solve
        self.X = rng.initial_block(0, 0, 3 * N ** 3, m)
        self.eigs = eigs

    def step(self) -> float:
        t = time.perf_counter()
        _, X, _, res = self.eigs.lobpcg(self.apply_A, self.apply_T, self.X, self.w.nbands, self.w.tol, 1, self.project)
        self.X = X
        return time.perf_counter() - t


def cpu_baseline(w, name: str, steps: int = 2):
    """The oracle on the host cores on a bounded sample of the workload: `steps` oracle LOBPCG iterations on one
    k-point, scaled by the oracle's own iterations per k-point."""
    ipk, rows = oracle_iters_per_kpoint(name)
    if ipk is None:
        return None
    st = OracleStepper(w)
    st.step()  # first call: caches and allocations
    secs = [st.step() for _ in range(steps)]
    per_it = float(np.mean(secs))
    return {"value": 1.0 / (per_it * ipk), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle LOBPCG (numpy/scipy FP64) on k-point {st.kidx} of the path: {steps} iterations after "
                       f"one untimed, {per_it:.2f} s each, times {ipk:.1f} iterations per k-point (the oracle's own "
                       f"count to tol {w.tol:g} at k-points {[r[0] for r in rows]}, tests/golden); BLAS on all "
                       f"cores, sparse matvec and FFT single-threaded")}


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    w = make_workload(args.workload)
    ipk, rows = oracle_iters_per_kpoint(args.workload)
    if ipk is None:
        print(json.dumps({"impl": "reference", "unavailable": (f"no oracle iteration count to the tolerance of "
                                                               f"{args.workload} under tests/golden (the oracle takes "
                                                               f"minutes per iteration at N = {w.N})")}), flush=True)
        return
    st = OracleStepper(w)
    iters_per_step = max(1, args.ref_iters)
    times = []
    for s in range(args.warmup + args.steps):
        secs = sum(st.step() for _ in range(iters_per_step))
        if s >= args.warmup:
            times.append(secs)
    t = statistics.mean(times)  # measured seconds per step (iters_per_step oracle iterations)
    value = iters_per_step / (t * ipk)
    sample = (f"each step: {iters_per_step} oracle LOBPCG iteration(s) (eigs.lobpcg with maxiter=1, continuing from "
              f"the previous step's block) on k-point {st.kidx} of the path; k-points/s = iterations per step / "
              f"(seconds per step x {ipk:.1f} oracle iterations per k-point to tol {w.tol:g}, measured by the "
              f"oracle at k-points {[r[0] for r in rows]}, tests/golden)")
    # n_gpus: the launch this line pairs with (the oracle itself runs on rank 0's host cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1], "N": w.N, "nbands": w.nbands, "tol": w.tol,
                       "kpoints_per_step": iters_per_step / ipk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_case(args):
    """One hot kernel alone on a small batch (for ncu captures): fcc-spheres-N32 structure, 16 k-points x 16 fields
    (complex64 blocks: 200 MB, complex128: 400 MB -- larger than the 129 MB L2). Prints per-launch event times."""
    import torch

    import paper_2503_19379_gb300 as pc

    # N = 32: the fcc-spheres-N32 structure, 16 k-points; N = 64: the diamond-air-N64 structure, 4 k-points (the
    # same bytes per launch); 16 fields each
    w = wl.workload_fcc_32() if args.kernel_n == 32 else wl.workload_diamond_64()
    eps = pc.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    solver = pc.Solver(w.N, eps)
    nb, m, N = (16 if w.N == 32 else 4), 16, w.N
    kp = w.kpts[:nb]
    gam = np.full(nb, 2.0 * N)
    dt = torch.complex64 if args.kernel_case.endswith(("32", "32c")) else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((nb, m, 3, N, N, N), dtype=dt, device="cuda", generator=g)
    L = 3 * N ** 3
    if args.kernel_case == "stencil_df":
        X = torch.randn((nb, m, 3, N, N, N), dtype=torch.complex128, device="cuda", generator=g)
        run = lambda: solver.apply_op(kp, gam, X, double_float=True)
    elif args.kernel_case.startswith("stencil"):
        run = lambda: solver.apply_op(kp, gam, X)
    elif args.kernel_case.startswith("precond"):
        Y = torch.empty_like(X)
        run = lambda: solver.apply_precond(kp, gam, X, out=Y)
    elif args.kernel_case == "rr":
        # 40 pencils of size 48 (3 x 16 columns) like one solver iteration: G = S^H S, H = S^H A S
        gr = np.random.default_rng(1)
        Sm = gr.standard_normal((40, 300, 48)) + 1j * gr.standard_normal((40, 300, 48))
        lam = np.linspace(1.0, 1e3, 300)
        Gm = np.einsum("bli,blj->bij", Sm.conj(), Sm)
        Hm = np.einsum("bli,l,blj->bij", Sm.conj(), lam, Sm)
        Gt = torch.from_numpy(Gm).cuda()
        Ht = torch.from_numpy(Hm).cuda()
        run = lambda: pc.rayleigh_ritz(Gt, Ht, 16)
    elif args.kernel_case == "solve4":
        # a mixed-precision solve of 4 k-points of the path: the solver's own kernels at production shapes (the
        # double-float stencil with the residual epilogue on pair storage, the double-float update and Gram)
        s4 = pc.Solver(w.N, eps, precision=pc.pc.PC_PREC_MIXED)
        k4 = w.kpts[[3, 13, 23, 33]] if w.N == 32 else w.kpts[[5, 20, 35, 50]]
        run = lambda: s4.solve(k4, w.nbands, w.tol)
    elif args.kernel_case == "gram32c":
        # the solver's pencil with its coupling block: [X W P] (48 columns), its image, and R (16 columns)
        S = X.reshape(nb, m, L)
        SS = torch.cat([S, S, S], 1).contiguous()
        ASS = torch.cat([S, S, S], 1).contiguous()  # its own buffer, as the operator image is in the solver
        R = S.clone()
        run = lambda: pc.gram_pair_coupled(SS, ASS, R)
    elif args.kernel_case.startswith("gram"):
        S = X.reshape(nb, m, L)
        AS = S.clone()
        SS = torch.cat([S, S, S], 1).contiguous()
        ASS = torch.cat([AS, AS, AS], 1).contiguous()
        run = lambda: pc.gram_pair(SS, ASS)
    else:
        raise SystemExit(f"unknown kernel case {args.kernel_case}")
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"kernel_case": args.kernel_case, "nb": nb, "m": m, "N": N, "ms": times}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="mixed: the chosen precision (complex64 search directions, FP64 block via double-float); "
                         "fp64: the plain FP64 solve")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain-FP64 comparison solve reported beside the chosen precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--groups", type=int, default=0,
                    help="k-point groups of the mixed solve on separate streams (0: the library default)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank solves the whole path (independent replicas); strong: the path's k-points "
                         "are split across ranks")
    ap.add_argument("--workload", default="diamond-air-N64", choices=sorted(WORKLOADS),
                    help="the benchmark configuration (default: the diamond cell at N = 64, 60 k-points, 12 bands)")
    ap.add_argument("--fp64-stride", type=int, default=0,
                    help="the plain-FP64 comparison solves every stride-th k-point of the path (0: the workload's "
                         "default; 1: all)")
    ap.add_argument("--kchunk", type=int, default=0, help="cap on the k-points per pass of pc_solve (0: what fits)")
    ap.add_argument("--ref-iters", type=int, default=1,
                    help="oracle LOBPCG iterations per reference step")
    ap.add_argument("--kernel-n", type=int, default=32, choices=[32, 64],
                    help="grid of the --kernel-case batch (32: 16 k-points, 64: 4 k-points; 16 fields each)")
    ap.add_argument("--kernel-case", default=None,
                    choices=["stencil64", "stencil32", "stencil_df", "precond64", "precond32", "gram64", "gram32",
                             "gram32c", "rr", "solve4"],
                    help="run one hot kernel alone on a small batch (profiling) instead of the benchmark")
    args = ap.parse_args()
    if args.kernel_case:
        kernel_case(args)
        return
    rank, ws, dist = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
        return

    import torch

    import paper_2503_19379_gb300 as pc

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = make_workload(args.workload)
    nk_path = len(w.kpts)
    prec = pc.pc.PC_PREC_MIXED if args.precision == "mixed" else pc.pc.PC_PREC_FP64
    eps = pc.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    stream = torch.cuda.current_stream()
    solver = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=prec, groups=args.groups, kchunk=args.kchunk)
    if args.scaling == "strong" and ws > 1:
        w.kpts = w.kpts[shard(len(w.kpts), rank, ws)]
    nk = len(w.kpts)

    for _ in range(args.warmup):
        out = solver.solve(w.kpts, w.nbands, w.tol)
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    solver.reset_stats()
    solver.set_timing(True)
    clocks = ClockSampler(dev)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, statuses = [], []
    for _ in range(args.steps):
        out = solver.solve(w.kpts, w.nbands, w.tol)
        iters.append(out["iters"].copy())
        statuses.append(out["status"])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    st = solver.stats()
    solver.set_timing(False)
    ms_step_max = max_over_ranks(ms_step, dist)
    total_k = nk * ws if args.scaling == "weak" else nk_path
    value = total_k / (ms_step_max / 1e3)
    mean_iters = float(np.mean(np.concatenate(iters)))
    max_iters = int(np.max(np.concatenate(iters)))

    # ---- end to end through the public API with host buffers: setup (eps H2D) + solve (evals D2H)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s2 = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=prec, groups=args.groups, kchunk=args.kchunk)
        o2 = s2.solve(w.kpts, w.nbands, w.tol)
        s2.close()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / args.steps * 1e3, dist)
    h2d = eps.nbytes + w.kpts.nbytes
    d2h = o2["evals"].nbytes + o2["iters"].nbytes + o2["resid"].nbytes

    # ---- roofline of the dominant stage (and of every stage, for reference)
    peaks, src = load_peaks()
    dom = max(st, key=lambda k: st[k]["ms"])
    roof = stage_roofline(dom, st[dom], args.precision, peaks, src)
    stage_roofs = {k: {kk: v for kk, v in stage_roofline(k, st[k], args.precision, peaks, src).items()
                       if kk in ("bound", "achieved", "unit", "frac")}
                   for k in st if st[k]["calls"] > 0}

    # ---- the plain FP64 solve of the same workload (every stride-th k-point of the path, one timed solve after one
    # untimed one), for the metric's comparison at equal accuracy
    fp64_cmp = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        stride = args.fp64_stride if args.fp64_stride > 0 else WORKLOADS[args.workload][2]
        sel = np.arange(0, nk, stride)
        ksub = np.ascontiguousarray(w.kpts[sel])
        s64 = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=pc.pc.PC_PREC_FP64, kchunk=args.kchunk)
        s64.solve(ksub, w.nbands, w.tol)
        barrier(dist)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        o64 = s64.solve(ksub, w.nbands, w.tol)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(f0.elapsed_time(f1), dist)
        ev_m, ev_64 = out["evals"][sel], o64["evals"]
        v64 = len(sel) * (ws if args.scaling == "weak" else 1) / (ms64 / 1e3)
        fp64_cmp = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": 1, "warmup": 1,
                    "kpoint_indices": [int(x) for x in sel],
                    "lobpcg_iterations_per_kpoint": [int(x) for x in o64["iters"]],
                    "kpoints": (f"every {stride}th k-point of the path ({len(sel)} of {nk}), one batched solve"
                                if stride > 1 else f"all {nk} k-points, one batched solve"),
                    "mean_lobpcg_iterations": float(np.mean(o64["iters"])), "status": int(o64["status"]),
                    "max_fp64_rel_resid": float(np.max(o64["resid"])),
                    "max_rel_eval_diff_vs_chosen": float(np.max(np.abs(ev_m - ev_64) / np.abs(ev_64))),
                    "speedup_of_chosen": value / v64}
        s64.close()
    sten = st["stencil"]
    sten_gbs = sten["bytes"] / max(sten["ms"], 1e-9) / 1e6
    # stage times are CUDA-event intervals on the stream that ran them; the solve's k-point groups run on separate
    # streams, so stage times of different groups overlap and their sum can exceed the wall time
    stages = {k: {"ms_per_step": v["ms"] / args.steps, "calls_per_step": v["calls"] / args.steps,
                  "share": v["ms"] / max(sum(x["ms"] for x in st.values()), 1e-9)} for k, v in st.items()}
    launches = int(sum(v["kernels"] for v in st.values()))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": args.scaling,
            "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else "c64+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1], "N": w.N,
                       "precision": args.precision, "nk_per_gpu": nk, "nbands": w.nbands, "tol": w.tol,
                       "kchunk": args.kchunk if args.kchunk > 0 else "what fits the free device memory",
                       "max_fp64_rel_resid": float(np.max(out["resid"])),
                       "kpoint_groups": args.groups if args.groups > 0 else "library default (4 from 16 k-points)",
                       "mean_lobpcg_iterations": mean_iters, "max_lobpcg_iterations": max_iters,
                       "lobpcg_iterations_per_kpoint": [int(x) for x in iters[-1]],
                       "fp64_finish_kpoints": [int(b) for b in np.nonzero(out["fp64_finish"])[0]],
                       "status": max(statuses),
                       "cache": (f"inputs larger than L2 (search blocks "
                                 f"{(192 if args.precision == 'fp64' else 136) * (w.nbands + min(w.nbands // 2 + 1, 21 - w.nbands)) * 3 * w.N ** 3 * nk / 1e9:.0f} GB per GPU), no flush")},
            "roofline": roof,
            "fp64_comparison": fp64_cmp,
            "stage_rooflines": stage_roofs,
            "stencil": {"achieved_gbs": sten_gbs, "peak_gbs": float(peaks["hbm_gbs"]),
                        "frac": sten_gbs / float(peaks["hbm_gbs"]),
                        "note": "algorithmic bytes (read X, write Op X, M0 once per launch) / event time"},
            "stages": stages,
            "e2e": {"value": total_k / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, args.workload)
        if cb is not None:
            line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
