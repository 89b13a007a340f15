#!/usr/bin/env python3
"""Benchmark: k-point eigensolves per second for a photonic-crystal band path (kernel-compensated MFD + LOBPCG).

Workload (one "step"): the FCC conventional cubic cell with four eps = 13 spheres (r = 0.25 a) in air, N = 32^3,
the lowest 10 bands at 40 Bloch vectors on Gamma-X-W-K-Gamma-L, LOBPCG to a relative residual of 1e-6 -- every
k-point solved together by one pc_solve call (all hot-path kernels). Synthetic, seeded input; the working set
(~9 GB of search blocks) is larger than L2, so no flush is needed between steps.

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
            line["note"] = ("one CTA per pencil: a launch of a 10-k-point group occupies 10 of the 152 SMs, so the "
                            "fraction of the occupied SMs' FP64 peak is 15.2x frac; the stage time is the interval "
                            "on the group's stream while three other groups share the GPU")
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


def oracle_sample(w, max_iters: int, kidx: int = 3):
    """Times the oracle on one k-point for a bounded number of LOBPCG iterations; returns (seconds, iterations)."""
    from oracle import eigs, geometry
    m0 = 1.0 / geometry.eps_edges(w.N, w.structure.as_array(), w.structure.eps_bg)
    t = time.perf_counter()
    guard = min(w.nbands // 2 + 1, 21 - w.nbands)  # the block size the CUDA solve uses by default
    out = eigs.solve_kpoint(w.N, w.kpts[kidx], m0, w.nbands, w.tol, guard=guard, maxiter=max_iters, max_doublings=0)
    return time.perf_counter() - t, max(1, out["iters"])


def cpu_baseline(w, iters_per_kpoint: float, max_iters: int = 12):
    secs, its = oracle_sample(w, max_iters)
    per_it = secs / its
    value = 1.0 / (per_it * iters_per_kpoint)
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle LOBPCG (numpy/scipy FP64) on k-point 3 of the path for {its} iterations "
                       f"({secs:.1f} s, {per_it:.2f} s/iteration), scaled to {iters_per_kpoint:.1f} iterations per "
                       f"k-point (the mean the GPU solve needed); BLAS on all cores, sparse matvec and FFT "
                       f"single-threaded")}


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    w = wl.workload_fcc_32()
    # iterations per k-point of this workload with the same block size, for the extrapolation: 60 is the mean the
    # CUDA solve measured on this path (59.65 in its FP64 bench line)
    ipk = float(os.environ.get("PC_BENCH_ITERS_PER_KPOINT", "60"))
    times = []
    for s in range(args.warmup + args.steps):
        secs, its = oracle_sample(w, args.ref_iters)
        if s >= args.warmup:
            times.append(secs / its * ipk)
    t = statistics.mean(times)
    value = 1.0 / t
    # n_gpus: the launch this line pairs with (the oracle itself runs on rank 0's host cores, see cpu_baseline)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "nbands": w.nbands, "tol": w.tol, "nk_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"each step: oracle LOBPCG on k-point 3 for {args.ref_iters} iterations, "
                                        f"scaled to {ipk:.0f} iterations per k-point")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_case(args):
    """One hot kernel alone on a small batch (for ncu captures): fcc-spheres-N32 structure, 16 k-points x 16 fields
    (complex64 blocks: 200 MB, complex128: 400 MB -- larger than the 129 MB L2). Prints per-launch event times."""
    import torch

    import paper_2503_19379_gb300 as pc

    w = wl.workload_fcc_32()
    eps = pc.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    solver = pc.Solver(w.N, eps)
    nb, m, N = 16, 16, w.N
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
        k4 = w.kpts[[3, 13, 23, 33]]
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
    ap.add_argument("--ref-iters", type=int, default=12)
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
    w = wl.workload_fcc_32()
    prec = pc.pc.PC_PREC_MIXED if args.precision == "mixed" else pc.pc.PC_PREC_FP64
    eps = pc.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    stream = torch.cuda.current_stream()
    solver = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=prec, groups=args.groups)
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
    total_k = nk * ws if args.scaling == "weak" else len(wl.workload_fcc_32().kpts)
    value = total_k / (ms_step_max / 1e3)
    mean_iters = float(np.mean(np.concatenate(iters)))
    max_iters = int(np.max(np.concatenate(iters)))

    # ---- end to end through the public API with host buffers: setup (eps H2D) + solve (evals D2H)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s2 = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=prec, groups=args.groups)
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

    # ---- the plain FP64 solve of the same workload, for the metric's comparison (fewer steps: ~13 s each)
    fp64_cmp = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        s64 = pc.Solver(w.N, eps, stream=stream.cuda_stream, precision=pc.pc.PC_PREC_FP64)
        s64.solve(w.kpts, w.nbands, w.tol)
        barrier(dist)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        o64 = s64.solve(w.kpts, w.nbands, w.tol)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(f0.elapsed_time(f1), dist)
        ev_m, ev_64 = out["evals"], o64["evals"]
        fp64_cmp = {"value": total_k / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": 1, "warmup": 1,
                    "mean_lobpcg_iterations": float(np.mean(o64["iters"])), "status": int(o64["status"]),
                    "max_rel_eval_diff_vs_chosen": float(np.max(np.abs(ev_m - ev_64) / np.abs(ev_64))),
                    "speedup_of_chosen": value / (total_k / (ms64 / 1e3))}
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
            "config": {"workload": ("fcc-spheres-N32: FCC conventional cell, 4 spheres eps=13 r=0.25a in air, N=32, "
                                    "10 bands, 40 k-points Gamma-X-W-K-Gamma-L, tol 1e-6, all k-points in one "
                                    "batched solve"),
                       "precision": args.precision, "nk_per_gpu": nk, "nbands": w.nbands, "tol": w.tol,
                       "kpoint_groups": args.groups if args.groups > 0 else "library default (4 from 16 k-points)",
                       "mean_lobpcg_iterations": mean_iters, "max_lobpcg_iterations": max_iters,
                       "status": max(statuses),
                       "cache": "inputs larger than L2 (search blocks ~9 GB per GPU), no flush"},
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
        line["cpu_baseline"] = cpu_baseline(w, mean_iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
