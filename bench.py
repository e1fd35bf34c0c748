"""Benchmark of the dd Rgemm / Rsyrk hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload default|plain|sliced|crt|grouped|served|potrf|sweep]
                    [--size S]

Default workload: one timed step is dd Rgemm NN, dd Rgemm TN and dd Rsyrk
(uplo U, trans N) at m = n = k = 8192 (the largest size of the plain
configuration), random dd inputs with alpha, beta random dd in [0.5, 2]
(seeded synthetic data), computed by the library's certified split-precision
path (mp_dd_Rgemm_crt / mp_dd_Rsyrk_crt: residues on the fp16 tensor cores,
each call certified on the device to meet the dd Rgemm accuracy bound).  The
metric is dd-GFlops (LAPACK operation counts, one dd add or multiply = one
flop: Rgemm 2mnk, Rsyrk k n (n+1)).  The inputs (8.6 GB per step) are larger
than the 129 MB L2, so no flush is needed between steps.  Beside it, in the
same run: the plain FP64 path on the same three problems (one call each,
CUDA events; 32 s, too slow for the timed loop), the digit-slice form and
the ill-scaled inputs at 8192, the grouped GEMM of 4096 problems and the
served SPD solves, each summarised at the end of the line.

``--workload plain`` times the plain FP64 path alone (the step above on the
FP64 pipe, ``--size``).

Prints one JSON line.  With N > 1 (torchrun, one process per GPU) every rank
runs an independent replica of the step (weak scaling, no collective on the
data path); value = total flops of all ranks / the slowest rank's time.

``--impl reference`` times the CPU oracle (the plain scalar dd loops) on
this host's cores on a bounded sample of the same workload, and prints the
same metric with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

METRIC = "dd-Rgemm/Rsyrk GFlops vs roofline; sliced vs plain at bound; p50/p99 solve ms"
UNIT = "dd-GFlop/s"
# nominal FP64 rate of GB300 (1.25 TFLOP/s counting an FMA as two flops) ->
# 625 G FP64 instructions per second; a dd multiply-add in the GEMM kernels
# costs 12.75 of them (1 DMUL + 3 DFMA + 8 DADD, FastTwoSum every 4 steps)
NOMINAL_FP64_INSTR = 1.25e12 / 2
FP64_OPS_PER_MAC = 12.75
QD_OPS_PER_MAC = 117.5   # qd multiply-add: 113 FP64 operations + 4.5 for the level pass
# dram__bytes_read.sum + dram__bytes_write.sum per launch, from single ncu
# captures of the current kernels (the summaries under profiles/ give the
# commands): the plain Rgemm NN launch at 4096 and the band kernel of the
# CRT form at 8192 (one-pass metrics, 30.20 GB read and 2.14 GB written,
# against 8.59 and 2.15 GB algorithmic)
PLAIN_NN_4096_DRAM_BYTES = 3626772736 + 278080000
BAND_CRT_8192_DRAM_BYTES = 30.20e9 + 2.14e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="default",
                    choices=["default", "plain", "sliced", "crt", "grouped", "served", "potrf",
                             "sweep"])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--groups", type=int, default=4096)
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--no-sections", action="store_true",
                    help="default workload: skip the sliced / grouped / served summaries")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sliced", action="store_true")
    ap.add_argument("--sliced-size", type=int, default=8192)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# workload: plain dd Rgemm NN + Rgemm TN + Rsyrk UN
# ----------------------------------------------------------------------------

class Ranks:
    """One replica per rank under torchrun (RANK / WORLD_SIZE / LOCAL_RANK
    from the environment): the process group, a barrier, the maximum of a
    timing over ranks and the whole-job value.  Every workload here is a set
    of independent problems, so ranks exchange only these scalars."""

    def __init__(self, backend: str | None = None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist

            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist
            self.device = f"cuda:{self.local}" if backend == "nccl" else "cpu"

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        """The largest x over all ranks (every rank gets it)."""
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job(self, units_per_rank: float, seconds_max: float) -> float:
        """Units processed by all ranks per second of the slowest rank."""
        return self.world * units_per_rank / seconds_max

    def close(self) -> None:
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def plain_problems(size: int):
    """The step's three problems as host (numpy) data."""
    nn = datagen.gemm_case(1, "N", "N", size, size, size)
    tn = datagen.gemm_case(2, "T", "N", size, size, size)
    g = datagen.rng(3)
    A = datagen.dd_matrix(g, size, size)
    C = datagen.dd_matrix(g, size, size)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    syrk = dict(uplo="U", trans="N", n=size, k=size, alpha=al, A=A, beta=be, C=C)
    return nn, tn, syrk


def plain_flops(size: int):
    g = 2.0 * size ** 3
    return {"Rgemm_NN": g, "Rgemm_TN": g, "Rsyrk_UN": float(size) * size * (size + 1)}


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"mpdd_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
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
        self.f.close()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None, "reasons": sorted(reasons),
                "samples": len(sms)}


# ----------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------

def run_plain_workload(args):
    """--workload plain: the step on the plain FP64 path at --size, with the
    other routines (Rtrsm, Rsyr2k, Rsymm, Rgetrf, Rpotrf, qd Rgemm) and the
    split-precision sections beside it."""
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks()
    world, rank = ranks.world, ranks.rank
    import paper_2109_13406_gb300 as mp

    size = args.size
    nn, tn, syrk = plain_problems(size)
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    dnn = (dev(nn.A), dev(nn.B), dev(nn.C))
    dtn = (dev(tn.A), dev(tn.B), dev(tn.C))
    dsy = (dev(syrk["A"]), dev(syrk["C"]))
    stream = torch.cuda.current_stream()
    # per-kernel events on the launching stream
    names = ["Rgemm_NN", "Rgemm_TN", "Rsyrk_UN"]
    ev = {n: [] for n in names}

    def step(record=False):
        for nm, c, (A, B, C) in (("Rgemm_NN", nn, dnn), ("Rgemm_TN", tn, dtn)):
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            mp.mp_dd_Rgemm(c.transa, c.transb, size, size, size, c.alpha, A, size, B, size,
                           c.beta, C, size)
            if record:
                e1.record(stream)
                ev[nm].append((e0, e1))
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        mp.mp_dd_Rsyrk("U", "N", size, size, syrk["alpha"], dsy[0], size, syrk["beta"], dsy[1],
                       size)
        if record:
            e1.record(stream)
            ev["Rsyrk_UN"].append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peak_fp64 = mp.mp_dd_peak_fp64() if rank == 0 else None
    ranks.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ranks.max(t0.elapsed_time(t1))
    flops = plain_flops(size)
    step_flops = sum(flops.values())
    value = ranks.whole_job(step_flops * args.steps, ms * 1e-3) / 1e9
    per = {}
    for nm in names:
        t = [a.elapsed_time(b) for a, b in ev[nm]]
        avg = sum(t) / len(t)
        per[nm] = {"ms": avg, "GFlops": flops[nm] / (avg * 1e-3) / 1e9}
    # dominant kernel: the Rgemm NN launch; algorithmic FP64 instructions
    nn_ms = per["Rgemm_NN"]["ms"]
    achieved = FP64_OPS_PER_MAC * float(size) ** 3 / (nn_ms * 1e-3) / 1e9
    roofline = {
        "bound": "alu", "kernel": "dd_gemm_plain_kernel<0,0> (Rgemm NN)",
        "achieved": achieved, "peak": NOMINAL_FP64_INSTR / 1e9, "unit": "GFP64instr/s",
        "frac": achieved / (NOMINAL_FP64_INSTR / 1e9),
        "peak_source": "nominal GB300 FP64 1.25 TFLOP/s = 625 G FP64 instr/s (derived)",
        "peak_measured_fp64_microbench": (peak_fp64 / 1e9) if peak_fp64 else None,
        "frac_of_measured": (achieved / (peak_fp64 / 1e9)) if peak_fp64 else None,
        # DRAM bytes of one Rgemm NN launch at 4096 from one ncu capture of
        # this kernel (profiles/dd_gemm_plain_4096.md); None at other sizes
        "traffic": PLAIN_NN_4096_DRAM_BYTES if size == 4096 else None,
        "fp64_instr_per_dd_mac": FP64_OPS_PER_MAC,
    }
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, mp, torch, nn, tn, syrk, ranks)
    sliced = None
    if not args.no_sliced:
        del dnn, dtn, dsy
        torch.cuda.empty_cache()
        sliced = {"vs_plain_2048": sliced_section(mp, torch, 2048, compare_plain=True),
                  "well_scaled": sliced_section(mp, torch, args.sliced_size),
                  "ill_scaled_outer": sliced_section(mp, torch, args.sliced_size, ill="outer"),
                  "crt_vs_plain_2048": sliced_section(mp, torch, 2048, compare_plain=True,
                                                      form="crt"),
                  "crt_well_scaled": sliced_section(mp, torch, args.sliced_size, form="crt"),
                  "crt_ill_scaled_outer": sliced_section(mp, torch, args.sliced_size,
                                                         ill="outer", form="crt"),
                  "crt_rsyrk": syrk_crt_section(mp, torch, args.sliced_size)}
    routines = None
    if not args.no_sliced:
        routines = routines_section(mp, torch, size)
    if rank == 0:
        cpu = None if args.no_cpu or world > 1 else cpu_baseline(size, budget_s=15.0)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64; dd entries hi~U(-1,1), lo=hi*2^-53*U(-1,1) "
                    "renormalised; alpha,beta random dd in [0.5,2])",
            "config": {"workload": f"plain dd path: Rgemm NN + Rgemm TN + Rsyrk U/N, "
                                   f"m=n=k={size}", "m": size, "n": size, "k": size,
                       "l2": f"inputs {3 * 3 * 2 * 8 * size * size / 1e6:.0f} MB > 129 MB L2, "
                             "no flush", "parallelism": f"replicas x{world}"},
            "per_call": per,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "sliced": sliced,
            "routines": routines,
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


# ----------------------------------------------------------------------------
# default workload: the step on the certified split-precision path at 8192,
# with the plain path, the other configurations and their summaries
# ----------------------------------------------------------------------------

def _sig(x, digits=4):
    """x rounded to a few significant digits (compact summaries)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or x != x:
        return x
    from math import floor, log10

    return round(float(x), -int(floor(log10(abs(x)))) + digits - 1)


def fp64_peak_line(r64):
    """The plain kernel's ceiling in dd-GFlop/s under the accounting of the
    plain path's roofline: 2 R64 / 15 (15 FP64 instructions per dd
    multiply-add, R64 the measured FP64 issue rate)."""
    return 2.0 * r64 / 15.0 / 1e9


def plain_section(mp, torch, size, problems, r64, rmac=None):
    """The plain FP64 path on the step's three problems, one call each timed
    with CUDA events (after the split-precision runs on the same inputs).
    Fractions: of 2 R64 / 15 (the survey's accounting, R64 the measured FP64
    FMA rate), of the FP64 pipe at the kernel's 12.75 instructions per
    multiply-add, and of the measured rate of the kernel's own multiply-add
    mix with operands in registers (mp_dd_peak_ddmac)."""
    nn, tn, syrk, dnn, dtn, dsy = problems
    st = torch.cuda.current_stream()
    flops = plain_flops(size)
    out = {}
    calls = (("Rgemm_NN", lambda: mp.mp_dd_Rgemm("N", "N", size, size, size, nn.alpha,
                                                  dnn[0], size, dnn[1], size, nn.beta, dnn[2],
                                                  size)),
             ("Rgemm_TN", lambda: mp.mp_dd_Rgemm("T", "N", size, size, size, tn.alpha,
                                                  dtn[0], size, dtn[1], size, tn.beta, dtn[2],
                                                  size)),
             ("Rsyrk_UN", lambda: mp.mp_dd_Rsyrk("U", "N", size, size, syrk["alpha"], dsy[0],
                                                  size, syrk["beta"], dsy[1], size)))
    ceiling = fp64_peak_line(r64) if r64 else None
    for nm, fn in calls:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gf = flops[nm] / (ms * 1e-3) / 1e9
        macs = flops[nm] / 2.0
        instr = FP64_OPS_PER_MAC * macs / (ms * 1e-3)
        out[nm] = {"ms": ms, "dd_GFlops": gf,
                   "frac_of_2R64_over_15": gf / ceiling if ceiling else None,
                   "fp64_pipe_frac": instr / r64 if r64 else None,
                   "frac_of_mac_mix_ceiling": gf / (2.0 * rmac / 1e9) if rmac else None}
    return out


def certified_step_calls(mp, size, problems, ws):
    """The three calls of the default step on the certified split-precision
    path (the library's residue-form Rgemm / Rsyrk)."""
    nn, tn, syrk, dnn, dtn, dsy = problems
    wsb = ws.numel()
    return (
        ("Rgemm_NN", lambda A=dnn[0], B=dnn[1], C=dnn[2]: mp.mp_dd_Rgemm_crt(
            "N", "N", size, size, size, nn.alpha, A, size, B, size, nn.beta, C, size, ws, wsb)),
        ("Rgemm_TN", lambda A=dtn[0], B=dtn[1], C=dtn[2]: mp.mp_dd_Rgemm_crt(
            "T", "N", size, size, size, tn.alpha, A, size, B, size, tn.beta, C, size, ws, wsb)),
        ("Rsyrk_UN", lambda A=dsy[0], C=dsy[1]: mp.mp_dd_Rsyrk_crt(
            "U", "N", size, size, syrk["alpha"], A, size, syrk["beta"], C, size, ws, wsb)),
    )


def certified_e2e(args, mp, torch, problems, ws, ranks):
    """The default step through the public API from pinned host buffers:
    every step copies its inputs to the device, runs the three certified
    calls and copies the three results back; host-side wall clock.  The
    copies are pipelined with the products: inputs go in on one stream and
    results come out on another, ordered by events against the compute
    stream, and the device operands alternate between two sets so that a
    step's inputs land while the previous step's products run."""
    size = args.size
    nn, tn, syrk, dnn, dtn, dsy = problems

    def pin(pair):
        return [torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T)).pin_memory()
                for x in pair]

    names = ("Rgemm_NN", "Rgemm_TN", "Rsyrk_UN")
    host = {"Rgemm_NN": [pin(nn.A), pin(nn.B), pin(nn.C)],
            "Rgemm_TN": [pin(tn.A), pin(tn.B), pin(tn.C)],
            "Rsyrk_UN": [pin(syrk["A"]), pin(syrk["C"])]}
    outs = {nm: [torch.empty_like(h[-1][0]).pin_memory(), torch.empty_like(h[-1][1]).pin_memory()]
            for nm, h in host.items()}
    twin = lambda mats: tuple(tuple(torch.empty_like(x) for x in pair) for pair in mats)
    sets = [(dnn, dtn, dsy), (twin(dnn), twin(dtn), twin(dsy))]
    devs = [dict(zip(names, st)) for st in sets]
    calls = [dict(certified_step_calls(mp, size, (nn, tn, syrk) + st, ws)) for st in sets]
    cs = torch.cuda.current_stream()
    hs, ds = torch.cuda.Stream(), torch.cuda.Stream()
    freed = {}   # (set, call) -> event: the set's C of that call has been read back

    def step(k):
        b = k % 2
        ev_in = {}
        with torch.cuda.stream(hs):
            for nm in names:
                if (b, nm) in freed:
                    hs.wait_event(freed[(b, nm)])
                for hp, dp in zip(host[nm], devs[b][nm]):
                    for h, d in zip(hp, dp):
                        d.copy_(h.view(d.shape[1], d.shape[0]).t(), non_blocking=True)
                ev_in[nm] = torch.cuda.Event()
                ev_in[nm].record(hs)
        ev_done = {}
        for nm in names:
            cs.wait_event(ev_in[nm])
            calls[b][nm]()
            ev_done[nm] = torch.cuda.Event()
            ev_done[nm].record(cs)
        with torch.cuda.stream(ds):
            for nm in names:
                ds.wait_event(ev_done[nm])
                for h, d in zip(outs[nm], devs[b][nm][-1]):
                    h.view(d.shape[1], d.shape[0]).t().copy_(d, non_blocking=True)
                freed[(b, nm)] = torch.cuda.Event()
                freed[(b, nm)].record(ds)

    step(0)
    step(1)
    torch.cuda.synchronize()
    ranks.barrier()
    # at least 12 steps: the first step's input copy and the last step's
    # read-back have no products to overlap, and are spread over the run
    steps = max(12, args.steps)
    t0 = time.perf_counter()
    for k in range(steps):
        step(k)
    torch.cuda.synchronize()
    dt = ranks.max(time.perf_counter() - t0)
    per_mat = 16 * size * size
    flops = sum(plain_flops(size).values())
    return {"value": ranks.whole_job(flops * steps, dt) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": 8 * per_mat, "d2h_bytes_per_step": 3 * per_mat,
            "steps": steps,
            "api": "Python binding mp_dd_Rgemm_crt / mp_dd_Rsyrk_crt, pinned host buffers "
                   "copied in and the results copied out inside the timed region, the copies "
                   "on two streams overlapping the products (two device operand sets)"}


def run_default(args):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks()
    world, rank = ranks.world, ranks.rank
    import paper_2109_13406_gb300 as mp

    size = args.size
    nn, tn, syrk = plain_problems(size)
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    problems = (nn, tn, syrk, (dev(nn.A), dev(nn.B), dev(nn.C)),
                (dev(tn.A), dev(tn.B), dev(tn.C)), (dev(syrk["A"]), dev(syrk["C"])))
    ws = mp.workspace(max(mp.mp_dd_Rgemm_crt_workspace(size, size, size),
                          mp.mp_dd_Rsyrk_crt_workspace(size, size)))
    calls = certified_step_calls(mp, size, problems, ws)
    st = torch.cuda.current_stream()

    def step():
        for _, fn in calls:
            fn()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    r64 = mp.mp_dd_peak_fp64()
    r8 = mp.mp_dd_peak_imma()
    rmac = mp.mp_dd_peak_ddmac()
    ranks.barrier()
    torch.cuda.synchronize()
    mp.mp_dd_sliced_timing(True)      # per-call phase events on this stream
    clk = ClockSampler(local)
    clk.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(args.steps):
        step()
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    log = mp.mp_dd_sliced_phase_log(3 * args.steps)
    mp.mp_dd_sliced_timing(False)
    ms = ranks.max(t0.elapsed_time(t1))
    flops = plain_flops(size)
    step_flops = sum(flops.values())
    value = ranks.whole_job(step_flops * args.steps, ms * 1e-3) / 1e9
    # per-call times and certificates (one more call of each, then its report)
    per = {}
    for q, (nm, fn) in enumerate(calls):
        rows = [log[3 * s_ + q] for s_ in range(args.steps)]
        tot = [sum(r) for r in rows]
        avg = sum(tot) / len(tot)
        fn()
        rep = mp.mp_dd_split_report(ws)
        per[nm] = {"ms": avg, "dd_GFlops": flops[nm] / (avg * 1e-3) / 1e9,
                   "phase_ms": {"scale_certify_residues": sum(r[0] for r in rows) / len(rows),
                                "tensor_products": sum(r[1] for r in rows) / len(rows),
                                "reconstruct_epilogue": sum(r[2] for r in rows) / len(rows)},
                   "width_bits": rep["width_bits"], "moduli": rep["count"],
                   "max_err_est": rep["max_err_est"], "status": rep["status"]}
    # dominant kernel: the residue products of the two Rgemm calls
    L = mp.mp_dd_crt_layout(size, size, size)
    nmod = per["Rgemm_NN"]["moduli"]
    band_flops = 2.0 * L["m_pad"] * L["n_pad"] * L["k_pad"] * nmod
    band_ms = (per["Rgemm_NN"]["phase_ms"]["tensor_products"] +
               per["Rgemm_TN"]["phase_ms"]["tensor_products"]) / 2
    peak, src = tensor_peak_tflops()
    achieved = band_flops / (band_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "kernel": "band_gemm_kernel<256> (residue products of the "
                "Rgemm NN / TN calls)", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": src,
                "algorithmic_flops_per_launch": band_flops,
                "traffic": BAND_CRT_8192_DRAM_BYTES if size == 8192 else None,
                "traffic_note": "dram__bytes_read.sum + write.sum of one launch (ncu); null "
                                "when the kernel changed since the capture"}
    e2e = None if args.no_e2e else certified_e2e(args, mp, torch, problems, ws, ranks)
    plain = plain_section(mp, torch, size, problems, r64, rmac)
    del problems, calls, ws
    torch.cuda.empty_cache()
    sections = {}
    if not args.no_sections:
        sections["config2_8192"] = {
            "crt_well_scaled": sliced_section(mp, torch, size, form="crt"),
            "crt_ill_scaled_outer": sliced_section(mp, torch, size, ill="outer", form="crt"),
            "sliced_well_scaled": sliced_section(mp, torch, size, slices=0)}
        sections["config3_grouped"] = grouped_section(mp, torch, ranks, args.groups, 3, 5)
        sections["config4_served"] = served_section(mp, torch, ranks, args.requests, args.load)
    if rank == 0:
        cpu = None if args.no_cpu or world > 1 else cpu_baseline(size, budget_s=15.0)
        gemm_ceiling = fp64_peak_line(r64)
        summary = {
            "config1_8192_certified": {
                "dd_GFlops": _sig(value), "band_frac_of_bf16_peak": _sig(roofline["frac"]),
                "width_bits": per["Rgemm_NN"]["width_bits"],
                "max_err_est": _sig(max(p["max_err_est"] for p in per.values()))},
            "config1_8192_plain": {
                nm: {"ms": _sig(v["ms"]), "dd_GFlops": _sig(v["dd_GFlops"]),
                     "frac_of_2R64_over_15": _sig(v["frac_of_2R64_over_15"]),
                     "fp64_pipe_frac": _sig(v["fp64_pipe_frac"]),
                     "frac_of_mac_mix": _sig(v["frac_of_mac_mix_ceiling"])}
                for nm, v in plain.items()},
            "certified_over_plain": _sig(plain["Rgemm_NN"]["ms"] / per["Rgemm_NN"]["ms"]),
        }
        if sections:
            c2 = sections["config2_8192"]
            summary["config2_8192"] = {
                k: {"ms": _sig(v["ms"]), "dd_TFlops": _sig(v["dd_GFlops"] / 1e3),
                    "width_bits": v["width_bits"], "max_err_est": _sig(v["max_err_est"]),
                    "band_frac": _sig(v["roofline_band_kernel"]["frac"])}
                for k, v in c2.items()}
            g = sections["config3_grouped"]
            summary["config3_grouped_4096"] = {
                "replay_ms": _sig(g["ms"]), "dd_GFlops": _sig(g["dd_GFlops"]),
                "loop_ms": _sig(g["per_problem_loop"]["ms"]),
                "speedup_over_loop": _sig(g["per_problem_loop"]["speedup_graph_over_loop"]),
                "frac_of_2R64_over_15": _sig(g["dd_GFlops"] / gemm_ceiling)}
            sv = sections["config4_served"]
            summary["config4_served_2000"] = {
                "p50_ms": _sig(sv["p50_ms"]), "p99_ms": _sig(sv["p99_ms"]),
                "solves_per_s": _sig(sv["solves_per_s"]), "dd_GFlops": _sig(sv["dd_GFlops"]),
                "max_residual_ratio": _sig(max(r["ratio"] for r in
                                               sv["residual_ratio_sample"]))}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 tensor (exact integer residues) + i64 + f64",
            "data": "synthetic (seeded PCG64; dd entries hi~U(-1,1), lo=hi*2^-53*U(-1,1) "
                    "renormalised; alpha,beta random dd in [0.5,2])",
            "config": {"workload": f"dd Rgemm NN + Rgemm TN + Rsyrk U/N, m=n=k={size}, on the "
                                   "certified split-precision path (residue form, fp16 tensor "
                                   "cores, accuracy bound certified per call)",
                       "m": size, "n": size, "k": size,
                       "l2": f"inputs {8 * 16 * size * size / 1e9:.1f} GB per step > 129 MB "
                             "L2, no flush", "parallelism": f"replicas x{world}"},
            "per_call": per,
            "measured_peaks": {"fp64_instr_per_s": r64, "imma_int8_ops_per_s": r8,
                               "dd_mac_mix_per_s": rmac,
                               "plain_ceiling_dd_GFlops_2R64_over_15": gemm_ceiling,
                               "plain_mac_mix_ceiling_dd_GFlops": 2.0 * rmac / 1e9},
            "plain_fp64_8192": plain,
            "sections": sections,
            "cpu_baseline": cpu,
            "e2e": e2e,
            # per step 10 + 10 + 9 launches: each Rgemm runs maxima x2, magnitude
            # planes x2, the magnitude product, residues x2, the products, the
            # reconstruction and the gated plain kernel; the Rsyrk one operand's
            # worth of those plus two triangle tables
            "gpu_launches": 29 * args.steps,
            "clocks": clocks,
            "roofline": roofline,
            "summary": summary,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


def _event_ms(torch, st, fn, reset=None, reps=2):
    """Mean CUDA-event time of fn() on stream st after one untimed call;
    reset() (untimed) restores the inputs before every call."""
    if reset:
        reset()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if reset:
            reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sum(ts) / len(ts)


def _fp64_line(workload, ms, flops, macs):
    """dd-GFlop/s and the FP64-pipe roofline of one routine call: the FP64
    work is its multiply-adds at the plain kernel's instructions per
    multiply-add."""
    instr = FP64_OPS_PER_MAC * macs / (ms * 1e-3) / 1e9
    return {"workload": workload, "ms": ms, "dd_GFlops": flops / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "achieved": instr, "peak": NOMINAL_FP64_INSTR / 1e9,
                         "unit": "GFP64instr/s", "frac": instr / (NOMINAL_FP64_INSTR / 1e9),
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s = 625 G FP64 "
                                        "instr/s (derived)"}}


def potrf_section(mp, torch, n, info=None, reps=3):
    """Rpotrf on the FP64 pipe and with the updates on the tensor cores
    (mp_dd_Rpotrf_crt), uplo 'U', on a diagonally dominant SPD matrix
    (symmetric U(-1,1) dd + 2n I), each timed with CUDA events (n^3 / 3
    flops)."""
    st = torch.cuda.current_stream()
    if info is None:
        info = torch.zeros(1, dtype=torch.int64, device="cuda")
    Sh, Sl = datagen.dd_matrix(datagen.rng(6), n, n)
    Sh = np.asfortranarray(np.triu(Sh) + np.triu(Sh, 1).T + 2.0 * n * np.eye(n))
    Sl = np.asfortranarray(np.triu(Sl) + np.triu(Sl, 1).T)
    S0 = tuple(mp.to_device(x) for x in (Sh, Sl))
    S = tuple(x.clone() for x in S0)

    def reset_s():
        for x, y in zip(S, S0):
            x.copy_(y)
    out = {}
    ms = _event_ms(torch, st, lambda: mp.mp_dd_Rpotrf("U", n, S, n, info), reset_s, reps)
    out[f"Rpotrf_U_{n}"] = _fp64_line(f"dd Rpotrf uplo=U, n={n}, diagonally dominant SPD", ms,
                                      float(n) ** 3 / 3, float(n) ** 3 / 6)
    out[f"Rpotrf_U_{n}"]["info"] = int(info.item())
    ws = mp.workspace(max(1, mp.mp_dd_Rpotrf_crt_workspace(n)))
    ms_c = _event_ms(torch, st, lambda: mp.mp_dd_Rpotrf_crt("U", n, S, n, info, ws, ws.numel()),
                     reset_s, reps)
    out[f"Rpotrf_crt_U_{n}"] = {
        "workload": f"dd Rpotrf uplo=U, n={n}, outer steps of 256 columns; panel and trailing "
                    "updates of >= 512 columns as residue-form Rgemm / Rsyrk on the fp16 tensor "
                    "cores", "ms": ms_c,
        "dd_GFlops": float(n) ** 3 / 3 / (ms_c * 1e-3) / 1e9, "speedup_vs_fp64_pipe": ms / ms_c,
        "info": int(info.item())}
    return out


def run_sweep_workload(args):
    """--workload sweep: the plain dd path over the square sizes of the plain
    configuration (Rgemm NN / TN at m = n = k in {1024, 2048, 4096, 8192},
    Rsyrk U/N at n = k in {1024, 4096, 8192}; alpha, beta random dd in
    [0.5, 2]) beside the residue-form (CRT) Rgemm / Rsyrk on the same
    inputs, each call timed with CUDA events (one untimed call first)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    import paper_2109_13406_gb300 as mp

    st = torch.cuda.current_stream()
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    rows = []
    gemm_sizes = (1024, 2048, 4096, 8192)
    syrk_sizes = (1024, 4096, 8192)
    for n in sorted(set(gemm_sizes) | set(syrk_sizes)):
        g = datagen.rng(11 + n)
        A, B, C = (dev(datagen.dd_matrix(g, n, n)) for _ in range(3))
        al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
        ws = mp.workspace(max(mp.mp_dd_Rgemm_crt_workspace(n, n, n),
                              mp.mp_dd_Rsyrk_crt_workspace(n, n)))
        reps = 1 if n >= 8192 else 2
        calls = []
        if n in gemm_sizes:
            for ta in ("N", "T"):
                calls.append((f"Rgemm_{ta}N", 2.0 * n ** 3, float(n) ** 3,
                              lambda ta=ta: mp.mp_dd_Rgemm(ta, "N", n, n, n, al, A, n, B, n, be,
                                                           C, n),
                              lambda ta=ta: mp.mp_dd_Rgemm_crt(ta, "N", n, n, n, al, A, n, B, n,
                                                               be, C, n, ws, ws.numel())))
        if n in syrk_sizes:
            calls.append(("Rsyrk_UN", float(n) * n * (n + 1), float(n) * n * (n + 1) / 2,
                          lambda: mp.mp_dd_Rsyrk("U", "N", n, n, al, A, n, be, C, n),
                          lambda: mp.mp_dd_Rsyrk_crt("U", "N", n, n, al, A, n, be, C, n, ws,
                                                     ws.numel())))
        for name, flops, macs, plain, crt in calls:
            ms = ranks.max(_event_ms(torch, st, plain, reps=reps))
            ms_c = ranks.max(_event_ms(torch, st, crt, reps=3))
            line = _fp64_line(f"dd {name} n={n}", ms, flops, macs)
            rows.append({"call": name, "n": n, "plain_ms": ms,
                         "plain_dd_GFlops": line["dd_GFlops"],
                         "plain_fp64_frac": line["roofline"]["frac"], "crt_ms": ms_c,
                         "crt_dd_GFlops": flops / (ms_c * 1e-3) / 1e9,
                         "crt_over_plain": ms / ms_c,
                         "workspace_status": mp.mp_dd_workspace_status(ws)})
        del A, B, C, ws
        torch.cuda.empty_cache()
    big = [r for r in rows if r["call"] == "Rgemm_NN" and r["n"] == max(gemm_sizes)][0]
    line = {"metric": "dd Rgemm/Rsyrk size sweep: plain FP64-pipe and residue-form dd-GFlop/s",
            "value": ranks.whole_job(big["plain_dd_GFlops"], 1.0), "unit": "dd-GFlop/s",
            "n_gpus": ranks.world, "steps": 1, "warmup": 1, "ms_per_step": big["plain_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64; dd entries hi~U(-1,1), lo=hi*2^-53*U(-1,1) "
                    "renormalised; alpha,beta random dd in [0.5,2])",
            "config": {"workload": "plain dd Rgemm NN/TN m=n=k in {1024,2048,4096,8192}, Rsyrk "
                                   "U/N n=k in {1024,4096,8192}; CRT form on the same inputs",
                       "value_is": "Rgemm NN 8192, plain"},
            "sweep": rows}
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def run_potrf_workload(args):
    """--workload potrf: the two Rpotrf forms at --size (default 4096)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    import paper_2109_13406_gb300 as mp

    n = args.size
    potrf_section(mp, torch, min(n, 512), reps=1)          # warm-up, untimed
    ranks.barrier()
    res = potrf_section(mp, torch, n, reps=max(1, args.steps))
    crt, fp = res[f"Rpotrf_crt_U_{n}"], res[f"Rpotrf_U_{n}"]
    ms = ranks.max(crt["ms"])
    line = {"metric": "dd Rpotrf GFlops (tensor-core updates)",
            "value": ranks.whole_job(float(n) ** 3 / 3 / 1e9, ms * 1e-3), "unit": "dd-GFlop/s",
            "n_gpus": ranks.world, "steps": max(1, args.steps), "warmup": 1, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64; symmetric U(-1,1) dd + 2n I)",
            "config": {"workload": crt["workload"], "n": n}, "fp64_pipe": fp,
            "speedup_vs_fp64_pipe": crt["speedup_vs_fp64_pipe"],
            "all_info_zero": crt["info"] == 0 and fp["info"] == 0}
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def routines_section(mp, torch, size):
    """The other routines at m = n = k = size, each timed with CUDA events on
    the launching stream: dd Rtrsm (two variants), Rsyr2k, Rsymm, Rgetrf,
    Rpotrf (FP64 pipe and tensor-core updates), and the quad-double Rgemm at
    min(size, 1024).  Flops are the LAPACK counts (Rtrsm n^3, Rsyr2k
    2 k n (n+1), Rsymm 2 n^3, Rgetrf 2 n^3 / 3, Rpotrf n^3 / 3, Rgemm
    2 n^3)."""
    st = torch.cuda.current_stream()
    n = size
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    out = {}
    for side, uplo, transa in (("L", "U", "N"), ("R", "L", "T")):
        c = datagen.trsm_case(3, side, uplo, transa, "N", n, n)
        A, B0 = dev(c.A), dev(c.B)
        B = tuple(x.clone() for x in B0)

        def reset():
            for x, y in zip(B, B0):
                x.copy_(y)
        ms = _event_ms(torch, st, lambda: mp.mp_dd_Rtrsm(side, uplo, transa, "N", n, n, c.alpha,
                                                         A, n, B, n), reset)
        out[f"Rtrsm_{side}{uplo}{transa}N_{n}"] = _fp64_line(
            f"dd Rtrsm side={side} uplo={uplo} transa={transa} diag=N, m=n={n}, diagonally "
            "dominant A", ms, float(n) ** 3, float(n) ** 3 / 2)
        del A, B0, B
    g = datagen.rng(4)
    A, B, C = (dev(datagen.dd_matrix(g, n, n)) for _ in range(3))
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    ms = _event_ms(torch, st, lambda: mp.mp_dd_Rsyr2k("U", "N", n, n, al, A, n, B, n, be, C, n))
    out[f"Rsyr2k_UN_{n}"] = _fp64_line(f"dd Rsyr2k uplo=U trans=N, n=k={n}", ms,
                                       2.0 * n * n * (n + 1), float(n) * n * (n + 1))
    ms = _event_ms(torch, st, lambda: mp.mp_dd_Rsymm("L", "U", n, n, al, A, n, B, n, be, C, n))
    out[f"Rsymm_LU_{n}"] = _fp64_line(f"dd Rsymm side=L uplo=U, m=n={n}", ms, 2.0 * n ** 3,
                                      float(n) ** 3)
    A0 = tuple(x.clone() for x in A)
    ipiv = torch.zeros(n, dtype=torch.int64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")

    def reset_lu():
        for x, y in zip(A, A0):
            x.copy_(y)
    ms = _event_ms(torch, st, lambda: mp.mp_dd_Rgetrf(n, n, A, n, ipiv, info), reset_lu)
    out[f"Rgetrf_{n}"] = _fp64_line(f"dd Rgetrf (partial pivoting), m=n={n}, U(-1,1) entries",
                                    ms, 2.0 * n ** 3 / 3, float(n) ** 3 / 3)
    out[f"Rgetrf_{n}"]["info"] = int(info.item())
    del A, B, C, A0
    out.update(potrf_section(mp, torch, n, info))
    # quad-double Rgemm (117.5 FP64 instructions per qd multiply-add)
    nq = min(n, 1024)
    gq = datagen.rng(5)
    Aq, Bq, Cq = (dev(datagen.qd_matrix(gq, nq, nq)) for _ in range(3))
    aq, bq = datagen.qd_scalar(gq), datagen.qd_scalar(gq)
    ms = _event_ms(torch, st, lambda: mp.mp_qd_Rgemm("N", "N", nq, nq, nq, aq, Aq, nq, Bq, nq,
                                                     bq, Cq, nq))
    line = _fp64_line(f"qd Rgemm NN m=n=k={nq}, qd entries x0~U(-1,1)", ms, 2.0 * nq ** 3,
                      float(nq) ** 3)
    instr = QD_OPS_PER_MAC * float(nq) ** 3 / (ms * 1e-3) / 1e9
    line["qd_GFlops"] = line.pop("dd_GFlops")
    line["roofline"].update(achieved=instr, frac=instr / (NOMINAL_FP64_INSTR / 1e9))
    line["fp64_instr_per_qd_mac"] = QD_OPS_PER_MAC
    out[f"qd_Rgemm_NN_{nq}"] = line
    return out


# ----------------------------------------------------------------------------
# sliced (split-precision, tensor-core) dd Rgemm
# ----------------------------------------------------------------------------

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


def tensor_peak_tflops():
    """Measured dense bf16 peak (burst) of the GB300s; fp16 runs at the
    same nominal rate, so it is the fp16 denominator too."""
    try:
        return float(json.load(open(MEASURED))["bf16_tflops"]), "measured (bf16 burst, = fp16 rate)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback (1.9 PFLOP/s bf16 burst)"


def syrk_crt_section(mp, torch, size, reps=3):
    """mp_dd_Rsyrk_crt U/N at n = k = size (dd-flops k n (n+1)) with CUDA
    events on the launching stream, and its per-phase times."""
    g = datagen.rng(6)
    A = tuple(mp.to_device(x) for x in datagen.dd_matrix(g, size, size))
    C = tuple(mp.to_device(x) for x in datagen.dd_matrix(g, size, size))
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(size, size))
    st = torch.cuda.current_stream()

    def call():
        mp.mp_dd_Rsyrk_crt("U", "N", size, size, al, A, size, be, C, size, ws, ws.numel())

    ms = _event_ms(torch, st, call, reps=reps)
    mp.mp_dd_sliced_timing(True)
    call()
    phases = mp.mp_dd_sliced_phase_ms()
    mp.mp_dd_sliced_timing(False)
    flops = float(size) * size * (size + 1)
    return {"workload": f"split-precision dd Rsyrk U/N n=k={size}, CRT form, upper triangle",
            "ms": ms, "dd_GFlops": flops / (ms * 1e-3) / 1e9,
            "phase_ms": {"scale_and_split": phases[0], "band_products": phases[1],
                         "recombine_epilogue": phases[2]},
            "status": mp.mp_dd_workspace_status(ws)}


def sliced_section(mp, torch, size, reps=3, slices=14, ill=None, compare_plain=False,
                   form="slices"):
    """Time the split-precision Rgemm (NN, m=n=k=size) -- ``form`` "slices"
    (mp_dd_Rgemm_sliced; 14 digits, 105 pair products, or chosen per call
    with slices = 0) or "crt" (mp_dd_Rgemm_crt, residues mod 32 moduli at
    112 bits) -- with CUDA events on the launching stream; per-phase times
    from the library's own events; the width and error estimate from the
    call's certificate."""
    c = datagen.gemm_case(2, "N", "N", size, size, size, ill=ill)
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    if form == "crt":
        ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(size, size, size))
    else:
        ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(size, size, size, slices))
    st = torch.cuda.current_stream()

    def call(Cout):
        if form == "crt":
            mp.mp_dd_Rgemm_crt("N", "N", size, size, size, c.alpha, A, size, B, size, c.beta,
                               Cout, size, ws, ws.numel())
        else:
            mp.mp_dd_Rgemm_sliced("N", "N", size, size, size, c.alpha, A, size, B, size,
                                  c.beta, Cout, size, slices, ws, ws.numel())

    C0 = tuple(x.clone() for x in C)
    call(C0)
    torch.cuda.synchronize()
    rep = mp.mp_dd_split_report(ws)
    status = rep["status"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mp.mp_dd_sliced_timing(True)
    phases = []
    e0.record(st)
    for _ in range(reps):
        Ct = tuple(x.clone() for x in C)
        call(Ct)
    e1.record(st)
    torch.cuda.synchronize()
    # per-phase times of the last call (clones sit between calls, not inside)
    phases = mp.mp_dd_sliced_phase_ms()
    mp.mp_dd_sliced_timing(False)
    total_ms = sum(phases)
    if form == "crt":
        L = mp.mp_dd_crt_layout(size, size, size)
        pairs = rep["count"]
    else:
        L = mp.mp_dd_sliced_layout(size, size, size, slices)
        pairs = rep["count"] * (rep["count"] + 1) // 2
    band_flops = 2.0 * L["m_pad"] * L["n_pad"] * L["k_pad"] * pairs
    peak, src = tensor_peak_tflops()
    achieved = band_flops / (phases[1] * 1e-3) / 1e12
    what = (f"CRT form, {pairs} moduli" if form == "crt"
            else f"sliced form, {rep['count']} slices ({pairs} pair products)")
    out = {
        "workload": f"split-precision dd Rgemm NN m=n=k={size}, {what}, "
                    f"{'well-scaled' if ill is None else ill + ' ill-scaled'}",
        "ms": total_ms, "dd_GFlops": 2.0 * size ** 3 / (total_ms * 1e-3) / 1e9,
        "phase_ms": {"scale_and_slice": phases[0], "band_products": phases[1],
                     "recombine_epilogue": phases[2]},
        "status": status, "width_bits": rep["width_bits"], "max_err_est": rep["max_err_est"],
        "roofline_band_kernel": {"bound": "tensor", "kernel": "band_gemm_kernel",
                                 "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                 "frac": achieved / peak, "peak_source": src,
                                 "algorithmic_flops": band_flops,
                                 "traffic": (BAND_CRT_8192_DRAM_BYTES
                                             if form == "crt" and size == 8192 else None)},
    }
    if compare_plain:
        # the plain FP64 path on the same inputs, and their agreement measured
        # against the accuracy bound (numpy |A||B| on sampled entries)
        Cp = tuple(x.clone() for x in C)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(st)
        mp.mp_dd_Rgemm("N", "N", size, size, size, c.alpha, A, size, B, size, c.beta, Cp, size)
        p1.record(st)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        g = datagen.rng(5)
        rows = g.integers(0, size, 512)
        cols = g.integers(0, size, 512)
        s_h, s_l = (mp.to_numpy(x)[rows, cols] for x in C0)
        p_h, p_l = (mp.to_numpy(x)[rows, cols] for x in Cp)
        ab = np.einsum("ij,ji->i", np.abs(c.A[0][rows, :]), np.abs(c.B[0][:, cols]))
        bound = 4 * size * 2.0 ** -104 * (abs(c.alpha[0]) * ab + abs(c.beta[0]) *
                                          np.abs(c.C[0][rows, cols])) * (1 + 2.0 ** -40)
        diff = np.abs((s_h - p_h) + (s_l - p_l))
        out["plain"] = {"ms": plain_ms, "dd_GFlops": 2.0 * size ** 3 / (plain_ms * 1e-3) / 1e9,
                        "speedup_sliced_over_plain": plain_ms / total_ms,
                        "max_abs_diff_over_bound_512_entries": float(np.max(diff / bound))}
    del A, B, C, C0, ws
    torch.cuda.empty_cache()
    return out


def run_e2e(args, mp, torch, nn, tn, syrk, ranks):
    """The same step through the host-buffer entry points (pinned host
    memory), host<->device copies inside the timed region."""
    size = args.size

    def pin(pair):
        out = []
        for x in pair:
            t = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T)).pin_memory()
            out.append(t)
        return out

    hnn = [pin(nn.A), pin(nn.B), pin(nn.C)]
    htn = [pin(tn.A), pin(tn.B), pin(tn.C)]
    hsy = [pin(syrk["A"]), pin(syrk["C"])]
    steps = max(1, min(args.steps, 3))

    walls = {"Rgemm_NN": [], "Rgemm_TN": [], "Rsyrk_UN": []}

    def step():
        for nm, c, (A, B, C) in (("Rgemm_NN", nn, hnn), ("Rgemm_TN", tn, htn)):
            t = time.perf_counter()
            mp.mp_dd_Rgemm_host(c.transa, c.transb, size, size, size, c.alpha, A, size, B, size,
                                c.beta, C, size)
            walls[nm].append(time.perf_counter() - t)
        t = time.perf_counter()
        mp.mp_dd_Rsyrk_host("U", "N", size, size, syrk["alpha"], hsy[0], size, syrk["beta"],
                            hsy[1], size)
        walls["Rsyrk_UN"].append(time.perf_counter() - t)

    step()
    torch.cuda.synchronize()
    ranks.barrier()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = ranks.max(time.perf_counter() - t0)
    clocks = clk.stop()
    per_mat = 16 * size * size
    h2d = 2 * 3 * per_mat + 2 * per_mat      # two GEMMs (A, B, C) + Rsyrk (A, C)
    d2h = 3 * per_mat
    flops = sum(plain_flops(size).values())
    return {"value": ranks.whole_job(flops * steps, dt) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "api": "mp_dd_Rgemm_host / mp_dd_Rsyrk_host (pinned host buffers)",
            "per_call_ms": {nm: 1e3 * sum(v[1:]) / max(1, len(v) - 1) for nm, v in walls.items()},
            "clocks": clocks}


# ----------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ----------------------------------------------------------------------------

def cpu_sample(size: int, cols: int):
    """A column panel of the Rgemm NN problem: C[:, :cols] with full k."""
    c = datagen.gemm_case(1, "N", "N", size, size, size)
    B = (c.B[0][:, :cols], c.B[1][:, :cols])
    C = (c.C[0][:, :cols], c.C[1][:, :cols])
    return c, B, C


def cpu_baseline(size: int, budget_s: float = 15.0):
    import oracle

    threads = oracle.num_threads()
    # calibrate on a narrow panel (one column per thread), then size the
    # sample to the time budget in whole multiples of the thread count
    cols = max(1, threads)
    c, B, C = cpu_sample(size, cols)
    t0 = time.perf_counter()
    oracle.dd_gemm("N", "N", c.alpha, c.A, B, c.beta, C, size, cols, size)
    dt = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(dt, 1e-3)))
    cols = int(min(size, cols * reps))
    c, B, C = cpu_sample(size, cols)
    t0 = time.perf_counter()
    oracle.dd_gemm("N", "N", c.alpha, c.A, B, c.beta, C, size, cols, size)
    dt = time.perf_counter() - t0
    return {"value": 2.0 * size * cols * size / dt / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle", "seconds": dt,
            "sample": f"scalar dd Rgemm NN, C[:, :{cols}] of the {size}^3 problem (full k)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    size = args.size
    threads = oracle.num_threads()
    cols = max(1, threads)          # one output column per host thread per step
    c, B, C = cpu_sample(size, cols)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.dd_gemm("N", "N", c.alpha, c.A, B, c.beta, C, size, cols, size)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    value = 2.0 * size * cols * size / per / 1e9
    sample = f"scalar dd Rgemm NN, C[:, :{cols}] of the {size}^3 problem (full k) per step"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": f"dd Rgemm NN + Rgemm TN + Rsyrk U/N, m=n=k={size}: timed on "
                               f"a sample, the CPU oracle's scalar dd Rgemm NN on the column "
                               f"panel C[:, :{cols}] (full k) per step",
                   "m": size, "n": size, "k": size, "sample_columns": cols},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sliced_workload(args):
    """--workload sliced: one step = one sliced dd Rgemm NN at m=n=k=size
    (well-scaled inputs); value in dd-GFlop/s; e2e through the Python
    binding with pinned host buffers copied in and the result copied out."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    import paper_2109_13406_gb300 as mp

    size, S = args.sliced_size, 14
    crt = args.workload == "crt"
    c = datagen.gemm_case(2, "N", "N", size, size, size)
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(size, size, size) if crt else
                      mp.mp_dd_Rgemm_sliced_workspace(size, size, size, S))
    st = torch.cuda.current_stream()

    def gemm(Ax, Bx, Cx):
        if crt:
            mp.mp_dd_Rgemm_crt("N", "N", size, size, size, c.alpha, Ax, size, Bx, size, c.beta,
                               Cx, size, ws, ws.numel())
        else:
            mp.mp_dd_Rgemm_sliced("N", "N", size, size, size, c.alpha, Ax, size, Bx, size,
                                  c.beta, Cx, size, S, ws, ws.numel())

    def step():
        gemm(A, B, C)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ranks.barrier()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(args.steps):
        step()
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ranks.max(t0.elapsed_time(t1))
    value = ranks.whole_job(2.0 * size ** 3 * args.steps, ms * 1e-3) / 1e9
    # per-phase times (the library's own events) from two more calls after
    # the timed region
    band = []
    for _ in range(2):
        mp.mp_dd_sliced_timing(True)
        step()
        band.append(mp.mp_dd_sliced_phase_ms())
    mp.mp_dd_sliced_timing(False)
    # the products the certified call ran: its moduli count (CRT) or the
    # digit pairs of its slice count (sliced form), from the call's report
    rep = mp.mp_dd_split_report(ws)
    if crt:
        L = mp.mp_dd_crt_layout(size, size, size)
        products = rep["count"]
    else:
        L = mp.mp_dd_sliced_layout(size, size, size, S)
        products = rep["count"] * (rep["count"] + 1) // 2
    band_ms = sum(b[1] for b in band) / len(band)
    flops = 2.0 * L["m_pad"] * L["n_pad"] * L["k_pad"] * products
    peak, src = tensor_peak_tflops()
    ach = flops / (band_ms * 1e-3) / 1e12
    # e2e: pinned host inputs -> device -> sliced Rgemm -> host result
    pin = lambda pair: [torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T))
                        .pin_memory() for x in pair]
    hA, hB, hC = pin(c.A), pin(c.B), pin(c.C)
    hOut = [torch.empty_like(hC[0]).pin_memory(), torch.empty_like(hC[1]).pin_memory()]
    dA = [torch.empty_like(x, device="cuda") for x in hA]
    dB = [torch.empty_like(x, device="cuda") for x in hB]
    dC = [torch.empty_like(x, device="cuda") for x in hC]

    def e2e_step():
        for d, h in zip(dA + dB + dC, hA + hB + hC):
            d.copy_(h, non_blocking=True)
        gemm((dA[0], dA[1]), (dB[0], dB[1]), (dC[0], dC[1]))
        for h, d in zip(hOut, dC):
            h.copy_(d, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ranks.barrier()
    tt = time.perf_counter()
    n_e2e = max(1, min(args.steps, 3))
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    dt = ranks.max(time.perf_counter() - tt)
    mat = 16 * size * size
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ranks.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 tensor (exact integer slices) + i64",
        "data": "synthetic (seeded PCG64; dd entries hi~U(-1,1), lo=hi*2^-53*U(-1,1) "
                "renormalised; alpha,beta random dd in [0.5,2])",
        "config": {"workload": (f"split-precision dd Rgemm NN m=n=k={size}, " +
                                (f"CRT form, {products} moduli" if crt else
                                 f"sliced form, {S} slices") + ", well-scaled"),
                   "m": size, "n": size, "k": size, "products": products,
                   "l2": f"inputs {3 * mat / 1e6:.0f} MB > 129 MB L2, no flush"},
        "roofline": {"bound": "tensor", "kernel": "band_gemm_kernel", "achieved": ach,
                     "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "peak_source": src,
                     "traffic": BAND_CRT_8192_DRAM_BYTES if crt and size == 8192 else None},
        "phase_ms": {"scale_and_split": band[-1][0], "tensor_products": band[-1][1],
                     "recombine_epilogue": band[-1][2]},
        "e2e": {"value": ranks.whole_job(2.0 * size ** 3 * n_e2e, dt) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": 3 * mat, "d2h_bytes_per_step": mat,
                "api": "Python binding mp_dd_Rgemm_" + ("crt" if crt else "sliced") +
                       ", pinned host buffers"},
        "gpu_launches": 6 * args.steps, "clocks": clocks,  # maxima x2, split x2, products, recombination
    }
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def grouped_problems_host(count: int, seed: int = 0):
    """Config of the grouped workload: m, n, k log-uniform integers in
    [16, 512], NN, alpha/beta random dd in [0.5, 2], entries as elsewhere."""
    sizes = datagen.grouped_problems(seed, count)
    return [datagen.gemm_case(100000 + i, "N", "N", int(m), int(n), int(k))
            for i, (m, n, k) in enumerate(sizes)]


def grouped_section(mp, torch, ranks, groups, warmup=3, steps=5):
    """The grouped workload: ``groups`` problems (m, n, k log-uniform in
    [16, 512], NN) in one CUDA-graph replay of the persistent grouped kernel,
    against a loop of one mp_dd_Rgemm call per problem and the library's
    default (untuned) tile shapes."""
    from paper_2109_13406_gb300 import grouped as gr

    cases = grouped_problems_host(groups)
    dev = lambda pair: tuple(mp.to_device(x) for x in pair)
    devs = [(dev(c.A), dev(c.B), dev(c.C)) for c in cases]
    problems = [(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, B, c.beta, C)
                for c, (A, B, C) in zip(cases, devs)]
    t_tune = time.perf_counter()
    table = gr.autotune()
    t_tune = time.perf_counter() - t_tune
    G = gr.GroupedGemm(problems, table)
    G.capture()
    for _ in range(warmup):
        G.replay()
    torch.cuda.synchronize()
    ranks.barrier()
    st = torch.cuda.current_stream()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        G.replay()
    e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ranks.max(e0.elapsed_time(e1)) / steps
    # per-problem launch loop on the same problems
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(st)
    for c, (A, B, C) in zip(cases, devs):
        mp.mp_dd_Rgemm("N", "N", c.m, c.n, c.k, c.alpha, A, c.m, B, c.k, c.beta, C, c.m)
    l1.record(st)
    torch.cuda.synchronize()
    loop_ms = l0.elapsed_time(l1)
    # untuned group (library default shapes) for comparison
    Gd = gr.GroupedGemm(problems, None)
    Gd.run()
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(st)
    Gd.run()
    d1.record(st)
    torch.cuda.synchronize()
    default_ms = d0.elapsed_time(d1)
    flops = G.flops
    macs = flops / 2.0
    nbytes = sum(16.0 * (c.m * c.k + c.k * c.n + 2 * c.m * c.n) for c in cases)
    achieved = FP64_OPS_PER_MAC * macs / (ms * 1e-3) / 1e9
    out = {
        "workload": f"grouped dd Rgemm, {groups} problems, one CUDA-graph launch of the "
                    "persistent kernel", "problems": groups, "total_dd_flops": flops,
        "ms": ms, "steps": steps, "dd_GFlops": ranks.whole_job(flops, ms * 1e-3) / 1e9,
        "l2": f"operands {nbytes / 1e9:.2f} GB > 129 MB L2, no flush",
        "roofline": {"bound": "alu", "kernel": "grouped_gemm_kernel", "achieved": achieved,
                     "peak": NOMINAL_FP64_INSTR / 1e9, "unit": "GFP64instr/s",
                     "frac": achieved / (NOMINAL_FP64_INSTR / 1e9),
                     "peak_source": "nominal GB300 FP64 1.25 TFLOP/s = 625 G FP64 instr/s "
                                    "(derived)", "traffic": None,
                     "useful_over_padded_macs": macs / G.padded_macs()},
        "hbm_GBs": nbytes / (ms * 1e-3) / 1e9,
        "per_problem_loop": {"ms": loop_ms, "dd_GFlops": flops / (loop_ms * 1e-3) / 1e9,
                             "launches": len(cases), "speedup_graph_over_loop": loop_ms / ms},
        "untuned_default_shapes_ms": default_ms,
        "autotune_seconds": t_tune, "clocks": clocks,
    }
    del G, Gd, devs, problems
    torch.cuda.empty_cache()
    return out


def run_grouped_workload(args):
    """--workload grouped: one step = the whole group of ``--groups``
    problems in one CUDA-graph replay of the persistent grouped kernel; the
    per-problem launch loop (one mp_dd_Rgemm call each) is timed beside it."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    import paper_2109_13406_gb300 as mp

    g = grouped_section(mp, torch, ranks, args.groups, args.warmup, args.steps)
    line = {
        "metric": METRIC, "value": g["dd_GFlops"], "unit": UNIT, "n_gpus": ranks.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; m,n,k log-uniform integers in [16,512], NN, random dd "
                "alpha/beta in [0.5,2])",
        "config": {"workload": g["workload"], "problems": args.groups,
                   "total_dd_flops": g["total_dd_flops"], "l2": g["l2"]},
        "roofline": g["roofline"], "hbm_GBs": g["hbm_GBs"],
        "per_problem_loop": g["per_problem_loop"],
        "untuned_default_shapes_ms": g["untuned_default_shapes_ms"],
        "autotune_seconds": g["autotune_seconds"],
        "gpu_launches": 2 * args.steps, "clocks": g["clocks"],
    }
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def served_section(mp, torch, ranks, requests, load):
    """Poisson arrivals of ``requests`` SPD solves (F = Rsyrk(G), Rpotrf(F),
    Rpotrs with 4 dd right-hand sides), n log-uniform in [64, 2048],
    continuous batching under a 120 GB budget; p50/p99 latency (arrival to
    result on the host), solves/s, dd-GFlop/s and LAPACK residual ratios of a
    size-stratified sample (residuals by the library's dd Rgemm; the tests
    check served solutions against the oracle's exact residuals)."""
    from paper_2109_13406_gb300 import grouped as gr
    from paper_2109_13406_gb300.server import Request, SpdServer, residual_ratio

    table = gr.autotune()
    sizes = datagen.request_sizes(0, requests)

    def req(i, n, arrival):
        return Request(rid=i, n=int(n), G=None, B=None, arrival=float(arrival),
                       loader=lambda i=i, n=n: datagen.spd_request_device(1000 + i, int(n)))

    # warm-up (first use of the generator and of every kernel), untimed
    SpdServer(table=table).serve([req(10 ** 7 + i, n, 0.0) for i, n in enumerate((64, 200))])
    torch.cuda.synchronize()
    # calibration: the solo throughput of a batch admitted at once
    cal_sizes = datagen.request_sizes(99, 24)
    t0 = time.perf_counter()
    SpdServer(table=table).serve([req(10 ** 6 + i, n, 0.0) for i, n in enumerate(cal_sizes)])
    cal_s = time.perf_counter() - t0
    cal_flops = sum(2 * n * n * (n + 1) + n ** 3 / 3 + 8 * n * n for n in cal_sizes)
    mean_flops = float(np.mean([2 * n * n * (n + 1) + n ** 3 / 3 + 8 * n * n for n in sizes]))
    solo_rate = cal_flops / cal_s / mean_flops          # solves/s at this size mix
    rate = load * solo_rate
    arrivals = datagen.poisson_arrivals(0, requests, rate)
    reqs = [req(i, n, a) for i, (n, a) in enumerate(zip(sizes, arrivals))]
    srv = SpdServer(budget_bytes=120e9, slots=256, table=table)
    ranks.barrier()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    t0 = time.perf_counter()
    done = srv.serve(reqs)
    wall = ranks.max(time.perf_counter() - t0)
    clocks = clk.stop()
    lat = np.array([(r.done_t - r.arrival) * 1e3 for r in done])
    wait = np.array([(r.admit_t - r.arrival) * 1e3 for r in done])
    serv = np.array([(r.done_t - r.admit_t) * 1e3 for r in done])
    big = np.array([r.n >= 1024 for r in done])
    makespan = ranks.max(max(r.done_t for r in done))
    # each replica serves its own copy of the stream: latencies are those of
    # the slowest replica, throughput adds up
    p50, p99 = (ranks.max(float(np.percentile(lat, q))) for q in (50, 99))
    flops = sum(r.flops() for r in done)
    # residual ratios on a size-stratified sample
    order = sorted(done, key=lambda r: r.n)
    sample = [order[int(q)] for q in np.linspace(0, len(order) - 1, 8)]
    ratios = []
    for r in sample:
        (gh, gl), (bh, bl) = datagen.spd_request_device(1000 + r.rid, r.n)
        n = r.n
        F = mp.dd_empty(n, n, fill=0.0)
        mp.mp_dd_Rsyrk("U", "N", n, 2 * n, (1.0, 0.0), (gh, gl), n, (0.0, 0.0), F, n)
        torch.cuda.synchronize()
        fh, fl = mp.to_numpy(F[0]), mp.to_numpy(F[1])
        Fs = (np.triu(fh) + np.triu(fh, 1).T, np.triu(fl) + np.triu(fl, 1).T)
        ratios.append({"n": n, "ratio": residual_ratio(Fs, r.X, (mp.to_numpy(bh),
                                                                 mp.to_numpy(bl)), mp)})
    return {
        "workload": f"served dd SPD solves: {requests} Poisson arrivals, n log-uniform in "
                    "[64, 2048], Rsyrk -> Rpotrf -> Rpotrs (4 rhs), 120 GB budget, 256 slots",
        "arrival_rate_per_s": rate, "offered_load": load, "solo_rate_solves_per_s": solo_rate,
        "wall_ms": wall * 1e3, "p50_ms": p50, "p99_ms": p99,
        "admission_wait_ms": {"p50": ranks.max(float(np.percentile(wait, 50))),
                              "p99": ranks.max(float(np.percentile(wait, 99)))},
        "service_ms": {"p50": ranks.max(float(np.percentile(serv, 50))),
                       "p99": ranks.max(float(np.percentile(serv, 99))),
                       "p50_n_ge_1024": ranks.max(float(np.percentile(serv[big], 50)))
                       if big.any() else None},
        "mean_ms": float(lat.mean()), "solves_per_s": ranks.whole_job(len(done), makespan),
        "dd_GFlops": ranks.whole_job(flops, makespan) / 1e9, "scheduler_steps": srv.steps,
        "launches": srv.launches, "max_concurrent": srv.max_active,
        "all_info_zero": all(r.info == 0 for r in done),
        "residual_ratio_sample": ratios,
        "residual_by": "the library's dd Rgemm (LAPACK ratio ||B - F X||_1 / "
                       "(||F||_1 ||X||_1 2^-104))", "clocks": clocks,
    }


def run_served_workload(args):
    """--workload served: the served SPD solves alone (see served_section)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    import paper_2109_13406_gb300 as mp

    sv = served_section(mp, torch, ranks, args.requests, args.load)
    line = {
        "metric": METRIC, "value": sv["p99_ms"], "unit": "ms (p99 latency)",
        "n_gpus": ranks.world, "steps": 1, "warmup": 0, "ms_per_step": sv["wall_ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; G = U[diag(s) 0]V^T, s geometric 1..1e-10, Householder "
                "orthogonal factors, generated on the device)",
        "config": {"workload": sv["workload"], "arrival_rate_per_s": sv["arrival_rate_per_s"],
                   "offered_load": sv["offered_load"],
                   "solo_rate_solves_per_s": sv["solo_rate_solves_per_s"]},
        "gpu_launches": sv["launches"],
    }
    line.update({k: v for k, v in sv.items() if k not in line and k != "workload"})
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("sliced", "crt"):
        run_sliced_workload(args)
    elif args.workload == "grouped":
        run_grouped_workload(args)
    elif args.workload == "served":
        run_served_workload(args)
    elif args.workload == "potrf":
        run_potrf_workload(args)
    elif args.workload == "sweep":
        run_sweep_workload(args)
    elif args.workload == "plain":
        run_plain_workload(args)
    else:
        run_default(args)


if __name__ == "__main__":
    main()
