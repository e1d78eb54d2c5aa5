"""Benchmark: mortar pairs integrated per second (D + M, FP64) with the adjoint,
on one GB300, against the FP64 roofline.

One step = the whole hot path on one synthetic interface, replayed as one
CUDA graph: element precompute, binned search, per-pair segment integration,
CSR assembly of D and M, and the adjoint (gradient of the weighted gap
lambda.(D Xs - M Xm) w.r.t. all nodal coordinates).  Inputs are resident in
HBM before the timed region; the working set (~2 GB) is far larger than L2, so
no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload planar_2000x1733] [--no-cpu-baseline]

Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of the
workload (the interface is not sharded, there is no collective on the data
path); value = all ranks' pairs / max-over-ranks time ("scaling": "weak").

``--impl reference`` times the CPU oracle (the only reference that exists for
this method: the paper ships no code) on a bounded sample of the same
workload, on the host cores.

Besides the step, the JSON line carries (none of it inside the timed step):
``forward_only`` (search + integration + assembly graph), ``batched`` (the
512 uneven interfaces in one graph against one graph per interface: the
batched speed-up and the CTA busy-time imbalance eta_t), ``element_based``
(the same forward graph with the element-based rule, n = 4 and 8, and the
deviation of its M from the segment-based M), ``dynamic`` (a master sliding
0.3 h_m per step: device copy of the new coordinates + the full step, bins
rebuilt every step), ``linearisation`` (the 3x3-block Jacobian of the weighted
gap vector), ``fp64_probe`` (a DFMA chain: the measured FP64 rate), ``e2e``
(the step through the C ABI with host buffers).
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mortar pairs integrated/sec (D+M, FP64) and fwd+adjoint time on 1 GB300 vs FP64 roofline"
UNIT = "pairs/s"

# Executed FP64 flops (2 x DFMA + DADD + DMUL thread instructions, predicated
# on) and DRAM bytes per pair of the per-pair kernels, from ncu counters of
# this build on planar_600x520 (same element types and density as the full
# workload, so per-pair figures carry over); see profiles/.
EXEC_PER_PAIR = {
    "fused": {"flops": 8492.3, "dram_bytes": 880.0},
    "integrate": {"flops": 2994.6, "dram_bytes": 283.0},
}

# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA lanes
# per SM per clock (4 flop/clk/SM) x 2070 MHz maximum SM clock = 1.259 TFLOP/s,
# which is the part's nominal 1.25 TFLOP/s FP64 rate.
SM_COUNT = 152
FP64_FLOP_PER_CLK_PER_SM = 4
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12


def measured_peaks() -> dict:
    """HBM copy bandwidth and bf16 GEMM rates measured on the GB300s
    (MEASURED_PEAKS.json beside this file), else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "kind": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "kind": "fallback"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planar_2000x1733")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sections",
                    default="forward,dynamic,element_based,linearisation,batched,quadratic,contact,probe",
                    help="extra sections measured after the timed step (comma list; 'none' for the step only)")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            with open(self.path) as f:
                for r in csv.reader(f):
                    if len(r) >= 9:
                        rows.append([x.strip() for x in r])
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    """Largest value over all ranks (timing is the slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample_step(itf, rows: int, threads: int):
    """One bounded sample of the workload through the oracle: the slave
    elements of the first `rows` element rows, all master elements; binned
    search, per-pair integration, assembly and the forward-mode gradient."""
    import numpy as np
    import oracle
    from paper_2202_03933_gb300 import inputs
    n = int(round(len(itf.conn_s) ** 0.5))
    ne = min(rows * n, len(itf.conn_s))   # the whole slave mesh at most
    sub = inputs.Interface("sample", itf.xs, itf.conn_s[:ne], itf.type_s, itf.xm, itf.conn_m, itf.type_m,
                           lm=itf.lm, delta=itf.delta)
    lam = np.random.default_rng(0).uniform(-1, 1, itf.xs.shape)
    o = oracle.make_opts(lm=itf.lm, delta=itf.delta, n_threads=threads)
    t0 = time.perf_counter()
    res = oracle.evaluate(sub, o)
    oracle.weighted_gap_grad(sub, lam, res.s, res.m, o)
    dt = time.perf_counter() - t0
    return int(res.s.size), dt, ne


def cpu_baseline(itf, target_s: float = 12.0) -> dict:
    threads = os.cpu_count() or 1
    pairs, dt, ne = oracle_sample_step(itf, 2, threads)
    rows = max(2, min(200, int(2 * target_s / max(dt, 1e-3))))
    pairs, dt, ne = oracle_sample_step(itf, rows, threads)
    rows = -(-ne // max(1, int(round(len(itf.conn_s) ** 0.5))))   # rows actually taken
    p1, d1, _ = oracle_sample_step(itf, 1, 1)   # one host thread, one element row
    return {"value": pairs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{ne} of {len(itf.conn_s)} slave elements ({rows} element rows) x all master "
                      f"elements: {pairs} pairs; oracle search + integration + assembly + "
                      f"forward-mode gradient, {dt:.1f} s on {threads} host threads",
            "single_thread": {"value": p1 / d1, "unit": UNIT, "cores": 1,
                              "sample": f"1 element row, {p1} pairs, {d1:.1f} s"}}


def oracle_sample_extra(itf, rows: int = 2) -> dict:
    """Oracle timings beside the extra bench sections, on the slave elements of
    `rows` element rows against all master elements: the linearisation
    (forward-mode Dual<24> blocks + assembly) and element-based integration
    (n = 8), each in pairs per second on all host cores."""
    import numpy as np  # noqa: F401
    import oracle
    from paper_2202_03933_gb300 import inputs
    threads = os.cpu_count() or 1
    n = int(round(len(itf.conn_s) ** 0.5))
    ne = rows * n
    sub = inputs.Interface("sample", itf.xs, itf.conn_s[:ne], itf.type_s, itf.xm, itf.conn_m, itf.type_m,
                           lm=itf.lm, delta=itf.delta)
    o = oracle.make_opts(lm=itf.lm, delta=itf.delta, n_threads=threads)
    s, m = oracle.search_binned(sub, o.delta)
    t0 = time.perf_counter()
    oracle.tangent(sub, s, m, sub.xs, sub.xm, o, add_direct=True)
    t_lin = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.evaluate_element_based(sub, 8, o, pairs=(s, m))
    t_eb = time.perf_counter() - t0
    what = f"{ne} of {len(itf.conn_s)} slave elements ({rows} element rows), {s.size} pairs, {threads} host threads"
    return {"linearisation": {"pairs_per_s": s.size / t_lin, "s": round(t_lin, 2), "sample": what},
            "element_based_n8": {"pairs_per_s": s.size / t_eb, "s": round(t_eb, 2), "sample": what}}


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle on a bounded sample per step."""
    if rank != 0:
        return
    from paper_2202_03933_gb300 import inputs
    itf = inputs.by_name(args.workload)
    threads = os.cpu_count() or 1
    # rows per step: about 5 s of oracle work by the 2-row estimate, so that
    # the step's fixed cost (binning all master elements) is spread over
    # enough pairs
    _, dt2, _ = oracle_sample_step(itf, 2, threads)
    rows = max(4, min(200, int(2 * 5.0 / max(dt2, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample_step(itf, rows, threads)
    tot_pairs, tot_s = 0, 0.0
    for _ in range(args.steps):
        p, dt, ne = oracle_sample_step(itf, rows, threads)
        tot_pairs += p
        tot_s += dt
    value = tot_pairs / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample_element_rows": rows},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{ne} slave elements ({rows} element rows) x all master elements "
                                       "per step, oracle search + integration + assembly + gradient"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU
def batched_measure(steps: int, warmup: int, stream, clk_gpu=None) -> dict:
    """512 uneven interfaces (the batched workload): one batched context (one
    search, one persistent pair kernel over all pairs, one CUDA graph; launch
    shape from the autotuner) against one context per interface, each
    replaying its own graph, back to back.  Forward + adjoint in both."""
    import numpy as np
    import torch
    from paper_2202_03933_gb300 import inputs, mortar

    itfs = inputs.batched_512()
    lam_all = np.random.default_rng(1).uniform(-1, 1, (sum(i.xs.shape[0] for i in itfs), 3))
    m = mortar.Mortar(lm=0, delta=1e-9, stream=stream.cuda_stream)
    m.set_batch(itfs)
    pick = m.autotune(lam_all)
    m.set_timing(True)
    lam_d = torch.from_numpy(lam_all).cuda()
    for _ in range(max(warmup, 3)):
        m.run_graph(lam_d)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = None
    if clk_gpu is not None:
        with ClockSampler(clk_gpu) as clk:
            e0.record(stream)
            for _ in range(steps):
                m.run_graph(lam_d)
            e1.record(stream)
            torch.cuda.synchronize()
        clocks = clk.summary()
    else:
        e0.record(stream)
        for _ in range(steps):
            m.run_graph(lam_d)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = m.stats()
    # one context (and one graph) per interface
    ctxs, lams = [], []
    off = 0
    for itf in itfs:
        c = mortar.Mortar(lm=0, delta=1e-9, stream=stream.cuda_stream)
        c.set_interface(torch.from_numpy(itf.xs).cuda(), torch.from_numpy(itf.conn_s).cuda(),
                        torch.from_numpy(itf.xm).cuda(), torch.from_numpy(itf.conn_m).cuda())
        lam = lam_d[off:off + itf.xs.shape[0]].contiguous()
        off += itf.xs.shape[0]
        for _ in range(2):
            c.run_graph(lam)
        ctxs.append(c)
        lams.append(lam)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(steps):
        for c, lam in zip(ctxs, lams):
            c.run_graph(lam)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_sep = f0.elapsed_time(f1) / steps
    for c in ctxs:
        c.close()
    out = {"interfaces": len(itfs), "pairs": st["n_pairs"],
           "slave_elements": int(sum(i.conn_s.shape[0] for i in itfs)),
           "step": "batched search + integrate + assemble + adjoint, one CUDA graph",
           "autotune": pick, "ms_per_step": round(ms, 4), "pairs_per_s": st["n_pairs"] / (ms / 1e3),
           "phases_ms": {"search": st["ms_search"], "pair_kernel": st["ms_integrate"],
                         "assemble": st["ms_assemble"], "adjoint_rest": st["ms_adjoint"]},
           "one_graph_per_interface_ms": round(ms_sep, 4), "batched_speedup": round(ms_sep / ms, 3),
           "eta_t": round(float(st.get("eta_t", 0.0)), 4),
           "graph_kernels": int(st.get("graph_kernels", 0))}
    if clocks is not None:
        out["clocks"] = clocks
    m.close()
    return out


def run_batched(args, world, rank, local):
    """--workload batched_512: the batched measurement as its own JSON line."""
    import torch
    from paper_2202_03933_gb300 import build

    build()
    stream = torch.cuda.current_stream()
    barrier(world)
    b = batched_measure(args.steps, args.warmup, stream, clk_gpu=local)
    ms = max_over_ranks(world, b["ms_per_step"])
    clocks = b.pop("clocks")
    line = {"metric": METRIC, "value": weak_value(world, b["pairs"], ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched_512", "interfaces": b["interfaces"], "pairs": b["pairs"],
                       "slave_elements": b["slave_elements"], "step": b["step"], "autotune": b["autotune"]},
            "phases_ms": b["phases_ms"], "one_graph_per_interface_ms": b["one_graph_per_interface_ms"],
            "batched_speedup": b["batched_speedup"], "eta_t": b["eta_t"],
            "gpu_launches": b["graph_kernels"] * args.steps,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)


class _Skip(Exception):
    """An extra section left out by --sections."""


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2202_03933_gb300 import build, inputs, mortar

    build()
    sections = set(args.sections.split(","))
    itf = inputs.by_name(args.workload)
    if isinstance(itf, list):
        raise SystemExit("use a single-interface workload for the headline benchmark")
    dev = torch.device("cuda", torch.cuda.current_device())
    xs = torch.from_numpy(itf.xs).to(dev)
    xm = torch.from_numpy(itf.xm).to(dev)
    cs = torch.from_numpy(itf.conn_s).to(dev)
    cm = torch.from_numpy(itf.conn_m).to(dev)
    lam_h = np.random.default_rng(1).uniform(-1, 1, itf.xs.shape)
    lam = torch.from_numpy(lam_h).to(dev)
    stream = torch.cuda.current_stream()
    m = mortar.Mortar(lm=itf.lm, delta=itf.delta, stream=stream.cuda_stream)
    m.set_interface(xs, cs, xm, cm)
    pick = m.autotune(lam)
    m.set_timing(True)
    for _ in range(max(args.warmup, 3)):
        m.run_graph(lam)
    torch.cuda.synchronize()
    st0 = m.stats()
    per_step = []
    t_int, t_adjp, t_adj, t_srch, t_asm = [], [], [], [], []
    barrier(world)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            m.run_graph(lam)
            s = m.stats()
            t_int.append(s["ms_integrate"])
            t_adjp.append(s["ms_adjoint_pairs"])
            t_adj.append(s["ms_adjoint"])
            t_srch.append(s["ms_search"])
            t_asm.append(s["ms_assemble"])
            per_step.append(s["ms_total"])
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(world, ms)
    st = m.stats()
    n_pairs = st["n_pairs"]
    value = weak_value(world, n_pairs, ms)

    # per-phase figures: median over the timed steps (CUDA events in the graph)
    med = statistics.median
    ms_pair = med(t_int)   # the pair kernel that produced the forward blocks (fused with the adjoint)
    fused = bool(st.get("fused", 0))
    # ---- roofline of the dominant kernel: executed FP64 flops / its CUDA-event time
    ex = EXEC_PER_PAIR["fused" if fused else "integrate"]
    roof = {"bound": "alu", "kernel": ("k_adjoint_batched: fused forward blocks + adjoint per pair" if fused
                                       else "k_integrate_batched"),
            "ms_per_launch": round(ms_pair, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "peak_kind": "derived FP64: 152 SM x 4 flop/clk x 2070 MHz (of derived; measured probe below)",
            "flops": "executed FP64 (ncu 2 DFMA + DADD + DMUL per pair, planar_600x520) x pairs",
            "achieved": None, "frac": None, "traffic": None}
    # the per-pair counters were taken on the planar quad4/quad4 dual family;
    # other element types execute other per-pair work, so they get no fraction
    same_family = args.workload.startswith("planar_") and itf.lm == 1
    if ex["flops"] and same_family:
        achieved = ex["flops"] * n_pairs / (ms_pair / 1e3) / 1e12
        roof.update(achieved=round(achieved, 4), frac=round(achieved / FP64_PEAK_TFLOPS, 4),
                    flops_per_pair=ex["flops"])
    elif ex["flops"]:
        roof["note"] = "executed FP64 per pair measured on the planar quad4/quad4 dual family only"
    if ex["dram_bytes"] and same_family:
        roof["traffic"] = int(ex["dram_bytes"] * n_pairs)

    # ---- HBM rates of the two memory-bound phases (algorithmic bytes / phase
    #      time): search = element boxes read (64 B per element, both sides) +
    #      master keys and bin lists (16 B per master element) + pairs written
    #      (8 B each) + per-slave counts and offsets (12 B per slave element);
    #      assembly = per-pair M blocks and flags read (129 B per pair) + element
    #      D blocks read (128 B per slave element) + CSR of D and M written
    #      (12 B per entry, 16 B per row)
    try:
        n_nzD, n_nzM = m.csr_size(mortar.MATRIX_D)[2], m.csr_size(mortar.MATRIX_M)[2]
        Es_, Em_ = itf.conn_s.shape[0], itf.conn_m.shape[0]
        b_search = 64 * (Es_ + Em_) + 16 * Em_ + 8 * n_pairs + 12 * Es_
        b_asm = 129 * n_pairs + 128 * Es_ + 12 * (n_nzD + n_nzM) + 16 * itf.xs.shape[0]
        phase_bw = {"search_GBps": round(b_search / (med(t_srch) / 1e3) / 1e9, 1),
                    "assemble_GBps": round(b_asm / (med(t_asm) / 1e3) / 1e9, 1),
                    "hbm_peak_GBps": measured_peaks().get("hbm_gbs"),
                    "note": "of measured copy bandwidth; the phases are gathers, latency-bound"}
    except Exception as ex_:   # reported, not fatal
        phase_bw = {"error": str(ex_)}

    # ---- forward only (search + integration + assembly graph): forward pairs/s
    #      and the integration kernel's executed-FP64 roofline fraction
    fwd = None
    try:
        if "forward" not in sections:
            raise _Skip()
        # a context of its own, autotuned for the forward pass (the integration
        # kernel's best launch shape differs from the fused kernel's)
        mf = mortar.Mortar(lm=itf.lm, delta=itf.delta, stream=stream.cuda_stream)
        mf.set_interface(xs, cs, xm, cm)
        pick_f = mf.autotune()
        mf.set_timing(True)
        for _ in range(3):
            mf.run_graph()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_fi = []
        g0.record(stream)
        for _ in range(args.steps):
            mf.run_graph()
            t_fi.append(mf.stats()["ms_integrate"])
        g1.record(stream)
        torch.cuda.synchronize()
        ms_f = g0.elapsed_time(g1) / args.steps
        mf.close()
        fwd = {"ms_per_step": round(ms_f, 4), "pairs_per_s": world * n_pairs / (ms_f / 1e3),
               "ms_integrate": round(med(t_fi), 4), "autotune": pick_f}
        exf = EXEC_PER_PAIR["integrate"]
        if exf["flops"] and args.workload.startswith("planar_") and itf.lm == 1:
            a = exf["flops"] * n_pairs / (med(t_fi) / 1e3) / 1e12
            fwd["roofline"] = {
                "bound": "alu", "kernel": "k_integrate_batched", "ms_per_launch": round(med(t_fi), 4),
                "achieved": round(a, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(a / FP64_PEAK_TFLOPS, 4), "flops_per_pair": exf["flops"],
                "flops": "executed FP64 (ncu 2 DFMA + DADD + DMUL per pair, planar_600x520) x pairs",
                "traffic": int(exf["dram_bytes"] * n_pairs) if exf["dram_bytes"] else None}
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        fwd = {"error": str(ex_)}

    # ---- dynamic interface (Algorithm 2 every step): the master slides by
    #      0.3 h_m per step in-plane; each step uploads the new master
    #      coordinates (device copy) and replays the forward + adjoint graph,
    #      which re-bins and re-searches from scratch; bins carry the
    #      2 dt |v| margin of Sec. 3.5
    dyn = None
    try:
        if "dynamic" not in sections:
            raise _Skip()
        K = max(min(args.steps, 8), 2)
        hm = 1.0 / itf.info.get("nm", 1) if "nm" in itf.info else 0.0
        shift = 0.3 * hm
        md = mortar.Mortar(lm=itf.lm, delta=itf.delta, stream=stream.cuda_stream, bin_margin=2 * shift)
        md.set_interface(xs, cs, xm, cm)
        md.set_launch(pick.get("variant", 0), pick.get("block", 0), 0, pick.get("rounds", 0))
        xm_k = [xm + torch.tensor([shift * (k + 1), 0.0, 0.0], dtype=torch.float64, device=dev)
                for k in range(K + 2)]
        for k in range(2):
            md.set_coordinates(None, xm_k[k])
            md.run_graph(lam)
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pairs_dyn = 0
        d0.record(stream)
        for k in range(K):
            md.set_coordinates(None, xm_k[k + 2])
            md.run_graph(lam)
            pairs_dyn += md.stats()["n_pairs"]
        d1.record(stream)
        torch.cuda.synchronize()
        ms_d = d0.elapsed_time(d1) / K
        dyn = {"ms_per_step": round(ms_d, 3), "pairs_per_s": world * pairs_dyn / K / (ms_d / 1e3),
               "steps": K, "shift_per_step": f"0.3 h_m = {shift:.3e}",
               "step": "device copy of the moved master coordinates + search + integrate + assemble + adjoint"}
        md.close()
        del xm_k
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        dyn = {"error": str(ex_)}

    # ---- element-based integration (Sec. 1, Sec. 2.3): forward graph with an
    #      n x n rule per slave element instead of clipping; time and the
    #      deviation of M from the segment-based M of this workload
    ebi = None
    try:
        if "element_based" not in sections:
            raise _Skip()
        import scipy.sparse as sp
        m.run_graph()
        ref = m.scipy(mortar.MATRIX_M)
        ebi = {}
        for n_r in (4, 8):
            me = mortar.Mortar(lm=itf.lm, delta=itf.delta, stream=stream.cuda_stream,
                               integration=mortar.INTEGRATE_ELEMENT, element_rule_n=n_r)
            me.set_interface(xs, cs, xm, cm)
            me.set_timing(True)
            for _ in range(3):
                me.run_graph()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t_e = []
            e0.record(stream)
            for _ in range(args.steps):
                me.run_graph()
                t_e.append(me.stats()["ms_integrate"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms_e = e0.elapsed_time(e1) / args.steps
            Me = me.scipy(mortar.MATRIX_M)
            dev_M = abs(Me - ref).max() / abs(ref).max()
            ebi[f"n{n_r}"] = {"forward_ms_per_step": round(ms_e, 3), "ms_integrate": round(med(t_e), 3),
                             "pairs_per_s": world * n_pairs / (ms_e / 1e3),
                             "max_rel_dev_M_vs_segment": float(dev_M), "sum_M": float(Me.sum())}
            me.close()
        ebi["segment_sum_M"] = float(ref.sum())
        del sp
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        ebi = {"error": str(ex_)}

    # ---- linearisation of D and M (Jacobian of the weighted gap vector, BSR):
    #      separate call, not part of the step; device time of its kernels
    lin = None
    try:
        if "linearisation" not in sections:
            raise _Skip()
        for _ in range(1):
            m.tangent(xs, xm, add_direct=True, out_device=True)
        t_l = []
        for _ in range(min(args.steps, 3)):
            m.tangent(xs, xm, add_direct=True, out_device=True)
            t_l.append(m.stats()["ms_tangent"])
        sl = m.stats()
        lin = {"ms": round(med(t_l), 3), "pairs_per_s": world * n_pairs / (med(t_l) / 1e3),
               "blocks_3x3": sl["nnzb_K"],
               "what": "K = d/dX[(D (x) I3) Xs - (M (x) I3) Xm] + [D (x) I3 | -M (x) I3]: pair blocks, "
                       "element blocks, BSR assembly"}
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        lin = {"error": str(ex_)}

    # ---- batched uneven interfaces (512 interfaces, one graph) against one
    #      graph per interface: the batched speed-up and the CTA imbalance eta_t
    bat = None
    try:
        if "batched" not in sections:
            raise _Skip()
        bat = batched_measure(max(min(args.steps, 10), 3), 3, stream)
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        bat = {"error": str(ex_)}

    # ---- quadratic slave elements (quad8 on the unit square: 1000 x 1000 with
    #      the full workload, 450 x 450 otherwise) against a noisy quad4 master
    #      (h_m / h_s = 1.155): forward graph (search + sub-element integration
    #      + assembly), and the oracle on a strip
    qd = None
    try:
        if "quadratic" not in sections:
            raise _Skip()
        nq = 1000 if args.workload == "planar_2000x1733" else 450
        nqm = int(round(nq / 1.155))
        q = inputs.quadratic_planar(nq, nqm, "quad8", name=f"quad8_{nq}x{nqm}")
        mq = mortar.Mortar(lm=0, delta=q.delta, stream=stream.cuda_stream)
        mq.set_interface(torch.from_numpy(q.xs).to(dev), torch.from_numpy(q.conn_s).to(dev),
                         torch.from_numpy(q.xm).to(dev), torch.from_numpy(q.conn_m).to(dev))
        mq.set_timing(True)
        for _ in range(3):
            mq.run_graph()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_q = []
        q0.record(stream)
        for _ in range(args.steps):
            mq.run_graph()
            t_q.append(mq.stats()["ms_integrate"])
        q1.record(stream)
        torch.cuda.synchronize()
        ms_q = q0.elapsed_time(q1) / args.steps
        sq = mq.stats()
        qd = {"workload": f"quad8 {nq}x{nq} slave vs noisy quad4 {nqm}x{nqm} master, standard LMs",
              "pairs": sq["n_pairs"], "nonempty_pairs": sq["n_nonempty"], "gauss_points": sq["n_gauss_points"],
              "forward_ms_per_step": round(ms_q, 3), "ms_integrate": round(med(t_q), 3),
              "pairs_per_s": world * sq["n_pairs"] / (ms_q / 1e3)}
        mq.close()
        if rank == 0 and not args.no_cpu_baseline:
            import oracle
            threads = os.cpu_count() or 1
            sub = inputs.Interface("sample", q.xs, q.conn_s[:2 * nq], q.type_s, q.xm, q.conn_m, q.type_m,
                                   lm=0, delta=q.delta)
            t0 = time.perf_counter()
            rq = oracle.evaluate(sub, oracle.make_opts(lm=0, delta=q.delta, n_threads=threads))
            dt = time.perf_counter() - t0
            qd["oracle"] = {"pairs_per_s": rq.s.size / dt, "s": round(dt, 2),
                            "sample": f"{2 * nq} of {nq * nq} slave elements (2 element rows), {rq.s.size} pairs, "
                                      f"search + integration + assembly, {threads} host threads"}
        del q
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        qd = {"error": str(ex_)}

    # ---- contact-specific terms on the evaluated interface: nodal normals,
    #      weighted normal gap, active set and complementarity residual; device
    #      inputs, no host copies; CUDA-event time of the call
    con = None
    try:
        if "contact" not in sections:
            raise _Skip()
        import ctypes
        m.run_graph()   # forward blocks of the current coordinates
        lam_n = torch.from_numpy(np.random.default_rng(2).uniform(-1.0, 0.0, itf.xs.shape[0])).to(dev)

        def contact_call():
            mortar.call("mortar_contact_terms", m.h, ctypes.c_void_p(lam_n.data_ptr()), 1.0, None, None, None,
                        None, 1, ok=(0, -2, -3))

        contact_call()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        K_c = max(min(args.steps, 10), 3)
        c0.record(stream)
        for _ in range(K_c):
            contact_call()
        c1.record(stream)
        torch.cuda.synchronize()
        ms_c = c0.elapsed_time(c1) / K_c
        con = {"ms": round(ms_c, 3), "slave_nodes": int(itf.xs.shape[0]),
               "nodes_per_s": world * itf.xs.shape[0] / (ms_c / 1e3),
               "what": "averaged nodal normals, weighted normal gap, active set and NCP residual per slave node"}
    except _Skip:
        pass
    except Exception as ex_:   # reported, not fatal
        con = {"error": str(ex_)}

    # ---- FP64 probe (measured peak, for context)
    probe = None
    try:
        if "probe" not in sections:
            raise _Skip()
        blocks, threads, iters = SM_COUNT * 8, 256, 20000
        sink = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
        mortar.probe_dfma(blocks, threads, 100, sink=sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mortar.probe_dfma(blocks, threads, iters, sink=sink)
        e1.record(stream)
        torch.cuda.synchronize()
        pm = e0.elapsed_time(e1)
        probe = {"tflops": round(blocks * threads * 8 * 2 * iters / (pm / 1e3) / 1e12, 4), "ms": round(pm, 3)}
    except _Skip:
        pass
    except Exception as ex:   # measurement context only
        probe = {"error": str(ex)}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        xs_p = torch.from_numpy(itf.xs).pin_memory()
        xm_p = torch.from_numpy(itf.xm).pin_memory()
        lam_p = torch.from_numpy(lam_h).pin_memory()
        nr, _, nnzD = m.csr_size(mortar.MATRIX_D)
        _, _, nnzM = m.csr_size(mortar.MATRIX_M)
        outs = {k: torch.empty(n, dtype=t).pin_memory() for k, n, t in (
            ("rpD", nr + 1, torch.int64), ("ciD", nnzD, torch.int32), ("vaD", nnzD, torch.float64),
            ("rpM", nr + 1, torch.int64), ("ciM", nnzM, torch.int32), ("vaM", nnzM, torch.float64),
            ("gs", itf.xs.size, torch.float64), ("gm", itf.xm.size, torch.float64))}
        import ctypes
        L = mortar.lib()
        P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        Jc = ctypes.c_double()

        def e2e_step():
            mortar.call("mortar_set_coordinates", m.h, P(xs_p), P(xm_p), 0)
            mortar.call("mortar_run_graph", m.h, P(lam_p), 0, ok=(0, -3))
            mortar.call("mortar_get_gradient", m.h, ctypes.byref(Jc), P(outs["gs"]), P(outs["gm"]), 0)
            mortar.call("mortar_csr_copy", m.h, 0, P(outs["rpD"]), P(outs["ciD"]), P(outs["vaD"]), nnzD, 0)
            mortar.call("mortar_csr_copy", m.h, 1, P(outs["rpM"]), P(outs["ciM"]), P(outs["vaM"]), nnzM, 0)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(world, (time.perf_counter() - t0) * 1e3 / args.steps)
        h2d = xs_p.numel() * 8 + xm_p.numel() * 8 + lam_p.numel() * 8
        d2h = sum(t.numel() * t.element_size() for t in outs.values()) + 8
        e2e = {"value": world * n_pairs / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": round(e2e_ms, 3),
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        del L

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "slave": "2000x2000 quad4" if args.workload == "planar_2000x1733"
                   else None, "lm": "dual" if itf.lm == 1 else "standard", "pairs": n_pairs,
                   "nonempty_pairs": st["n_nonempty"], "gauss_points": st["n_gauss_points"],
                   "step": "search + integrate + assemble D,M + adjoint, one CUDA graph",
                   "l2": "inputs and workspaces (~GBs) larger than the 129 MB L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"search": round(med(t_srch), 4), "pair_kernel": round(ms_pair, 4),
                      "fused_forward_adjoint": fused, "assemble": round(med(t_asm), 4),
                      "adjoint_rest": round(med(t_adj) - med(t_adjp), 4),
                      "adjoint_pairs_separate": round(med(t_adjp), 4), "graph_total": round(med(per_step), 4)},
        "autotune": pick,
        "phase_bandwidth": phase_bw,
        "forward_only": fwd,
        "linearisation": lin,
        "batched": bat,
        "element_based": ebi,
        "dynamic": dyn,
        "quadratic": qd,
        "contact": con,
        "roofline": roof,
        "fp64_probe": probe,
        "e2e": e2e,
        "gpu_launches": int(st0.get("graph_kernels", 0)) * args.steps,
        "eta_t": round(float(st.get("eta_t", 0.0)), 4),
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(itf)
        try:
            line["oracle_beside_sections"] = oracle_sample_extra(itf)
        except Exception as ex_:   # reported, not fatal
            line["oracle_beside_sections"] = {"error": str(ex_)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup()
    if args.workload == "batched_512":
        run_batched(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
