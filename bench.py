"""Benchmark of the sliced sparse-state contraction + sampling on GB300.

One step = the whole hot path over one batch: contract every kept slice of the
workload into the head tensor (FP64 accumulation), look up all L x 2^h
amplitudes, normalise (FP64 norms) and draw one sample per group.

Workload (default): 30-qubit 5x6 grid, 14 cycles, seeded Sycamore-like gates,
10 open qubits x 64 tails = 65,536 amplitudes, 6 sliced edges (2^6 slices, all
summed), largest intermediate <= 2^28 elements.  Synthetic inputs (the paper's
circuit files are not used).

Prints one JSON line (rank 0).  `value` is slice TFLOP/s = 8 T_c(slice) x
slices / step time (the paper's efficiency convention, 8 real flops per
complex multiply-add, T_c the plan's algorithmic count), device-resident
inputs; `e2e` is the same metric through the C ABI with host buffers.
`--impl reference` times the CPU oracle on a bounded sample of the same
workload instead.

Several GPUs (`--gpus N`, one process per GPU under torch.distributed.run,
which bench.py starts itself when no launcher did): the kept slice range is
split into contiguous per-rank ranges, each rank contracts its range into its
own head, and one host-side sum-reduce of the heads (gloo) gives rank 0 the
full head, which it looks up, normalises and samples.  Strong scaling: the
whole job is the same 64 slices at every N.  `--replicas` instead runs the
whole workload on every GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import circuit_inputs as ci  # noqa: E402

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch,
# from a single-kernel ncu capture of the current kernel; keyed by the GEMM
# engine, the GEMM tiling ("cta" or "pair") and the launch's algorithmic
# complex MACs and bytes (tn_plan_step_info).  A dominant launch with no
# entry reports traffic null.
MEASURED_TRAFFIC = {
    ("fp16", "pair", 270582939648, 1329594368): (5.423687e9 + 0.266117888e9,
                                                 "profiles/gemm_tc_pair_fp16x3_grid5x6_m14_open10_L64_k6.md"),
}

KIND_NAMES = {0: "small_operand", 1: "permute", 2: "bprep_tc", 3: "gemm_tc_3xtf32", 4: "bprep_simt",
              5: "gemm_simt_fp32", 6: "operand_max", -1: "accumulate"}
ORDER_TRIALS = 2048


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _workload(name):
    if name == "sliced30":
        return ci.config_sliced30()
    if name == "tiny":
        return ci.config_tiny()
    if name == "grid25":
        return ci.config_grid25()
    if name == "syc53":
        # 53-qubit Sycamore topology at reduced depth (8 cycles): 6 open qubits x
        # 1024 tails; automatic slicing to a 2^30-element cap, so the one slice
        # runs as 2^n_internal passes
        circ = ci.make_sycamore_circuit(8, seed=5)
        n = circ.n_qubits
        oq = list(range(n - 6, n))
        return dict(circuit=circ, open_qubits=oq, tails=ci.draw_tails(n, oq, 1024, seed=55), edges=[],
                    name="sycamore53_m8_open6_L1024", plan_opts=dict(max_log2_elements=30, auto_slice=16))
    if name == "precision40":
        # 40-qubit 5x8 grid, 16 cycles, 12 open qubits x 1 tail, 2^10 slices of
        # which the kept 1/8 (128) are summed; a step times the first
        # --slices of them (default 4) and the line projects the kept sum
        cfg = ci.config_precision40(16)
        cfg.update(plan_opts=dict(max_log2_elements=32, auto_slice=24), order_trials=4096, default_slices=4)
        return cfg
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index
        # raw samples: $BENCH_CLOCKS_DIR if set, else the system temp directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        mx = float(rows[0][2])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(cfg, n_slices):
    """The workload as both arms print it: circuit and sparse-state sizes
    only (no implementation detail), plus how the GPU arm treats L2."""
    circ = cfg["circuit"]
    h, L = len(cfg["open_qubits"]), len(cfg["tails"])
    k = sum(1 for e in cfg["edges"] if e[2] in (ci.EDGE_SLICE, ci.EDGE_COMPANION))
    return {"workload": cfg["name"], "qubits": circ.n_qubits, "cycles": circ.cycles, "open_qubits": h,
            "groups": L, "amplitudes": L << h, "sliced_edges": k, "slices": n_slices,
            "l2": "GPU arm: L2 flushed between timed steps (512 MiB write); intermediates up to 2 GiB exceed L2"}


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _spawn_ranks(n):
    """--gpus N with no launcher around this process: run N ranks of this same
    command under torch.distributed.run (one process per GPU)."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch

    import paper_2111_03011_gb300 as tn

    from paper_2111_03011_gb300.shard import reduce_heads, slice_share

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfg = _workload(args.workload)
    gemm = {"tc": tn.TN_GEMM_TC_3XTF32, "simt": tn.TN_GEMM_SIMT_FP32, "bf16": tn.TN_GEMM_TC_BF16X3,
            "fp16": tn.TN_GEMM_TC_FP16X3}[args.engine]
    t0 = time.time()
    popts = cfg.get("plan_opts", {})
    trials = cfg.get("order_trials", ORDER_TRIALS if args.workload in ("sliced30", "syc53") else 0)
    if rank == 0 and args.autotune > 0:
        plan = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"],
                                   n_candidates=args.autotune, gemm=gemm, order_trials=trials, **popts)
    elif rank == 0:
        plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                          order_trials=trials, **popts)
    if ws > 1:
        # every rank contracts with rank 0's plan: its order goes to the others
        import torch.distributed as dist
        # (with its CTA-pair choice and the tile variant the step tuner chose for each step)
        box = [(tn.tn_plan_order(plan).tolist(), tn.tn_plan_get_stats(plan)["gemm_pair"],
                [s["variant"] for s in tn.tn_plan_describe(plan)["steps"]]) if rank == 0 else None]
        dist.broadcast_object_list(box, src=0)
        if rank != 0:
            plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                              order=np.array(box[0][0], dtype=np.int32).reshape(-1, 2), gemm_pair=box[0][1],
                              **popts)
            for i, v in enumerate(box[0][2]):
                tn.tn_plan_set_step_variant(plan, i, v)
    plan_s = time.time() - t0
    st = tn.tn_plan_get_stats(plan)
    k = st["n_sliced"]
    n_slices = cfg.get("kept", 1 << k)            # the kept prefix [0, kept) of the 2^k slices
    if args.slices:
        n_slices = min(n_slices, args.slices)     # profiling runs only: fewer launches per step
    L, h = int(st["n_tails"]), int(st["n_open"])
    n_amp = L << h
    n_samples = L
    oq, tails = cfg["open_qubits"], cfg["tails"]
    mask = 0
    for q in oq:
        mask |= 1 << q
    base = (tails.astype(np.uint64) & np.uint64(~mask & ((1 << 64) - 1)))
    mu = np.arange(1 << h, dtype=np.uint64)
    dep = np.zeros(1 << h, dtype=np.uint64)
    for j, q in enumerate(oq):
        dep |= ((mu >> np.uint64(j)) & np.uint64(1)) << np.uint64(q)
    bits_host = (base[:, None] | dep[None, :]).reshape(-1)
    bits_pinned = torch.from_numpy(bits_host.view(np.int64)).pin_memory()
    bits_dev = bits_pinned.to(dev)
    amp_dev = torch.empty(n_amp, dtype=torch.complex128, device=dev)
    smp_dev = torch.empty(n_samples, dtype=torch.int64, device=dev)
    amp_host = torch.empty(n_amp, dtype=torch.complex128).pin_memory()
    smp_host = torch.empty(n_samples, dtype=torch.int64).pin_memory()
    head_buf = torch.zeros((L, 1 << h), dtype=torch.complex128, device=dev)
    head = tn.tn_head_create(plan, head_buf)
    sharded = ws > 1 and not args.replicas
    b0, e0_ = slice_share(0, n_slices, rank, ws) if sharded else (0, n_slices)
    my_slices = e0_ - b0
    head_host = torch.empty((L, 1 << h), dtype=torch.complex128).pin_memory() if sharded else None
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    n_pass = 1 << int(st["n_internal_sliced"])     # passes of the launch list per slice
    n_launch = int(st["n_launches"]) // n_pass     # launches of one pass
    use_graph = n_slices * n_pass * n_launch <= 50000   # graphs of up to 50k kernel nodes
    step_ms_acc = np.zeros(n_launch)

    def step(host_io, profile):
        tn.tn_head_reset(head, stream)
        if my_slices == 0:
            pass
        elif profile:
            step_ms_acc[:] += tn.tn_profile_slices(plan, b0, e0_, head, stream)
        elif use_graph:
            # the step's slices replay as one captured CUDA graph (captured in warm-up)
            tn.tn_contract_slices_graph(plan, b0, e0_, head, stream)
        else:
            tn.tn_contract_slices(plan, b0, e0_, head, stream)
        if sharded:
            # the exchange step: sum of the ranks' heads on the host (gloo);
            # rank 0 continues with the full head
            head_host.copy_(head_buf, non_blocking=True)
            stream.synchronize()
            reduce_heads(head_host)
            if rank != 0:
                return
            head_buf.copy_(head_host, non_blocking=True)
            tn.tn_head_set_fidelity(head, n_slices / (1 << k))
        if host_io:
            tn.tn_amplitudes(head, bits_pinned, out=amp_host, dtype=tn.TN_C128, stream=stream)
            tn.tn_head_norm(head, stream=stream)
            tn.tn_sample(head, n_samples, 0.0, 12345, out=smp_host, stream=stream)
        else:
            tn.tn_amplitudes(head, bits_dev, out=amp_dev, dtype=tn.TN_C128, stream=stream)
            tn.tn_head_norm(head, stream=stream)
            tn.tn_sample(head, n_samples, 0.0, 12345, out=smp_dev, stream=stream)

    def timed(host_io, profile):
        for _ in range(args.warmup):
            step(host_io, False)
        torch.cuda.synchronize(dev)
        _barrier(ws)
        torch.cuda.synchronize(dev)
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush between timed iterations (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(host_io, profile)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize(dev)
        _barrier(ws)
        return _max(ws, total / args.steps)

    with Clocks(local) as clk:
        ms_prof = timed(False, True)      # per-launch CUDA events: the roofline figures
        ms = timed(False, False)          # the value: no per-launch events
    ms_e2e = timed(True, False)
    clocks = clk.summary()

    flops_step = 8.0 * st["tc_macs"] * n_slices
    jobs = ws if (ws > 1 and not sharded) else 1          # replicas each run the whole workload
    value = jobs * flops_step / (ms * 1e-3) / 1e12
    e2e = jobs * flops_step / (ms_e2e * 1e-3) / 1e12
    if rank != 0:
        return
    peaks, peak_src = _peaks()
    # dominant launch over the timed steps
    per_launch = step_ms_acc / args.steps / (max(my_slices, 1) * n_pass)   # ms per launch
    i_dom = int(np.argmax(per_launch))
    kind, macs, abytes = tn.tn_plan_step_info(plan, i_dom)
    t_dom = per_launch[i_dom] * 1e-3
    kind_totals = {}
    for i in range(n_launch):
        kk, _, _ = tn.tn_plan_step_info(plan, i)
        name = KIND_NAMES[kk]
        if args.engine in ("bf16", "fp16"):
            name = name.replace("gemm_tc_3xtf32", f"gemm_tc_{args.engine}x3")
        kind_totals[name] = kind_totals.get(name, 0.0) + per_launch[i]
    tot = sum(kind_totals.values())
    if kind in (3,) and args.engine in ("bf16", "fp16"):
        peak = peaks["bf16_tflops_sustained"] / 3.0
        achieved = 8.0 * macs / t_dom / 1e12
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": f"gemm_tc_{args.engine}x3",
                "peak_note": f"{peak_src} sustained bf16 / 3 (kind::f16 runs bf16 and fp16 at one rate; "
                             f"the split issues 3 MMAs per product)"}
    elif kind in (3,):
        tf32 = peaks["bf16_tflops_sustained"] * (1.1 / 2.25)
        peak = tf32 / 3.0
        achieved = 8.0 * macs / t_dom / 1e12
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": KIND_NAMES[kind],
                "peak_note": f"{peak_src} sustained bf16 x 1.1/2.25 (tf32) / 3 (3xTF32 issues 3 MMAs per product)"}
    elif kind == 5:
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        achieved = 8.0 * macs / t_dom / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": KIND_NAMES[kind],
                "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    else:
        peak = peaks["hbm_gbs"]
        achieved = abytes / t_dom / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": KIND_NAMES[kind],
                "peak_note": f"{peak_src} hbm_gbs"}
    tiling = "pair" if st["gemm_pair"] == 0 and args.engine in ("fp16", "bf16") else "cta"
    tr = MEASURED_TRAFFIC.get((args.engine, tiling, int(round(macs)), int(round(abytes))))
    if tr:
        roof["traffic"] = tr[0]
        roof["traffic_note"] = (f"ncu dram bytes of one launch of this kernel and shape ({tr[1]}); algorithmic "
                                f"bytes {abytes:.4g}")
    roof["dominant_launch_ms"] = round(per_launch[i_dom], 4)
    roof["ms_per_step_profiled"] = round(ms_prof, 3)
    roof["kernel_time_share"] = {k2: round(v / tot, 4) for k2, v in sorted(kind_totals.items(), key=lambda x: -x[1])}
    # path roofline: sum over launches of max(flops / peak of the step's engine,
    # algorithmic bytes / HBM) against the sum of their live times
    tf32_split = peaks["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0
    f16_split = peaks["bf16_tflops_sustained"] / 3.0
    simt_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    t_roof = 0.0
    for i in range(n_launch):
        kk, m_i, b_i = tn.tn_plan_step_info(plan, i)
        pk = {3: f16_split if args.engine in ("bf16", "fp16") else tf32_split, 5: simt_peak}.get(kk)
        t_flop = 8.0 * m_i / (pk * 1e12) if pk else 0.0
        t_roof += max(t_flop, b_i / (peaks["hbm_gbs"] * 1e9))
    roof["path_fraction"] = round(t_roof / (tot * 1e-3), 4)
    roof["path_fraction_note"] = ("sum of per-launch rooflines max(8 MACs / engine peak, bytes / HBM) over the sum "
                                  "of their live times; GEMM steps of K = 2 counted at the split engine's peak")

    out = {
        "metric": "slice TFLOP/s",
        "value": round(value, 3),
        "unit": "TFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "c64 (bf16x3 GEMM steps)", "fp16": "c64 (fp16x3 GEMM steps)"}.get(args.engine, "c64"),
        "data": "synthetic (seeded Sycamore-like circuit; paper's circuit files not used)",
        "config": workload_config(cfg, n_slices),
        "parallelism": (f"slice ranges sharded over {ws} GPUs, heads summed on the host (gloo)" if sharded else
                        f"replicas x{ws}" if ws > 1 else "single GPU"),
        "run": {"internal_sliced_edges": int(st["n_internal_sliced"]), "passes_per_slice": n_pass,
                "max_log2_elements": round(st["max_log2_elements"], 2), "gemm_engine": args.engine,
                "execution": ("each step replays its slices as one captured CUDA graph (tn_contract_slices_graph)"
                              if use_graph else "plain launches (tn_contract_slices)") +
                             "; the roofline's per-launch times come from a separate timed region of plain "
                             "launches with CUDA events around each (tn_profile_slices)",
                "plan_seconds": round(plan_s, 2), "order_trials": trials,
                "autotune_candidates": st["autotune_candidates"], "rank0_slices": [b0, e0_],
                "step_tuning": {"steps_off_default": int(st["n_tuned_steps"]),
                                "slice_ms_default_variants": round(st["tune_default_ms"], 3),
                                "slice_ms_tuned_variants": round(st["tune_tuned_ms"], 3)},
                "gemm_tiles": "CTA pairs (cta_group::2, 256x256) where they apply" if st["gemm_pair"] == 0 and
                              args.engine in ("fp16", "bf16") else "one-CTA 128-row tiles",
                "partial_slices_for_profiling": bool(args.slices) and "kept" not in cfg},
        "amplitudes_per_s": round(jobs * n_amp / (ms * 1e-3), 1),
        "slices_per_s": round(jobs * n_slices / (ms * 1e-3), 2),
        "ms_per_pass": round(ms / (n_slices * n_pass), 3),
        "tc_macs_per_slice": st["tc_macs"],
        "alg_bytes_per_slice": st["alg_bytes"],
        "e2e": {"value": round(e2e, 3), "unit": "TFLOP/s", "ms_per_step": round(ms_e2e, 3),
                "h2d_bytes_per_step": int(n_amp * 8), "d2h_bytes_per_step": int(n_amp * 16 + n_samples * 8 + 8)},
        "gpu_launches": int(args.steps * (n_slices * n_pass * n_launch + 4)),
        "roofline": roof,
        "clocks": clocks,
    }
    if "kept" in cfg:
        out["kept_slices"] = cfg["kept"]
        out["timed_slices_per_step"] = n_slices
        out["projected_s_for_kept_sum"] = round(ms * 1e-3 / n_slices * cfg["kept"], 1)
    if ws == 1 and not args.no_cpu_baseline and "kept" in cfg:
        out["cpu_baseline"] = {"unavailable": f"one (group, slice) unit of this network is {st['tc_macs']:.2e} complex "
                                              f"MACs on the planner's order (more on the oracle's own), far beyond a "
                                              f"bounded CPU sample"}
    elif ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(out), flush=True)


def _oracle_unit(cfg, i):
    """The oracle (O2, complex128 numpy tensordot) on (slice i mod 2^k, group
    i mod L) of the workload; returns its complex multiply-adds."""
    import oracle as O
    se = [(g, l) for (g, l, k, v) in cfg["edges"] if k == ci.EDGE_SLICE]
    k, L = len(se), len(cfg["tails"])
    stats = {}
    s = i % (1 << k)
    O.network_amplitudes(cfg["circuit"], cfg["open_qubits"], cfg["tails"], se, slice_range=(s, s + 1),
                         groups=[i % L], stats=stats)
    return stats["complex_macs"]


def _oracle_sample_text(cfg):
    return (f"one (group, slice) unit of {cfg['name']} ({1 << len(cfg['open_qubits'])} amplitude contributions) per "
            f"step: complex128 numpy tensordot on the oracle's own contraction order; flops = 8 x the oracle's "
            f"own complex multiply-adds")


def cpu_baseline(cfg, repeats=1):
    """The oracle on one (group, slice) unit of the same workload, as slice
    TFLOP/s counted on the oracle's own contraction (8 flops per complex
    multiply-add of its tensordots)."""
    t0 = time.time()
    macs = sum(_oracle_unit(cfg, r) for r in range(repeats))
    dt = time.time() - t0
    return {"value": round(8.0 * macs / dt / 1e12, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle", "seconds_per_unit": round(dt / repeats, 2), "complex_macs_per_unit": macs / repeats,
            "sample": _oracle_sample_text(cfg)}


def run_serve(args):
    """Serving form: a Poisson stream of amplitude-batch and sampling requests
    on a mix of circuits through the library's request server; p50/p99
    latency and throughput, tensor-core engine vs the plain complex64 engine."""
    import torch

    import paper_2111_03011_gb300 as tn
    torch.cuda.set_device(0)
    mix = ci.serving_mix()
    reqs = ci.poisson_requests(args.requests, args.rate, len(mix))
    rng = np.random.default_rng(11)
    bits_of = []
    for q in reqs:
        cfg = mix[q["circuit"]]
        if q["kind"] == 0:
            oq, tails = cfg["open_qubits"], cfg["tails"]
            g = rng.integers(0, len(tails), q["n"])
            mu = rng.integers(0, 1 << len(oq), q["n"]).astype(np.uint64)
            mask = np.uint64(sum(1 << x for x in oq))
            b = tails[g].astype(np.uint64) & ~mask
            for j, x in enumerate(oq):
                b |= ((mu >> np.uint64(j)) & np.uint64(1)) << np.uint64(x)
            bits_of.append(b)
        else:
            bits_of.append(None)
    results = {}
    for engine, gemm in (("fp16", tn.TN_GEMM_TC_FP16X3), ("bf16", tn.TN_GEMM_TC_BF16X3), ("tc", tn.TN_GEMM_TC_3XTF32),
                         ("simt", tn.TN_GEMM_SIMT_FP32)):
        plans = [tn.tn_plan(c["circuit"], c["open_qubits"], c["tails"], c["edges"], gemm=gemm, order_trials=16)
                 for c in mix]
        head_bytes = [tn.tn_plan_get_stats(p)["n_tails"] * (16 << tn.tn_plan_get_stats(p)["n_open"]) for p in plans]
        # cold start, and an HBM budget that holds about half of the heads, so
        # evicted heads are rebuilt (contracted) inside the measurement
        budget = max(max(head_bytes), sum(sorted(head_bytes)[: len(head_bytes) // 2 + 1]))
        sv = tn.tn_server_create(n_slots=8, hbm_budget_bytes=budget)
        for p in plans:
            k = tn.tn_plan_get_stats(p)["n_sliced"]
            tn.tn_server_add_circuit(sv, p, 0, 1 << k)
        base = 0
        t0 = time.time()
        tickets = []
        lat = []
        for q, b in zip(reqs, bits_of):
            dt = q["t"] - (time.time() - t0)
            if dt > 0:
                time.sleep(dt)
            if q["kind"] == 0:
                tickets.append(tn.tn_server_submit(sv, q["circuit"], tn.TN_REQ_AMPLITUDES, 0, bitstrings=b))
            else:
                tickets.append(tn.tn_server_submit(sv, q["circuit"], tn.TN_REQ_SAMPLE, q["n"], seed=q["seed"]))
        for t in tickets:
            lat.append(tn.tn_server_wait(sv, t)[1])
        wall = time.time() - t0
        st = tn.tn_server_get_stats(sv)
        lat = np.sort(np.array(lat))
        n_amp = sum(q["n"] for q in reqs if q["kind"] == 0)
        results[engine] = {"p50_ms": round(float(np.percentile(lat, 50)) / 1e3, 3),
                           "p99_ms": round(float(np.percentile(lat, 99)) / 1e3, 3),
                           "requests_per_s": round(len(reqs) / wall, 1),
                           "amplitudes_per_s": round(n_amp / wall, 1),
                           "completed": st["completed"] - base, "evictions": st["evictions"]}
        tn.tn_server_free(sv)
    out = {"metric": "p99 request latency", "value": results["fp16"]["p99_ms"], "unit": "ms",
           "higher_is_better": False, "n_gpus": 1, "mode": "serving",
           "config": {"workload": "poisson mix of 6 circuits (20-25 qubits, 8-12 cycles, 6-8 open, 32-256 tails)",
                      "cache": "cold start; HBM budget holds about half the heads (evicted heads are recontracted)",
                      "requests": args.requests, "rate_per_s": args.rate, "slots": 8,
                      "sizes": "amplitude batches 1e3-1e5 (log-uniform), samples 1e2-1e4"},
           "fp16x3": results["fp16"], "bf16x3": results["bf16"], "tc_3xtf32": results["tc"],
           "plain_c64_simt": results["simt"],
           "p99_vs_plain_c64": {k: round(results[k]["p99_ms"] / results["simt"]["p99_ms"], 3)
                                for k in ("fp16", "bf16", "tc")}}
    print(json.dumps(out), flush=True)


def run_torch(args):
    """Comparison arm, not the product: the same plan (leaves, order, sparse-
    state pattern maps from tn_plan_describe) contracted with stock PyTorch
    complex64 einsum on the GPU -- the software approach of the paper's own
    runs -- timed like the main arm (64 slices per step)."""
    import string

    import torch

    import paper_2111_03011_gb300 as tn
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    cfg = _workload(args.workload)
    popts = cfg.get("plan_opts", {})
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True,
                      order_trials=ORDER_TRIALS if args.workload in ("sliced30", "syc53") else 0, order_seed=1, **popts)
    st = tn.tn_plan_get_stats(plan)
    d = tn.tn_plan_describe(plan, with_data=True)
    tm = [int(t) & d["tail_mask"] for t in cfg["tails"]]
    L, h = len(tm), len(cfg["open_qubits"])

    def pats(tq):
        return sorted(set(t & tq for t in tm))

    leaves, vbits = [], []
    for lf in d["leaves"]:
        arr = (np.array(lf["re"]) + 1j * np.array(lf["im"])).astype(np.complex64)
        leaves.append(torch.from_numpy(arr.reshape(1 << len(lf["var_slice_bits"]), lf["P"], -1)).to(dev))
        vbits.append(lf["var_slice_bits"])
    vts = d["vts"]
    seen, ops = set(), []
    for stp in d["steps"]:
        if stp["contraction"] in seen:
            continue
        seen.add(stp["contraction"])
        a, b, c = stp["vt_a"], stp["vt_b"], stp["vt_c"]
        la, lb, lc = vts[a]["legs"], vts[b]["legs"], vts[c]["legs"]
        pa, pb, pc = pats(vts[a]["tq"]), pats(vts[b]["tq"]), pats(vts[c]["tq"])
        mA = [pa.index(x & vts[a]["tq"]) for x in pc]
        mB = [pb.index(x & vts[b]["tq"]) for x in pc]
        letter = {}
        for l in la + lb:
            letter.setdefault(l, string.ascii_letters[len(letter)])
        eq = ("Z" + "".join(letter[l] for l in reversed(la)) + ",Z" + "".join(letter[l] for l in reversed(lb)) +
              "->Z" + "".join(letter[l] for l in reversed(lc)))
        ops.append((a, b, c, None if mA == list(range(len(pa))) else torch.tensor(mA, device=dev),
                    None if mB == list(range(len(pb))) else torch.tensor(mB, device=dev), eq,
                    [len(pc)] + [2] * len(la), [len(pc)] + [2] * len(lb), len(pc)))
    fin = d["final"]
    fp = pats(d["tail_mask"])
    rowidx = torch.tensor([fp.index(t) for t in tm], device=dev)
    colidx = torch.tensor([sum(1 << fin["open_pos"][j] for j in range(h) if (mu >> j) & 1) for mu in range(1 << h)],
                          device=dev)
    H = torch.zeros(L, 1 << h, dtype=torch.complex128, device=dev)
    k, ni = st["n_sliced"], st["n_internal_sliced"]
    n_slices = min(1 << k, args.slices) if args.slices else 1 << k

    def one_pass(s):
        T = {}
        for i, vb in enumerate(vbits):
            T[i] = leaves[i][sum(((s >> bit) & 1) << t for t, bit in enumerate(vb))]
        for (a, b, c, mA, mB, eq, sa, sb, pc) in ops:
            A = T.pop(a)
            B = T.pop(b)
            A = A if mA is None else A.index_select(0, mA)
            B = B if mB is None else B.index_select(0, mB)
            T[c] = torch.einsum(eq, A.reshape(sa), B.reshape(sb)).reshape(pc, -1)
        H.add_(T[fin["vt"]].index_select(0, rowidx).index_select(1, colidx).to(torch.complex128))

    def step():
        H.zero_()
        for s in range(n_slices):
            for t in range(1 << ni):
                one_pass(s | (t << k))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    out = {"metric": "slice TFLOP/s", "value": round(8.0 * st["tc_macs"] * n_slices / (ms * 1e-3) / 1e12, 3),
           "unit": "TFLOP/s", "engine": "pytorch complex64 einsum (comparison arm, not the product)",
           "torch": torch.__version__, "allow_tf32": bool(torch.backends.cuda.matmul.allow_tf32),
           "ms_per_step": round(ms, 2), "steps": args.steps, "warmup": args.warmup,
           "config": {"workload": cfg["name"], "slices": n_slices, "order": "the planner's seed-1 order"}}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched form: 256 mixed grid circuits (16-28 qubits, 8-16 cycles) as
    parallel branches of one captured CUDA graph (tn_contract_batch) on the
    tensor-core engine, against the plain complex64 engine launching the
    circuits one after another."""
    import torch

    import paper_2111_03011_gb300 as tn
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    mix = ci.batch_mix(args.circuits)
    res = {}
    for engine, gemm, graph in (("tc_graph", tn.TN_GEMM_TC_3XTF32, True), ("fp16_graph", tn.TN_GEMM_TC_FP16X3, True),
                                ("simt_plain", tn.TN_GEMM_SIMT_FP32, False)):
        t0 = time.time()
        plans = [tn.tn_plan(c["circuit"], c["open_qubits"], c["tails"], c["edges"], gemm=gemm, order_trials=16,
                            max_log2_elements=26, auto_slice=8) for c in mix]
        plan_s = time.time() - t0
        stats = [tn.tn_plan_get_stats(p) for p in plans]
        heads = [tn.tn_head_create(p) for p in plans]
        ranges = [(0, 1 << st["n_sliced"]) for st in stats]
        flops = 8.0 * sum(st["tc_macs"] for st in stats)
        launches = sum(st["n_launches"] for st in stats)

        def step():
            for h in heads:
                tn.tn_head_reset(h, stream)
            if graph:
                tn.tn_contract_batch(plans, ranges, heads, stream)
            else:
                for p, r, h in zip(plans, ranges, heads):
                    tn.tn_contract_slices(p, r[0], r[1], h, stream)

        warm, steps = (args.warmup, args.steps) if graph else (1, 1)
        for _ in range(warm):
            step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[engine] = {"ms_per_batch": round(ms, 2), "TFLOP/s": round(flops / (ms * 1e-3) / 1e12, 2),
                       "circuits_per_s": round(len(mix) / (ms * 1e-3), 1), "steps": steps,
                       "launches_per_batch": launches, "plan_seconds": round(plan_s, 1),
                       "workspace_GB": round(sum(st["workspace_bytes"] for st in stats) / 1e9, 1)}
        del heads, plans
        torch.cuda.synchronize(dev)
    out = {"metric": "batch TFLOP/s", "value": res["tc_graph"]["TFLOP/s"], "unit": "TFLOP/s",
           "higher_is_better": True, "n_gpus": 1, "mode": "batched",
           "config": {"workload": f"{len(mix)} grid circuits, 16-28 qubits, 8-16 cycles, 6 open x 16 tails, "
                                  f"cap 2^26 with automatic slicing"},
           "engines": res,
           "tc_graph_vs_plain_c64": round(res["simt_plain"]["ms_per_batch"] / res["tc_graph"]["ms_per_batch"], 2),
           "fp16_graph_vs_plain_c64": round(res["simt_plain"]["ms_per_batch"] / res["fp16_graph"]["ms_per_batch"], 2)}
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The CPU oracle as the reference arm (the paper ships no code): one
    (group, slice) unit per step, on the host cores; the product library is
    not loaded."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = _workload(args.workload)
    k = sum(1 for e in cfg["edges"] if e[2] in (ci.EDGE_SLICE, ci.EDGE_COMPANION))
    n_slices = min(1 << k, args.slices) if args.slices else 1 << k
    for i in range(args.warmup):
        _oracle_unit(cfg, i)
    t0 = time.time()
    macs = sum(_oracle_unit(cfg, args.warmup + i) for i in range(args.steps))
    dt = (time.time() - t0) / args.steps
    v = 8.0 * macs / args.steps / dt / 1e12
    out = {"impl": "reference", "metric": "slice TFLOP/s", "value": round(v, 6), "unit": "TFLOP/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 1),
           "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None,
           "dtype": "c128", "data": "synthetic", "config": workload_config(cfg, n_slices),
           "cpu_baseline": {"value": round(v, 6), "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                            "seconds_per_unit": round(dt, 2), "complex_macs_per_unit": macs / args.steps,
                            "sample": _oracle_sample_text(cfg)},
           "e2e": {"value": round(v, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sliced30",
                    choices=["sliced30", "tiny", "grid25", "syc53", "precision40", "serve", "batch"])
    ap.add_argument("--circuits", type=int, default=256, help="batch workload: number of circuits")
    ap.add_argument("--engine", default="fp16", choices=["tc", "simt", "bf16", "fp16", "torch"],
                    help="GEMM-step engine: fp16 = FP16x3 (complex64 accuracy, default), tc = 3xTF32, "
                         "bf16 = BF16x3 (1e-4), simt = plain complex64 on CUDA cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=4,
                    help="plan candidates timed on the GPU by tn_plan_autotune (0: plain tn_plan)")
    ap.add_argument("--requests", type=int, default=300, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--slices", type=int, default=0,
                    help="contract only the first N slices per step (for ncu launch lists; not a bench number)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs, run the whole workload on each (weak scaling) instead of sharding "
                         "its slices")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "precision40" and not args.slices:
        args.slices = _workload("precision40")["default_slices"]
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(_spawn_ranks(args.gpus))
    if ws != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={ws}: launch one process per GPU")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.engine == "torch":
        run_torch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
