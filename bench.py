"""Benchmark of the batched Flowtree on GB300.

Workload (one "step"): the image-shaped configuration -- ground set = the
28x28 integer grid, 60,000 database and 1,000 query distributions of 100-200
pixels (synthetic Bezier strokes, mass proportional to intensity), quadtree
with L = 12 -- Flowtree for every (query, database) pair (6e7 pairs) in one
persistent launch, then the 10 nearest per query.  Inputs are resident in HBM;
L2 is flushed (a 512 MiB write) before every timed step.

Other legs reported on the same JSON line (rank 0): the plain one-launch-per-
pair form on a sample of the same pairs, forward+backward pairs/s on the
differentiation workload (30,000 x 300 vocabulary, 4,096 pairs), the
text-shaped kNN pipeline (quadtree scan -> top-1,000 -> Flowtree -> top-10),
the roofline of the dominant kernel, and the CPU oracle timed on the host.

Multi-GPU (torchrun): every rank runs its own query batch against the same
database (weak scaling, no data-path collective); value = all ranks' pairs /
the slowest rank's time.

--impl reference times the CPU oracle (the plain FP64 restatement of the
paper used by the tests) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

T_START = time.time()
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Flowtree pairs/s, batched vs per-pair GPU (rel err≤1e-5); fwd+bwd pairs/s"
UNIT = "pairs/s"
N_DB, N_Q, LEVELS, TOPK = 60000, 1000, 12, 10
WORKLOAD = ("image-shaped: 28x28 grid ground set, 60,000 db x 1,000 query distributions of 100-200 pixels, "
            "L=12, Flowtree for every query-database pair + top-10 per query")
ALU_LANES_PER_SM = 128  # FP32/INT32 lanes per SM (4 SMSPs x 32)
ALGO_NAMES = ["auto", "warp", "thread", "blocked"]  # ft_flowtree_config.algo
FLOW_KERNEL = {1: "k_flowtree_persistent", 2: "k_flowtree_thread", 3: "k_flowtree_blocked"}


def flow_kernel(tree, a, b) -> str:
    """The Flowtree kernel a batch of (a, b) pairs launches with the tree's configuration."""
    from paper_1910_04126_gb300 import _ffi
    algo = tree.get_config()[2]
    if algo == _ffi.ALGO_AUTO:
        maxn = ((a.info.max_support + b.info.max_support + 31) // 32) * 32
        algo = _ffi.ALGO_BLOCKED if maxn <= _ffi.BLOCKED_MAX_ITEMS else _ffi.ALGO_WARP
    name = FLOW_KERNEL[algo]
    if algo == _ffi.ALGO_BLOCKED and a.info.max_support + b.info.max_support > _ffi.BLOCKED_WARP_ITEMS:
        name += " + k_flowtree_team"  # the pairs beyond the warp's staging, a CTA each
    return name


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="small workload (smoke of the bench itself)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--skip-scale", action="store_true", help="omit the 1,000,000-document scale leg")
    ap.add_argument("--recall-oracle-queries", type=int, default=10,
                    help="scale leg: queries whose exhaustive top-10 the CPU oracle computes (on all host cores but "
                         "one, beside the GPU legs; about 40 s each on 16 Grace cores)")
    ap.add_argument("--profile-case", nargs=2, type=int, metavar=("N_DB", "N_Q"),
                    help="only run the image-shaped batch N_Q x N_DB three times (a case for ncu); no timing")
    ap.add_argument("--config", default="0,0,0", help="warps_per_cta,stage_items,algo for --profile-case")
    ap.add_argument("--profile-scan", nargs=2, type=int, metavar=("N_DB", "N_Q"),
                    help="only run the quadtree scan + top-1,000 of N_Q text-shaped queries over N_DB documents "
                         "(vocabulary 100,000 x 300) three times (a case for ncu); no timing")
    ap.add_argument("--profile-exact", nargs=2, type=int, metavar=("N_Q", "PER_Q"),
                    help="only run exact W1 on N_Q text-shaped queries x PER_Q random documents of 20,000 "
                         "(vocabulary 100,000 x 300) three times (a case for ncu); no timing")
    ap.add_argument("--profile-text", type=int, metavar="N_Q",
                    help="only run the Flowtree launch of the text pipeline (N_Q queries x their 1,000 quadtree "
                         "candidates of 100,000 documents, vocabulary 100,000 x 300, launch configuration from "
                         "--config) three times (a case for ncu); no timing")
    ap.add_argument("--profile-backward", type=int, metavar="N_PAIRS",
                    help="only run forward (flows saved) + backward on N_PAIRS pairs of the differentiation workload "
                         "(vocabulary 30,000 x 300) three times (a case for ncu); no timing")
    return ap.parse_args()


def profile_case(args):
    import torch
    from paper_1910_04126_gb300 import api, synth
    n_db, n_q = args.profile_case
    db, q = synth.stroke_images(n_db, 202), synth.stroke_images(n_q, 203)
    tree = api.Tree(torch.as_tensor(synth.grid_points(), device="cuda"), LEVELS, synth.random_shift(2, 201))
    tree.set_config(*[int(x) for x in args.config.split(",")])
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    out = torch.empty(n_db * n_q, device="cuda")
    for _ in range(3):
        api.flowtree_batch(tree, tree.points, Q, D, out=out)
    torch.cuda.synchronize()
    print("profile case done: %d pairs, config %s, status %d" % (n_db * n_q, args.config, tree.status()))


def profile_scan(args):
    import torch
    from paper_1910_04126_gb300 import api, synth
    n_db, n_q = args.profile_scan
    vocab = synth.mixture_vocab(100000, 300, 1000, 0.3, 500)
    db = synth.zipf_docs_bulk(100000, n_db, 502, device="cuda")
    q = synth.zipf_docs_bulk(100000, n_q, 503, device="cuda")
    tree = api.Tree(torch.as_tensor(vocab, device="cuda"), LEVELS, synth.random_shift(300, 501))
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    k1 = min(1000, n_db)
    ws = torch.empty(api._ffi.load().ft_quadtree_scan_workspace_size(tree.handle, Q.handle, D.handle, k1),
                     dtype=torch.uint8, device="cuda")
    for _ in range(3):
        api.quadtree_scan(tree, Q, D, k1, workspace=ws)
    torch.cuda.synchronize()
    print("profile scan done: %d x %d, %d db embedding entries, status %d"
          % (n_q, n_db, D.info.n_embed, tree.status()))


def profile_exact(args):
    import torch
    from paper_1910_04126_gb300 import api, synth
    n_q, per_q = args.profile_exact
    vocab = synth.mixture_vocab(100000, 300, 1000, 0.3, 300)
    db = synth.zipf_docs(100000, 20000, 302)
    q = synth.zipf_docs(100000, n_q, 303)
    tree = api.Tree(torch.as_tensor(vocab, device="cuda"), LEVELS, synth.random_shift(300, 301))
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    rng = np.random.default_rng(0)
    pa = torch.as_tensor(np.repeat(np.arange(n_q), per_q), dtype=torch.int32, device="cuda")
    pb = torch.as_tensor(rng.integers(0, db.n, n_q * per_q), dtype=torch.int32, device="cuda")
    ws = torch.empty(api.exact_w1_workspace_size(Q, D, n_q * per_q), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        api.exact_w1(tree, tree.points, Q, D, pa, pb, workspace=ws)
    torch.cuda.synchronize()
    print("profile exact done: %d pairs, status %d" % (n_q * per_q, tree.status()))


def profile_text(args):
    import torch
    from paper_1910_04126_gb300 import api, synth
    n_q, k1 = args.profile_text, 1000
    vocab = synth.mixture_vocab(100000, 300, 1000, 0.3, 300)
    db, q = synth.zipf_docs(100000, 100000, 302), synth.zipf_docs(100000, n_q, 303)
    tree = api.Tree(torch.as_tensor(vocab, device="cuda"), LEVELS, synth.random_shift(300, 301))
    tree.set_config(*[int(x) for x in args.config.split(",")])
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    cand = api.quadtree_scan(tree, Q, D, k1).reshape(-1)
    pa = torch.arange(n_q, dtype=torch.int32, device="cuda").repeat_interleave(k1)
    for _ in range(3):
        api.flowtree_batch(tree, tree.points, Q, D, pa, cand)
    torch.cuda.synchronize()
    print("profile text done: %d pairs, config %s, status %d" % (n_q * k1, args.config, tree.status()))


def profile_backward(args):
    import torch
    from paper_1910_04126_gb300 import api, synth
    n = args.profile_backward
    wl = synth.diff_pairs(n_words=30000, n_pairs=n)
    tree = api.Tree(torch.as_tensor(wl.points, device="cuda"), wl.levels, wl.shift)
    tree.set_config(*[int(x) for x in args.config.split(",")])
    A, B = api.Docs.from_csr(tree, wl.db), api.Docs.from_csr(tree, wl.queries)
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    flows = api.Flows(tree, A, B, idx, idx)
    gcost = torch.ones(n, device="cuda")
    gv = torch.zeros_like(tree.points)
    for _ in range(3):
        api.flowtree_batch(tree, tree.points, A, B, flows.pair_a, flows.pair_b, flows=flows)
        api.flowtree_backward(tree, A, B, flows, tree.points, gcost, grad_vocab=gv)
    torch.cuda.synchronize()
    print("profile backward done: %d pairs, config %s, status %d" % (n, args.config, tree.status()))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
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
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_image(rank: int, quick: bool):
    from paper_1910_04126_gb300 import synth
    n_db, n_q = (6000, 100) if quick else (N_DB, N_Q)
    pts = synth.grid_points()
    shift = synth.random_shift(2, 201)
    db = synth.stroke_images(n_db, 202)
    q = synth.stroke_images(n_q, 203 + 1000 * rank)
    return pts, shift, db, q


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("ft_flow.cuh", "ft_flow_blocked.cuh", "ft_flow.cu"):
        with open(os.path.join(ROOT, "paper_1910_04126_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(n_pairs: int):
    """DRAM bytes per launch from the committed ncu summary, if it matches this kernel."""
    p = os.path.join(ROOT, "profiles", "flowtree_image_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_pair"]) * n_pairs


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(pts, shift, db, q, target_s: float, n_threads: int, seed: int = 0):
    import oracle as O
    ot = O.OracleTree(pts, LEVELS, shift)
    rng = np.random.default_rng(seed)
    sq = ot.embed_docs(q.row_ptr, q.word, q.weight)
    sd = ot.embed_docs(db.row_ptr, db.word, db.weight)
    n = 256
    while True:
        pa = rng.integers(0, q.n, n)
        pb = rng.integers(0, db.n, n)
        t0 = time.perf_counter()
        ot.flowtree_batch(pts, sq, sd, pa, pb, n_threads=n_threads)
        dt = time.perf_counter() - t0
        if dt >= target_s or n >= 1 << 24:
            return n / dt, n, dt
        n = int(min(n * max(2.0, 1.2 * target_s / max(dt, 1e-3)), 1 << 24))


def host_cpu() -> dict:
    """The host CPU the oracle ran on: nproc, machine, and lscpu's model name and sockets when available."""
    import platform
    import subprocess
    info = {"nproc": os.cpu_count() or 1, "machine": platform.machine()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() in ("Model name", "Socket(s)", "Core(s) per socket", "Thread(s) per core"):
                info[key.strip().lower().replace(" ", "_").replace("(s)", "s")] = val.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return info


def run_reference(args, rank, world):
    if rank != 0:
        return
    pts, shift, db, q = make_image(0, args.quick)
    cores = os.cpu_count() or 1
    rates = []
    sample = None
    per_step = 8.0 if not args.quick else 1.0
    total = args.warmup + args.steps
    for i in range(total):
        r, n, dt = oracle_rate(pts, shift, db, q, per_step, cores, seed=i)
        sample = n
        if i >= args.warmup:
            rates.append(r)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "random (query, db) pairs of the workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
                         "sample": "%d random pairs per step of the %s workload" % (sample, "quick" if args.quick else "full")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case:
        profile_case(args)
        return
    if args.profile_scan:
        profile_scan(args)
        return
    if args.profile_exact:
        profile_exact(args)
        return
    if args.profile_backward:
        profile_backward(args)
        return
    if args.profile_text:
        profile_text(args)
        return

    import torch
    import torch.distributed as dist
    from paper_1910_04126_gb300 import api
    from paper_1910_04126_gb300 import build as fbuild

    if not os.path.exists(fbuild.LIB):
        fbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    pts, shift, db_h, q_h = make_image(rank, args.quick)
    tree = api.Tree(torch.as_tensor(pts, device=dev), LEVELS, shift)
    D = api.Docs.from_csr(tree, db_h)
    Q = api.Docs.from_csr(tree, q_h)
    # launch configuration picked by the library's autotuner on a 50-query sample
    Qs = api.Docs.from_csr(tree, q_h.subset(np.arange(min(50, q_h.n))))
    tuned = api.flowtree_autotune(tree, tree.points, Qs, D)
    del Qs
    nq, nd = Q.n_docs, D.n_docs
    n_pairs = nq * nd
    vocab = tree.points
    costs = torch.empty(n_pairs, dtype=torch.float32, device=dev)
    ws = torch.empty(api.flowtree_workspace_size(tree, Q, D, n_pairs), dtype=torch.uint8, device=dev)
    ids = torch.empty((nq, TOPK), dtype=torch.int32, device=dev)
    vals = torch.empty((nq, TOPK), dtype=torch.float32, device=dev)
    from paper_1910_04126_gb300 import _ffi
    ws_topk = torch.empty(_ffi.load().ft_topk_f32_workspace_size(nq, nd), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    k_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step(record_kernel=None):
        if record_kernel is not None:
            record_kernel[0].record(stream)
        api.flowtree_batch(tree, vocab, Q, D, out=costs, workspace=ws)
        if record_kernel is not None:
            record_kernel[1].record(stream)
        api.topk_f32(costs.view(nq, nd), TOPK, ids=ids, vals=vals, workspace=ws_topk)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(k_ev)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(k_ev[0].elapsed_time(k_ev[1]))
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = clk.summary()
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n_pairs / (ms * 1e-3)

    # end to end through the public API, host buffers in and out
    rp = torch.as_tensor(q_h.row_ptr).pin_memory()
    wd = torch.as_tensor(q_h.word).pin_memory()
    wt = torch.as_tensor(q_h.weight).pin_memory()
    ids_h = torch.empty((nq, TOPK), dtype=torch.int32).pin_memory()
    vals_h = torch.empty((nq, TOPK), dtype=torch.float32).pin_memory()
    h2d = rp.numel() * 8 + wd.numel() * 4 + wt.numel() * 4
    d2h = ids_h.numel() * 4 + vals_h.numel() * 4

    def e2e_step():
        Qe = api.Docs(tree, rp.to(dev, non_blocking=True), wd.to(dev, non_blocking=True),
                      wt.to(dev, non_blocking=True))
        api.flowtree_batch(tree, vocab, Qe, D, out=costs, workspace=ws)
        api.topk_f32(costs.view(nq, nd), TOPK, ids=ids, vals=vals, workspace=ws_topk)
        ids_h.copy_(ids, non_blocking=True)
        vals_h.copy_(vals, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    barrier()
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = world * n_pairs / (statistics.mean(e2e_ms) * 1e-3)

    pk, pk_kind = peaks()
    # algorithmic work of the dominant kernel (the Flowtree launch), per launch:
    # (L+2)(s_mu+s_nu) integer scan steps + (s_mu+s_nu-1)(3d+1) FLOP per pair
    lq = np.diff(q_h.row_ptr).astype(np.float64)
    ld = np.diff(db_h.row_ptr).astype(np.float64)
    S = nd * lq.sum() + nq * ld.sum()  # sum over pairs of s_mu + s_nu
    d = 2
    ops = (LEVELS + 2) * S + (3 * d + 1) * (S - n_pairs)
    kms = statistics.mean(kern_ms)
    sm_clock = pk.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * ALU_LANES_PER_SM * sm_clock * 1e6
    achieved = ops / (kms * 1e-3)
    traffic = profiled_traffic(n_pairs)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + (" [quick]" if args.quick else ""), "pairs_per_step_per_gpu": n_pairs,
                   "l2": "flushed (512 MiB write) before every timed step", "parallelism": "weak, %d shard(s)" % world,
                   "launch_config": {"warps_per_cta": tuned[0], "stage_items": tuned[1],
                                     "algo": ALGO_NAMES[tuned[2]], "stage_tables": tuned[3],
                                     "picked_by": "ft_flowtree_autotune"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms)},
        # per step: the Flowtree launch, then keys + select
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": flow_kernel(tree, Q, D), "kernel_ms": kms,
                     "peak_basis": "%d SMs x %d lanes x %.0f MHz (%s sm_max_mhz)" % (n_sm, ALU_LANES_PER_SM, sm_clock, pk_kind)},
    }
    if rank == 0:
        progress("main leg: %.4g pairs/s" % value)
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(extras(args, tree, D, Q, q_h, db_h, pts, shift, value, dev, pk, pk_kind))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def progress(msg):
    """One line per finished leg on stderr (the JSON line alone goes to stdout)."""
    print("[bench %7.1f s] %s" % (time.time() - T_START, msg), file=sys.stderr, flush=True)


def extras(args, tree, D, Q, q_h, db_h, pts, shift, batched_value, dev, pk, pk_kind):
    import torch
    from paper_1910_04126_gb300 import api, synth
    out = {}
    # CPU oracle on the host cores (bounded sample of the same image workload), first: nothing else runs on
    # the host cores meanwhile
    cores = os.cpu_count() or 1
    r_n, n_n, dt_n = oracle_rate(pts, shift, db_h, q_h, 12.0 if not args.quick else 2.0, cores, seed=1)
    r_1, n_1, dt_1 = oracle_rate(pts, shift, db_h, q_h, 3.0 if not args.quick else 0.5, 1, seed=2)
    out["cpu_baseline"] = {"value": r_n, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": "%d random (query, db) pairs of the image workload, %.1f s" % (n_n, dt_n),
                           "single_thread": {"value": r_1, "sample_pairs": n_1}, "host": host_cpu()}
    progress("cpu baseline")
    recall_job = None
    scale_data = None
    if not args.skip_scale:
        try:  # the scale workload first, so that the oracle's recall reference runs beside all the GPU legs
            scale_data = make_scale_data(args, dev)
            recall_job = OracleRecall(scale_data["vocab"], scale_data["shift"], scale_data["db"], scale_data["q"],
                                      max(0, args.recall_oracle_queries if not args.quick else 1), TOPK)
            recall_job.start()
        except Exception as ex:  # report, do not lose the main line
            out["scale_knn_pipeline"] = {"error": "%s: %s" % (type(ex).__name__, ex)}
    progress("scale data made, oracle recall started")
    # plain one-launch-per-pair form on a sample of the same pairs
    n_plain = 2000
    rng = np.random.default_rng(5)
    pa = torch.as_tensor(rng.integers(0, Q.n_docs, n_plain), dtype=torch.int32, device=dev)
    pb = torch.as_tensor(rng.integers(0, D.n_docs, n_plain), dtype=torch.int32, device=dev)
    api.flowtree_plain(tree, tree.points, Q, D, pa, pb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.flowtree_plain(tree, tree.points, Q, D, pa, pb)
    e1.record()
    e1.synchronize()
    plain = n_plain / (e0.elapsed_time(e1) * 1e-3)
    out["plain_per_pair"] = {"value": plain, "unit": UNIT, "sample_pairs": n_plain,
                             "batched_speedup": batched_value / plain}
    out["match_depth_histogram"] = depth_histogram(tree, Q, D, pa, pb)

    progress("plain form, depth histogram")
    # forward + backward (differentiation workload)
    nw, npairs = (30000, 4096) if not args.quick else (5000, 512)
    wl = synth.diff_pairs(n_words=nw, n_pairs=npairs)
    t2 = api.Tree(torch.as_tensor(wl.points, device=dev), wl.levels, wl.shift)
    A, B = api.Docs.from_csr(t2, wl.db), api.Docs.from_csr(t2, wl.queries)
    idx = torch.arange(npairs, dtype=torch.int32, device=dev)
    tuned_fb = api.flowtree_autotune(t2, t2.points, A, B, idx, idx)
    flows = api.Flows(t2, A, B, idx, idx)
    cst = torch.empty(npairs, device=dev)
    gcost = torch.ones(npairs, device=dev)
    gv = torch.zeros_like(t2.points)
    fws = torch.empty(api.flowtree_workspace_size(t2, A, B, npairs), dtype=torch.uint8, device=dev)
    bws = torch.empty(int(api._ffi.load().ft_flowtree_backward_workspace_size(t2.handle, flows.handle)),
                      dtype=torch.uint8, device=dev)

    def fb():
        api.flowtree_batch(t2, t2.points, A, B, flows.pair_a, flows.pair_b, flows=flows, out=cst, workspace=fws)
        api.flowtree_backward(t2, A, B, flows, t2.points, gcost, grad_vocab=gv, workspace=bws)

    # the step a user writes: loss = sum of Flowtree values through torch.autograd, the adjoint into the
    # vocabulary's gradient; the flows are held by the caller (created once for these pairs)
    vparam = t2.points.clone().requires_grad_(True)

    def fb_autograd(fl):
        vparam.grad = None
        api.flowtree(vparam, t2, A, B, idx, idx, flows=fl).sum().backward()

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = 10
    fb_ms = timed(lambda: fb_autograd(flows), reps)
    rebind = api.Flows.with_capacity(t2, A, B, npairs)
    fb_rebind_ms = timed(lambda: fb_autograd(rebind))
    raw_ms = timed(fb)
    e0.record()
    for _ in range(reps):
        api.flowtree_batch(t2, t2.points, A, B, flows.pair_a, flows.pair_b, out=cst, workspace=fws)
    e1.record()
    e1.synchronize()
    f_ms = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        api.flowtree_backward(t2, A, B, flows, t2.points, gcost, grad_vocab=gv, workspace=bws)
    e1.record()
    e1.synchronize()
    b_ms = e0.elapsed_time(e1) / reps
    out["fwd_bwd"] = {"value": npairs / (fb_ms * 1e-3), "unit": UNIT, "forward_only": npairs / (f_ms * 1e-3),
                      "ms_per_step": fb_ms, "backward_ms": b_ms,
                      "path": "torch.autograd: api.flowtree(vocab, ...).sum().backward(), caller-held flows",
                      "launch_config": {"warps_per_cta": tuned_fb[0], "stage_items": tuned_fb[1],
                                        "algo": ALGO_NAMES[tuned_fb[2]], "deep_loads": tuned_fb[4],
                                        "picked_by": "ft_flowtree_autotune"},
                      "raw_api_ms_per_step": raw_ms,
                      "rebinding_flows": {"value": npairs / (fb_rebind_ms * 1e-3), "ms_per_step": fb_rebind_ms,
                                          "note": "Flows.with_capacity rebound every step (pairs may change)"},
                      "workload": "vocab %d x 300 (1,000-cluster mixture), %d doc pairs, lengths 20-300" % (nw, npairs)}

    progress("fwd+bwd")
    # text-shaped kNN pipeline
    nwt, ndb, nqt, k1 = (100000, 100000, 1000, 1000) if not args.quick else (20000, 10000, 100, 256)
    V = synth.mixture_vocab(nwt, 300, 1000, 0.3, 300)
    t3 = api.Tree(torch.as_tensor(V, device=dev), 12, synth.random_shift(300, 301))
    tdb = synth.zipf_docs(nwt, ndb, 302)
    tq = synth.zipf_docs(nwt, nqt, 303)
    D3, Q3 = api.Docs.from_csr(t3, tdb), api.Docs.from_csr(t3, tq)
    # launch configuration for these documents, tuned on a 2-query cross product
    Qs3 = api.Docs.from_csr(t3, tq.subset(np.arange(2)))
    tuned3 = api.flowtree_autotune(t3, t3.points, Qs3, D3)
    del Qs3
    kws = torch.empty(api.knn_workspace_size(t3, D3, Q3, k1, TOPK), dtype=torch.uint8, device=dev)
    kid = torch.empty((nqt, TOPK), dtype=torch.int32, device=dev)
    kdist = torch.empty((nqt, TOPK), dtype=torch.float32, device=dev)
    for _ in range(2):
        api.knn(t3, t3.points, D3, Q3, k1, TOPK, workspace=kws, ids=kid, dist=kdist)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.knn(t3, t3.points, D3, Q3, k1, TOPK, workspace=kws, ids=kid, dist=kdist)
    g.replay()
    torch.cuda.synchronize()
    lat = []
    for _ in range(5):
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    ms3 = statistics.median(lat)
    out["text_knn_pipeline"] = {
        "flowtree_pairs_per_s": nqt * k1 / (ms3 * 1e-3), "queries_per_s": nqt / (ms3 * 1e-3),
        "scan_pairs_per_s": nqt * ndb / (ms3 * 1e-3), "batch_ms_median": ms3, "graph": True,
        "launch_config": list(tuned3),
        "scan_roofline": scan_roofline(t3, Q3, D3, pk, pk_kind),
        "flowtree_roofline": text_flowtree_roofline(t3, Q3, D3, tq, tdb, k1, dev, pk, pk_kind),
        "workload": "vocab %d x 300, %d docs (log-normal lengths, Zipf(1.1) words), %d queries, top-%d -> top-%d"
                    % (nwt, ndb, nqt, k1, TOPK)}

    progress("text pipeline")
    # the Mean method (centroid distance) as the first stage instead of the quadtree
    try:
        mws = torch.empty(api._ffi.load().ft_mean_scan_workspace_size(Q3.handle, D3.handle, k1), dtype=torch.uint8,
                          device=dev)
        api.mean_scan(t3, t3.points, Q3, D3, k1, workspace=mws)
        torch.cuda.synchronize()
        e0.record()
        m_ids, _ = api.mean_scan(t3, t3.points, Q3, D3, k1, workspace=mws)
        e1.record()
        e1.synchronize()
        mean_ms = e0.elapsed_time(e1)
        del mws
        q_ids = api.quadtree_scan(t3, Q3, D3, k1)
        # exhaustive Flowtree top-10 of the first queries: how much of it each first stage keeps
        nx = min(50, nqt)
        Qx = api.Docs.from_csr(t3, tq.subset(np.arange(nx)))
        costs = api.flowtree_batch(t3, t3.points, Qx, D3)
        ex_ids, _ = api.topk_f32(costs.view(nx, ndb), TOPK)
        del costs
        ex, mi, qi = ex_ids.cpu().numpy(), m_ids[:nx].cpu().numpy(), q_ids[:nx].cpu().numpy()
        out["text_mean_prefilter"] = {
            "scan_ms": mean_ms, "pairs_per_s": nqt * ndb / (mean_ms * 1e-3), "k1": k1,
            "exhaustive_flowtree_top10_kept_by_mean_top_k1": float(np.mean([len(set(e) & set(m)) / TOPK
                                                                          for e, m in zip(ex, mi)])),
            "exhaustive_flowtree_top10_kept_by_quadtree_top_k1": float(np.mean([len(set(e) & set(q_)) / TOPK
                                                                              for e, q_ in zip(ex, qi)])),
            "queries_checked": nx,
            "stage": "centroid distances: FP32 centroids, tiled FP32 cross terms with the distance epilogue fused, radix select of the k1 smallest per query (ft_mean_scan)"}
    except Exception as ex:  # report, do not lose the main line
        out["text_mean_prefilter"] = {"error": "%s: %s" % (type(ex).__name__, ex)}

    progress("mean prefilter")
    # three-stage pipeline: quadtree -> top-1,000 -> Flowtree -> top-20 -> exact W1 -> top-10
    try:
        nq_x = 100 if not args.quick else 20
        Qx3 = api.Docs.from_csr(t3, tq.subset(np.arange(nq_x)))
        k2 = 2 * TOPK  # Flowtree as an intermediate stage keeps c = max(10, 2 c_next)
        kx = min(k1, 1000)
        wsx = torch.empty(api.knn_exact_workspace_size(t3, D3, Qx3, kx, k2, TOPK), dtype=torch.uint8, device=dev)
        api.knn_exact(t3, t3.points, D3, Qx3, kx, k2, TOPK, workspace=wsx)
        torch.cuda.synchronize()
        e0.record()
        ex_ids, ex_d = api.knn_exact(t3, t3.points, D3, Qx3, kx, k2, TOPK, workspace=wsx)
        e1.record()
        e1.synchronize()
        msx = e0.elapsed_time(e1)
        ft_ids, _ = api.knn(t3, t3.points, D3, Qx3, kx, TOPK)
        a_, b_ = ex_ids.cpu().numpy(), ft_ids.cpu().numpy()
        out["text_knn_exact_pipeline"] = {
            "batch_ms": msx, "queries": nq_x, "k1": kx, "k2": k2, "k": TOPK,
            "exact_pairs_per_s": nq_x * k2 / (msx * 1e-3),
            "top10_overlap_with_flowtree_only": float(np.mean([len(set(x) & set(y)) / TOPK for x, y in zip(a_, b_)])),
            "stage": "exact W1 by successive shortest paths, one warp per pair (ft_exact_w1_batch)"}
        del wsx
    except Exception as ex:  # report, do not lose the main line
        out["text_knn_exact_pipeline"] = {"error": "%s: %s" % (type(ex).__name__, ex)}

    progress("three-stage pipeline")
    if scale_data is not None:
        try:
            out["scale_knn_pipeline"], got, lib = scale_leg(args, dev, pk, pk_kind, scale_data)
            recall_job.got, recall_job.lib = got, lib
        except Exception as ex:  # report, do not lose the main line
            out["scale_knn_pipeline"] = {"error": "%s: %s" % (type(ex).__name__, ex)}

    progress("scale pipeline")
    # random-model planted experiment (Sec. 4.2 model, Sec. 5.1 figure "Results on random data")
    try:
        from paper_1910_04126_gb300 import planted
        t0 = time.time()
        ns_a = [20, 50, 100, 1000, 10000, 100000] if not args.quick else [20, 100]
        ns_b = [200, 1000, 3000] if not args.quick else [200]
        pa_ = planted.run(ns_a, dim=10, s=10, eps=0.25, reps=100 if not args.quick else 10, seed=0)
        pb_ = planted.run(ns_b, dim=10, s=100, eps=0.4, reps=30 if not args.quick else 5, seed=1)
        ra_ = planted.run(ns_a, dim=10, s=10, eps=0.25, reps=100 if not args.quick else 10, seed=0,
                          competitors="random")
        rb_ = planted.run(ns_b, dim=10, s=100, eps=0.4, reps=30 if not args.quick else 5, seed=1,
                          competitors="random")
        out["planted_random_model"] = {
            "competitors": "planted support vs all s(N-s) single swaps; success = strictly smallest score",
            "d10_s10_eps0.25": pa_["results"], "d10_s100_eps0.4": pb_["results"],
            "vs_random_subsets": {"competitors": "planted support vs 2,000 uniformly random s-subsets of X",
                                  "d10_s10_eps0.25": ra_["results"], "d10_s100_eps0.4": rb_["results"]},
            "wall_s": time.time() - t0}
    except Exception as ex:  # report, do not lose the main line
        out["planted_random_model"] = {"error": "%s: %s" % (type(ex).__name__, ex)}

    progress("planted experiment")
    if recall_job is not None:  # the oracle's exhaustive Flowtree of the scale leg, run beside the legs above
        recall_job.join()
        sc = out.get("scale_knn_pipeline", {})
        if "oracle_top10" in recall_job.result and isinstance(sc, dict) and "error" not in sc and \
                len(recall_job.result["oracle_top10"]):
            ref = recall_job.result["oracle_top10"]
            n_or = len(ref)
            got, lib = recall_job.got[:n_or], recall_job.lib[:n_or]
            sc["recall_at_10_vs_oracle"] = float(np.mean([len(set(got[i]) & set(ref[i])) / TOPK
                                                          for i in range(n_or)]))
            sc["library_exhaustive_vs_oracle_top10"] = float(np.mean([len(set(lib[i]) & set(ref[i])) / TOPK
                                                                      for i in range(n_or)]))
            sc["oracle_recall_queries"] = n_or
            sc["oracle_recall_s"] = recall_job.result["wall_s"]
            sc["oracle_recall_threads"] = recall_job.result["threads"]
        elif isinstance(sc, dict):
            sc["oracle_recall_error"] = recall_job.result.get("error", "not run")
    progress("oracle recall joined")
    out["roofline_hbm"] = hbm_roofline(q_h, db_h, batched_value, pk, pk_kind)
    return out


def make_scale_data(args, dev):
    """The scale workload: 400,000 x 300 vocabulary, 1,000,000 documents, a 256-query batch."""
    from paper_1910_04126_gb300 import synth
    n_words, n_db, nq = (400000, 1000000, 256) if not args.quick else (20000, 20000, 64)
    t0 = time.time()
    d = {"vocab": synth.mixture_vocab(n_words, 300, 1000, 0.3, 500), "shift": synth.random_shift(300, 501),
         "db": synth.zipf_docs_bulk(n_words, n_db, 502, device=str(dev)),
         "q": synth.zipf_docs_bulk(n_words, nq, 503, device=str(dev))}
    d["gen_s"] = time.time() - t0
    return d


def scale_leg(args, dev, pk, pk_kind, data):
    """Scale configuration: 400,000 x 300 vocabulary, 1,000,000 documents, 256-query batches.

    quadtree scan -> top-1,000 -> batched Flowtree -> top-10, captured once as a
    CUDA graph and replayed; p50/p99 batch latency over the replays; recall@10
    of the pipeline against exhaustive Flowtree (no prefilter) over all
    documents for the first 100 queries.
    """
    import torch
    from paper_1910_04126_gb300 import api, synth
    n_words, n_db, nq, k1, k = (400000, 1000000, 256, 1000, TOPK) if not args.quick else (20000, 20000, 64, 200, TOPK)
    vocab, db, q, gen_s = data["vocab"], data["db"], data["q"], data["gen_s"]
    t0 = time.time()
    tree = api.Tree(torch.as_tensor(vocab, device=dev), LEVELS, data["shift"])
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    torch.cuda.synchronize()
    prep_s = time.time() - t0
    # launch configuration for these documents, tuned on a 2-query cross product
    Qs = api.Docs.from_csr(tree, q.subset(np.arange(2)))
    tuned = api.flowtree_autotune(tree, tree.points, Qs, D)
    del Qs
    ws = torch.empty(api.knn_workspace_size(tree, D, Q, k1, k), dtype=torch.uint8, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            api.knn(tree, tree.points, D, Q, k1, k, workspace=ws, ids=ids, dist=dist, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.knn(tree, tree.points, D, Q, k1, k, workspace=ws, ids=ids, dist=dist)
    g.replay()
    torch.cuda.synchronize()
    lat = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(20):
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat.sort()
    p50, p99 = lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    # exhaustive Flowtree for the first queries: the recall reference
    n_ex = min(100, nq)
    Qx = api.Docs.from_csr(tree, q.subset(np.arange(n_ex)))
    costs = api.flowtree_batch(tree, tree.points, Qx, D)
    ex_ids, _ = api.topk_f32(costs.view(n_ex, n_db), k)
    del costs
    got, ref = ids[:n_ex].cpu().numpy(), ex_ids.cpu().numpy()
    recall = float(np.mean([len(set(got[i]) & set(ref[i])) / k for i in range(n_ex)]))
    return {"flowtree_pairs_per_s": nq * k1 / (p50 * 1e-3), "scan_pairs_per_s": nq * n_db / (p50 * 1e-3),
            "batch_ms_p50": p50, "batch_ms_p99": p99, "replays": len(lat), "graph": True,
            "scan_roofline": scan_roofline(tree, Q, D, pk, pk_kind),
            "recall_at_10_vs_exhaustive_flowtree": recall, "recall_queries": n_ex,
            "generate_s": gen_s, "tree_and_embed_s": prep_s, "launch_config": list(tuned),
            "db_items": int(D.info.n_items), "db_embed_entries": int(D.info.n_embed),
            "workload": "vocab %d x 300, %d docs (log-normal median 150, 10-2,000 words, Zipf(1.05)), "
                        "%d-query batch, top-%d -> top-%d" % (n_words, n_db, nq, k1, k)}, got, ref


class OracleRecall(threading.Thread):
    """The oracle's exhaustive Flowtree top-k (FP64, every document) of the first n_q queries: the reference for
    the scale pipeline's recall, computed on all host cores but one in a background thread (the oracle is C++
    behind ctypes, which releases the interpreter lock) while the GPU legs run."""

    def __init__(self, vocab, shift, db, q, n_q, k):
        super().__init__(daemon=True)
        self.vocab, self.shift, self.db, self.q, self.n_q, self.k = vocab, shift, db, q, n_q, k
        self.result = {}

    def run(self):
        try:
            # lowest CPU priority for this thread and the oracle's worker threads (which inherit it on Linux),
            # so that the GPU legs' host work and its BLAS threads are not starved meanwhile
            try:
                os.setpriority(os.PRIO_PROCESS, 0, 19)
            except (AttributeError, OSError):
                pass
            import oracle as O
            t0 = time.time()
            threads = max(1, (os.cpu_count() or 2) - 1)
            ot = O.OracleTree(self.vocab, LEVELS, self.shift)
            Sd = ot.embed_docs(self.db.row_ptr, self.db.word, self.db.weight)
            qs = self.q.subset(np.arange(self.n_q))
            Sq = ot.embed_docs(qs.row_ptr, qs.word, qs.weight)
            nd = self.db.n
            tops = []
            for qi in range(self.n_q):
                c = ot.flowtree_batch(self.vocab, Sq, Sd, np.full(nd, qi), np.arange(nd), n_threads=threads)
                tops.append(O.topk_ids(c, self.k))
            self.result = {"oracle_top10": np.stack(tops), "wall_s": time.time() - t0, "threads": threads}
        except Exception as ex:  # reported in the line
            self.result = {"error": "%s: %s" % (type(ex).__name__, ex)}


def depth_histogram(tree, Q, D, pa, pb):
    """Tree depth at which the flow's pairs are matched, over a sample of pairs:
    share of the matched pairs and of the transported mass per depth (0 =
    root, LEVELS + 1 = same point)."""
    from paper_1910_04126_gb300 import api
    flows = api.Flows(tree, Q, D, pa, pb)
    api.flowtree_batch(tree, tree.points, Q, D, pa, pb, flows=flows)
    ex = flows.export()
    dep = np.concatenate([x[3] for x in ex]).astype(np.int64)
    f = np.concatenate([x[2] for x in ex]).astype(np.float64)
    cnt = np.bincount(dep, minlength=LEVELS + 2)
    mass = np.bincount(dep, weights=f, minlength=LEVELS + 2)
    return {"sample_pairs": int(len(pa)), "pairs_per_depth": (cnt / cnt.sum()).round(4).tolist(),
            "mass_per_depth": (mass / mass.sum()).round(4).tolist(),
            "matched_pairs_per_pair": float(cnt.sum()) / len(pa)}


def read_peak_gbs(dev, nbytes: int, passes: int) -> float:
    """Read bandwidth of ft_read_probe over an nbytes buffer (median of 5 timed calls after a warm pass)."""
    import torch
    from paper_1910_04126_gb300 import api
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    api.read_probe(buf, 1, sink)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(5):
        e0.record()
        api.read_probe(buf, passes, sink)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    del buf
    return nbytes * passes / (statistics.median(ts) * 1e-3) / 1e9


def text_flowtree_roofline(tree, Q, D, q_h, db_h, k1, dev, pk, pk_kind):
    """L2 and HBM roofline of the Flowtree launch of the text pipeline (the same k1 candidates per query,
    timed alone).  Algorithmic bytes per pair: two 4d-byte rows per priced (distinct-point) matched pair
    + 8 B per support item + 4 B out, all through L2 (the query's rows are shared by its k1 candidates);
    the HBM view counts the candidate side once: its rows, supports and the output.  The L2 peak is
    ft_read_probe over buffers that fit in L2 (the best of 32, 64 and 96 MiB); the priced pairs per pair
    come from the saved flows of the first 20 queries' candidates."""
    import torch
    from paper_1910_04126_gb300 import api
    nq = Q.n_docs
    cand = api.quadtree_scan(tree, Q, D, k1).reshape(-1)
    pa = torch.arange(nq, dtype=torch.int32, device=dev).repeat_interleave(k1)
    n = int(pa.numel())
    out = torch.empty(n, dtype=torch.float32, device=dev)
    ws = torch.empty(api.flowtree_workspace_size(tree, Q, D, n), dtype=torch.uint8, device=dev)
    api.flowtree_batch(tree, tree.points, Q, D, pa, cand, out=out, workspace=ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(5):
        e0.record()
        api.flowtree_batch(tree, tree.points, Q, D, pa, cand, out=out, workspace=ws)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    del ws, out
    ns = min(nq, 20) * k1
    flows = api.Flows(tree, Q, D, pa[:ns], cand[:ns])
    api.flowtree_batch(tree, tree.points, Q, D, flows.pair_a, flows.pair_b, flows=flows)
    dep = np.concatenate([x[3] for x in flows.export()]).astype(np.int64)
    priced = float((dep <= LEVELS).sum()) / ns
    pa_h, pb_h = pa.cpu().numpy(), cand.cpu().numpy()
    s_q = float(q_h.lengths()[pa_h].mean())
    s_d = float(db_h.lengths()[pb_h].mean())
    row = 4.0 * tree.points.shape[1]
    l2_bytes = priced * 2 * row + 8.0 * (s_q + s_d) + 4.0
    hbm_bytes = s_d * row + 8.0 * s_d + 4.0
    l2_peak = {mb: read_peak_gbs(dev, mb << 20, 50) for mb in (32, 64, 96)}
    peak = max(l2_peak.values())
    l2_gbs = l2_bytes * n / (ms * 1e-3) / 1e9
    hbm_gbs = hbm_bytes * n / (ms * 1e-3) / 1e9
    return {"bound": "l2", "achieved": l2_gbs, "peak": peak, "unit": "GB/s", "frac": l2_gbs / peak,
            "peak_kind": "measured (ft_read_probe, L2-resident buffer)",
            "l2_read_peak_gbs_by_buffer_mib": {str(k): v for k, v in l2_peak.items()},
            "kernel": flow_kernel(tree, Q, D), "kernel_ms": ms, "pairs": n, "pairs_per_s": n / (ms * 1e-3),
            "priced_pairs_per_pair": priced, "support_items_per_pair": s_q + s_d, "bytes_per_pair": l2_bytes,
            "hbm_view": {"bytes_per_pair": hbm_bytes, "achieved": hbm_gbs, "peak": pk["hbm_gbs"],
                         "frac": hbm_gbs / pk["hbm_gbs"], "peak_kind": pk_kind}}


def scan_roofline(tree, Q, D, pk, pk_kind):
    """HBM roofline of the quadtree scan kernel (dense-L1 form: the same kernel
    as the pipeline's, writing int64 L1 instead of select keys): algorithmic
    bytes = 8 per posting visited + 8 per (query, document) output."""
    import torch
    from paper_1910_04126_gb300 import api
    matches = api.quadtree_scan_matches(tree, Q, D)
    out = torch.empty((Q.n_docs, D.n_docs), dtype=torch.int64, device=tree.device)
    lib = api._ffi.load()
    st = torch.cuda.current_stream()
    run = lambda: api.check(lib.ft_quadtree_l1_dense(tree.handle, Q.handle, D.handle, api._ptr(out),
                                                     api._stream(st)), "ft_quadtree_l1_dense")
    run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(5):
        e0.record(st)
        run()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    nbytes = 8.0 * matches + 8.0 * Q.n_docs * D.n_docs
    gbs = nbytes / (ms * 1e-3) / 1e9
    del out
    # the postings are read once from HBM and then served from L2 to every resident query (83% L2 hits in the
    # ncu capture): the bound is the L2 read rate, measured here by ft_read_probe over an L2-resident buffer;
    # HBM is the second view
    l2_peak = max(read_peak_gbs(tree.device, mb << 20, 50) for mb in (32, 64, 96))
    return {"bound": "l2", "achieved": gbs, "peak": l2_peak, "unit": "GB/s", "frac": gbs / l2_peak,
            "peak_kind": "measured (ft_read_probe, L2-resident buffer)",
            "hbm_view": {"peak": pk["hbm_gbs"], "frac": gbs / pk["hbm_gbs"], "peak_kind": pk_kind},
            "kernel": "k_qt_scan", "kernel_ms": ms, "postings_visited": matches,
            "postings_per_pair": matches / (Q.n_docs * D.n_docs), "algorithmic_bytes": nbytes}


def hbm_roofline(q_h, db_h, pairs_per_s, pk, pk_kind):
    # algorithmic bytes per pair at the candidate side: its support
    # (rank, mass, point id: 12 B/item), one LCA byte per merged adjacency,
    # its rows (d = 2 floats), and the 4-byte result
    s_q = float(np.diff(q_h.row_ptr).mean())
    s_d = float(np.diff(db_h.row_ptr).mean())
    per_pair = s_d * 12 + (s_q + s_d) * 1 + s_d * 8 + 4
    achieved = per_pair * pairs_per_s / 1e9
    return {"bytes_per_pair": per_pair, "achieved": achieved, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
            "frac": achieved / pk.get("hbm_gbs", 6800.0), "peak_kind": pk_kind}


if __name__ == "__main__":
    main()
