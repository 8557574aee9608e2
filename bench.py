"""Benchmark: batched Smith-Waterman protein alignment with CIGAR traceback.

Workload (one step = one filtr_align_batch call over the whole batch): 100,000
protein pairs, lengths i.i.d. U[100, 1000], query 30-70% identical to the
reference, seeded 20x20 substitution matrix, affine gaps (open 11, extend 1),
local alignment, score + end coordinates + CIGAR.  Metric: GCUPS (cells whose
recurrence was evaluated / second), inputs resident in HBM.

Also reported on the same JSON line: the same call through the host-buffer
entry point (e2e), the plain one-launch-per-pair form and the whole-GPU
per-pair form (filtr_align_long) on samples, the roofline of the forward
kernels against the measured integer throughput of their cell widths, the CPU
oracle on a bounded sample (its results compared with the GPU's), SM clocks
sampled during the timed region, and under "configs" the same record for the
short-DNA, long-read and megabase-pair workloads.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os

# The serving measurement runs many streams at once: with CUDA's lazy module
# loading, the first launch of each kernel waits for the device's running work
# and stalls every batch in flight on the other streams (a 124 ms banded pair
# held seven small requests up to 72 ms each).  Load every kernel up front.
os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "protein-sw-100k"
WORKLOAD_DESC = {
    "protein-sw-100k": "local affine o=11 e=1, seeded 20x20 matrix, traceback+CIGAR, lengths U[100,1000]",
    "short-dna-1k": "global affine +2/-4 o=4 e=2, score only, 1000 pairs of 128 bp at 5% error",
    "long-reads-10k": "global affine DNA, band 256 (widened) + X-drop 400, traceback+CIGAR, "
                      "10k reads U[10k,50k] at 6/3/1% ins/del/sub",
    "long-pair-1m": "global affine DNA, X-drop 1000, checkpointed traceback, 1 Mbp at 1% + 5 kb insertion",
    "long-reads-10k-zdrop": "the long-read workload with Z-drop 400 (Sec. 9.3) in place of X-drop",
}
METRIC = "GCUPS batched vs plain per-pair launch (bit-exact); serving p50/p99 latency"
# integer operations per cell in the affine local update with traceback, as the
# recurrence states them: E (1 add-max), F (1 add-max), H - (o+e) (1 add),
# diagonal + s (1 add), H (1 three-way max with 0), 4 choice bits (4 compares)
OPS_PER_CELL = 9
CPU_SAMPLE_PAIRS = 5000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="protein-sw-100k",
                    choices=["protein-sw-100k", "short-dna-1k", "long-reads-10k", "long-pair-1m",
                             "long-reads-10k-zdrop"])
    ap.add_argument("--pairs", type=int, default=0, help="0: the workload's own size")
    ap.add_argument("--lmin", type=int, default=0,
                    help="long-read workload: shortest reference (0: 10,000; profiling cases)")
    ap.add_argument("--lmax", type=int, default=0,
                    help="long-read workload: longest reference (0: 50,000; profiling cases)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain per-pair forms (profiling runs)")
    ap.add_argument("--plain-sample", type=int, default=0,
                    help="pairs of the plain per-pair sample (0: the workload's default)")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_PAIRS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # 96 GB: the long-read workload's traceback (10,000 reads x (M + N + 1) rows of
    # 128 bytes, about 77 GB) fits one wave; the protein workload needs about 20 GB
    ap.add_argument("--workspace-gb", type=float, default=96.0)
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-lanes", type=int, default=8, help="concurrent serving lanes")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving measurement and print it")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the sub-records of the other workloads (short DNA, long reads, "
                         "the megabase pair) on the default protein run")
    ap.add_argument("--precision", default="auto", choices=["auto", "i32", "i16x2"],
                    help="cell width of the tiled kernels (results are identical)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan with the built-in shape costs instead of timed ones")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the captured-pipeline (filtr_graph) leg")
    ap.add_argument("--graph-workspace-gb", type=float, default=40.0)
    ap.add_argument("--no-search", action="store_true",
                    help="skip the search-versus-antidiagonal edit-distance table")
    ap.add_argument("--search-only", action="store_true",
                    help="run only the search-versus-antidiagonal table and print it")
    ap.add_argument("--no-fold", action="store_true",
                    help="skip the RNA folding X-drop transfer table")
    ap.add_argument("--fold-only", action="store_true",
                    help="run only the RNA folding table and print it")
    ap.add_argument("--fold-lengths", default=None,
                    help="folding table rows to run, 'length:sequences,...' (default: all four)")
    ap.add_argument("--search-cells", default=None,
                    help="table cells to run, 'length:divergence:pairs,...' (default: all nine)")
    ap.add_argument("--tune-save", default=None,
                    help="write the autotuned shape costs to this JSON file")
    ap.add_argument("--tune-load", default=None,
                    help="install shape costs from this JSON file instead of timing them "
                         "(so a profiled run plans as the unprofiled one did)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.samples)}
        if not self.samples:
            return out
        try:
            sm = [float(s[1]) for s in self.samples]
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(float(s[2]) for s in self.samples)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            seen = set()
            for s in self.samples:
                for k, nm in enumerate(names):
                    if s[5 + k].lower().startswith("active"):
                        seen.add(nm)
            out["reasons"] = sorted(seen)
            out["power_w_max"] = max(float(s[3]) for s in self.samples)
        except Exception:
            pass
        return out


TILED_SOURCES = ("k_strip.cuh", "k_full_impl.cuh", "k_pack_impl.cuh")


def tiled_source_sha():
    """sha256 prefix of the tiled forward kernels' sources, concatenated."""
    import hashlib

    h = hashlib.sha256()
    for name in TILED_SOURCES:
        with open(os.path.join(ROOT, "paper_2607_06225_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per cell of the tiled forward kernels from the committed ncu
    summary, or None when their sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "tiled_forward_protein_sw.md")
    if not os.path.exists(path):
        return None
    cur = tiled_source_sha()
    sha, per_cell = None, None
    for line in open(path):
        if line.startswith("source_sha:"):
            sha = line.split(":")[1].strip()
        if "dram_bytes_per_cell:" in line:
            try:
                per_cell = float(line.split("dram_bytes_per_cell:")[1].split()[0].strip("|"))
            except Exception:
                per_cell = None
    return per_cell if sha == cur else None


SERVE_KINDS = {
    "sw_protein": dict(mode="local", affine=True, gap_open=11, gap_extend=1, traceback=True),
    "band_dna": dict(mode="global", affine=True, gap_open=4, gap_extend=2, band=256, traceback=True),
    "xdrop_dna": dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=400, traceback=True),
}


def reduce_over_ranks(ms: float, cells: float, dist, device) -> tuple:
    """Whole-job timing for N replicas: the step time is the slowest rank's and
    the work is every rank's cells (weak scaling: each rank aligns its own
    batch; no data moves between ranks)."""
    import torch

    if dist is None:
        return ms, cells
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([cells], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


# a fixed request rate, so that latencies compare across builds whose
# capacities (and so whose relative load) differ
SERVE_FIXED_RATE_HZ = 900.0


def serve_bench(F, ctx, seconds: float, load_frac: float, budget_gb: float, lanes: int, seed: int = 4):
    """Serving mix at a fixed offered load: first the burst capacity of the mix
    (every request submitted at once), then Poisson arrivals at `load_frac` of
    that capacity for `seconds`; latency = completion - submission.  A second
    run at SERVE_FIXED_RATE_HZ gives the latencies at one absolute rate."""
    import synth

    srv = F.Server(ctx, int(budget_gb * (1 << 30)), max_inflight=lanes)
    psub = synth.protein_subst(np.random.default_rng(2))
    params = {k: F.make_params(psub if k == "sw_protein" else synth.dna_subst(2, -4), **v)
              for k, v in SERVE_KINDS.items()}

    refused = {"n": 0}

    def run(reqs, paced):
        t0 = time.perf_counter()
        tickets = []
        for rq in reqs:
            if paced:
                delay = rq.t_arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            try:
                tickets.append((rq, srv.submit(params[rq.kind], rq.q, rq.r)))
            except F.FiltrError as ex:  # over a lane's share of the budget: refused
                if ex.code != F._lib.ERR_BUSY:
                    raise
                refused["n"] += 1
        lat, cells, done = [], 0, []
        for rq, t in tickets:
            res, _, times = srv.wait(t)
            lat.append((times[2] - times[0]) * 1e-6)
            cells += int(res["cells"])
            done.append(rq)
        return time.perf_counter() - t0, lat, cells, done

    def pct(x, q):
        return float(np.percentile(np.asarray(x), q)) if len(x) else None

    burst, _ = synth.serve_mix(400, rate_hz=1e9, seed=seed + 100)
    wall, _, cells, done = run(burst, paced=False)
    capacity = cells / wall  # cells per second for this mix
    mean_cells = cells / max(len(done), 1)
    rate = load_frac * capacity / mean_cells
    n = max(50, int(rate * seconds))
    reqs, _ = synth.serve_mix(n, rate_hz=rate, seed=seed)
    refused["n"] = 0
    wall, lat, cells, done = run(reqs, paced=True)
    refused_main = refused["n"]
    fixed_reqs, _ = synth.serve_mix(max(50, int(SERVE_FIXED_RATE_HZ * seconds)), rate_hz=SERVE_FIXED_RATE_HZ,
                                    seed=seed)
    _, flat, _, _ = run(fixed_reqs, paced=True)
    srv.close()
    per_kind = {}
    for kind in SERVE_KINDS:
        lk = [x for x, rq in zip(lat, done) if rq.kind == kind]
        per_kind[kind] = {"requests": len(lk), "p50_ms": pct(lk, 50), "p99_ms": pct(lk, 99)}
    lat = np.array(lat)
    return {"requests": n, "offered_rate_hz": rate, "load_frac_of_capacity": load_frac,
            "offered_gcups": rate * mean_cells / 1e9, "capacity_gcups": capacity / 1e9,
            "achieved_gcups": cells / wall / 1e9, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "per_kind": per_kind,
            "fixed_rate": {"offered_rate_hz": SERVE_FIXED_RATE_HZ, "requests": len(flat),
                           "p50_ms": pct(flat, 50), "p99_ms": pct(flat, 99),
                           "refused": refused["n"] - refused_main},
            "refused": refused_main,
            "refused_note": "requests over a lane's share of the budget (budget / lanes) get "
                            "FILTR_ERR_BUSY at submission and are not in the latencies",
            "mix": "40% SW protein / 40% band-256 NW DNA / 20% X-drop-400 DNA, log-normal lengths "
                   "(median 2000, sigma 1, clipped 100-100000), traceback on",
            "budget_gb": budget_gb, "lanes": lanes}


def trimmed_mean(xs, drop=2):
    """Mean after dropping the `drop` smallest and largest values (the paper's
    protocol: 10 runs, the 2 fastest and 2 slowest dropped)."""
    xs = sorted(xs)
    if len(xs) > 2 * drop:
        xs = xs[drop:len(xs) - drop]
    return sum(xs) / len(xs)


def cpu_baseline(batch, sc, res, cig_t, npairs, time_pairs, runs=10):
    """The oracle on the GPU machine's host cores.  First a parity pass: the oracle
    on the first `npairs` pairs, every field and CIGAR compared with the GPU
    step's results for those pairs.  Then the timing: `runs` runs over the first
    `time_pairs` pairs on all cores, and as many on one core over a sample as
    many times smaller as there are cores; each figure is the trimmed mean
    (runs >= 10: the 2 fastest and 2 slowest dropped)."""
    import oracle

    nth = os.cpu_count() or 1
    n = min(npairs, batch.n)
    sub = batch.subset(np.arange(n))
    t = time.perf_counter()
    ores, oops, ooff = oracle.align_batch(sub, nthreads=nth, **sc)
    dt_parity = time.perf_counter() - t
    tb = bool(sc.get("traceback"))
    fields = ("score", "q_end", "r_end", "status", "cells")
    eq = np.ones(n, dtype=bool)
    for f in fields:
        eq &= res[f][:n].astype(np.int64) == ores[f].astype(np.int64)
    cig_eq = None
    if tb:
        hi = int((res["cigar_off"][:n].astype(np.int64) + res["cigar_len"][:n]).max()) if n else 0
        gc = cig_t[:hi].cpu().numpy().view(np.uint32) if hi else np.zeros(0, np.uint32)
        cig_eq = 0
        for p in range(n):
            o, k = int(res["cigar_off"][p]), int(res["cigar_len"][p])
            a = int(ooff[p])
            ok = (k == int(ores["n_ops"][p]) and np.array_equal(gc[o:o + k], oops[a:a + k])
                  and int(res["q_begin"][p]) == int(ores["q_begin"][p])
                  and int(res["r_begin"][p]) == int(ores["r_begin"][p]))
            eq[p] &= ok
            cig_eq += int(ok)
    parity = {"pairs": n, "equal": int(eq.sum()), "fields": list(fields) + (["cigar", "begin"] if tb else []),
              "cigars_equal": cig_eq, "oracle_s": round(dt_parity, 2)}
    tn = min(time_pairs, batch.n)
    tsub = batch.subset(np.arange(tn))
    times, cells = [], 0
    for _ in range(runs):
        t = time.perf_counter()
        r, _, _ = oracle.align_batch(tsub, nthreads=nth, **sc)
        times.append(time.perf_counter() - t)
        cells = int(r["cells"].sum())
    n1 = max(1, tn // nth)
    s1 = batch.subset(np.arange(n1))
    times1, c1 = [], 0
    for _ in range(runs):
        t = time.perf_counter()
        r1, _, _ = oracle.align_batch(s1, nthreads=1, **sc)
        times1.append(time.perf_counter() - t)
        c1 = int(r1["cells"].sum())
    tm, tm1 = trimmed_mean(times), trimmed_mean(times1)
    proto = f"trimmed mean of {runs} runs (2 fastest and 2 slowest dropped)" if runs >= 10 else \
        f"mean of {runs} run(s)"
    return {"value": cells / tm / 1e9, "unit": "GCUPS", "cores": nth, "nproc": nth, "kind": "oracle",
            "sample": f"first {tn} of the {batch.n} pairs ({cells} cells), {proto}, {tm:.2f} s per run",
            "one_core": {"value": c1 / tm1 / 1e9, "unit": "GCUPS",
                         "sample": f"first {n1} pairs ({c1} cells), {proto}, {tm1:.2f} s per run"},
            "parity": parity}


def run_reference(args):
    import synth

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a bounded sample of the protein workload (--pairs 0 means the workload's own
    # 100,000 pairs, of which the oracle times the first cpu_sample)
    batch = synth.protein_pairs(n=min(args.pairs or 100_000, max(args.cpu_sample, 1)), seed=2)
    sc = dict(batch.scoring)
    times, cells = [], 0
    per_step = max(1, min(args.cpu_sample // max(args.steps + args.warmup, 1), batch.n))
    import oracle

    nth = os.cpu_count() or 1
    for s in range(args.warmup + args.steps):
        lo = (s * per_step) % batch.n
        sub = batch.subset(np.arange(lo, min(lo + per_step, batch.n)))
        t = time.perf_counter()
        res, _, _ = oracle.align_batch(sub, nthreads=nth, **sc)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
            cells += int(res["cells"].sum())
    tot = sum(times)
    v = cells / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / max(len(times), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_step": per_step,
                       "note": "CPU oracle (plain C, int64, all host cores) on a bounded sample of the workload"},
            "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": nth, "kind": "oracle",
                             "sample": f"{per_step} pairs per step of the {WORKLOAD} workload"},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_entry_e2e(F, ctx, params, batch, db, res, cells, steps, tb_on):
    """The same call through the host-buffer entry point (pinned host memory):
    host-to-device copies of the inputs and device-to-host copies of results
    and CIGARs are inside the timed region."""
    import torch

    pin = {}
    for name in ("q_seq", "q_off", "q_len", "r_seq", "r_off", "r_len"):
        a = np.ascontiguousarray(getattr(batch, name))
        pin[name] = torch.from_numpy(a.view(np.uint8)).pin_memory()
    hout = torch.empty(db.n * F.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hcig = torch.empty(max(db.cigar_upper, 1) * 4, dtype=torch.uint8).pin_memory()
    ptr = [pin[n].data_ptr() for n in ("q_seq", "q_off", "q_len", "r_seq", "r_off", "r_len")]
    e2e_t = []
    for k in range(2 + steps):
        t0 = time.perf_counter()
        rc = ctx.align_batch_host_ptr(params, db.n, *ptr, hout.data_ptr(),
                                      hcig.data_ptr() if tb_on else None,
                                      db.cigar_upper if tb_on else 0)
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())
        if k >= 2:
            e2e_t.append(time.perf_counter() - t0)
    hres = hout.numpy().view(F.RESULT_DTYPE)
    assert np.array_equal(hres, res), "host entry point disagrees with the device entry point"
    total_ops = int(hres["cigar_off"][-1] + hres["cigar_len"][-1]) if tb_on else 0
    h2d = sum(int(pin[n].numel()) for n in pin)
    d2h = db.n * F.RESULT_DTYPE.itemsize + total_ops * 4
    return {"value": cells / (sum(e2e_t) / len(e2e_t)) / 1e9, "unit": "GCUPS",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def long_pair_e2e(F, ctx, params, batch, steps, res, stream, dev):
    """The long pair end to end: pinned host codes copied in, filtr_align_long,
    the result and CIGAR copied back."""
    import torch

    q, r = batch.pair(0)
    hq = torch.from_numpy(np.ascontiguousarray(q)).pin_memory()
    hr = torch.from_numpy(np.ascontiguousarray(r)).pin_memory()
    dq = torch.empty_like(hq, device=dev)
    dr = torch.empty_like(hr, device=dev)
    cap = len(q) + len(r) + 1
    dout = torch.empty(F.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    dcig = torch.empty(cap, dtype=torch.int32, device=dev)
    hout = torch.empty(F.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hcig = torch.empty(cap, dtype=torch.int32).pin_memory()
    times = []
    for k in range(1 + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dq.copy_(hq, non_blocking=True)
        dr.copy_(hr, non_blocking=True)
        rc = ctx.align_long_ptr(params, dq.data_ptr(), len(q), dr.data_ptr(), len(r),
                                dout.data_ptr(), dcig.data_ptr(), cap, stream=stream.cuda_stream)
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())
        hout.copy_(dout, non_blocking=True)
        n_ops = int(res[0]["cigar_len"])
        hcig[:n_ops].copy_(dcig[:n_ops], non_blocking=True)
        torch.cuda.synchronize()
        if k >= 1:
            times.append(time.perf_counter() - t0)
    got = hout.numpy().view(F.RESULT_DTYPE)
    assert np.array_equal(got, res), "end-to-end long pair disagrees"
    cells = int(res[0]["cells"])
    return {"value": cells / (sum(times) / len(times)) / 1e9, "unit": "GCUPS",
            "h2d_bytes_per_step": len(q) + len(r),
            "d2h_bytes_per_step": F.RESULT_DTYPE.itemsize + 4 * int(res[0]["cigar_len"])}


def plain_per_pair(F, ctx, params, batch, nsample, stream, dev, tb_on):
    """The plain form: one kernel launch per pair, on a sample of the same pairs,
    timed beside the batched call on that sample; results must agree."""
    import torch

    ns = min(nsample, batch.n)
    sub = batch.subset(np.arange(ns))
    sdb = F.DeviceBatch(sub, dev)
    sout, scig = F.alloc_outputs(sdb.n, sdb.cigar_upper, dev)

    def timed(plain):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = ctx.align_batch_ptr(params, sdb.n, *sdb.ptrs(), sout.data_ptr(),
                                 scig.data_ptr() if tb_on else None,
                                 sdb.cigar_upper if tb_on else 0, stream=stream.cuda_stream,
                                 plain=plain)
        b.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())
        return a.elapsed_time(b), F.results_to_numpy(sout, sdb.n)

    timed(False)
    tb_ms, rb = timed(False)
    tp_ms, rp = timed(True)
    assert np.array_equal(rb, rp), "plain and batched results differ"
    scells = int(rb["cells"].sum())
    return {"pairs": ns, "gcups_plain": scells / (tp_ms * 1e-3) / 1e9,
            "gcups_batched_same_pairs": scells / (tb_ms * 1e-3) / 1e9,
            "ms_plain": tp_ms, "ms_batched": tb_ms}


def graph_bench(F, ctx, params, batch, db, res_ref, cells, steps, warmup, stream, flush, dev,
                tb_on, ws_gb):
    """The same workload through the captured pipeline (filtr_graph_launch: one
    CUDA graph per step, no host synchronisation inside the step)."""
    import torch

    max_len = int(max(batch.q_len.max(), batch.r_len.max()))
    g = F.Graph(ctx, params, db.n, max_len, int(ws_gb * (1 << 30)))
    out_t, cig_t = F.alloc_outputs(db.n, db.cigar_upper, dev)

    def gstep():
        rc = g.launch_ptr(db.n, *db.ptrs(), out_t.data_ptr(), cig_t.data_ptr() if tb_on else None,
                          db.cigar_upper if tb_on else 0, stream=stream.cuda_stream)
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())

    try:
        for _ in range(max(warmup, 1)):
            gstep()
        torch.cuda.synchronize()
        status = g.status()
        res = F.results_to_numpy(out_t, db.n)
        assert status == 0 and np.array_equal(res, res_ref), "graph results differ"
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_((k + 7) & 0xFF)
            ev[k][0].record(stream)
            gstep()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        return {"value": cells / (ms * 1e-3) / 1e9, "unit": "GCUPS", "ms_per_step": ms,
                "call": "filtr_graph_launch (captured pipeline, no host synchronisation)",
                "status": status}
    finally:
        g.close()


# Sec. 9.4's comparison of the search traversal with the antidiagonal one for
# edit distance: (length, pairs per batch) and divergences; the paper's CPU
# speedups (search over antidiagonal, its Table) for context.
SEARCH_TABLE = ((500, 32768), (2000, 16384), (4000, 8192))
SEARCH_DIVS = (0.01, 0.05, 0.30)
PAPER_SEARCH_SPEEDUP = {(500, 0.01): 97, (2000, 0.01): 98, (4000, 0.01): 300,
                        (500, 0.05): 27, (2000, 0.05): 14, (4000, 0.05): 23,
                        (500, 0.30): 0.45, (2000, 0.30): 0.45, (4000, 0.30): 0.72}


def search_cells(spec):
    """The table's (length, divergence, pairs) cells, or those `spec` names."""
    if not spec:
        return [(length, div, n) for length, n in SEARCH_TABLE for div in SEARCH_DIVS]
    out = []
    for item in spec.split(","):
        length, div, n = item.split(":")
        out.append((int(length), float(div), int(n)))
    return out


def search_table(F, ctx, steps, warmup, stream, flush, dev, cpu=True, cells=None):
    """Edit distance of one batch per (length, divergence) through the search
    traversal (filtr_search_batch, score only) and through the antidiagonal
    kernels (filtr_align_batch with unit costs, whose score is minus the edit
    distance): CUDA events on the stream, L2 flushed between steps, distances
    checked equal.  With cpu, the oracle's search on a few pairs (one thread)."""
    import torch

    import synth

    def timed(fn):
        for _ in range(max(warmup, 1)):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_((k + 3) & 0xFF)
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sorted(a.elapsed_time(b) for a, b in ev)[steps // 2]

    sp = F.make_search_params(traceback=False, alphabet=4)
    tuned = False
    rows = []
    for length, div, n in search_cells(cells):
        b = synth.edit_pairs(n, length, div, seed=6)
        db = F.DeviceBatch(b, dev)
        out_s, _ = F.alloc_outputs(db.n, 0, dev)
        out_a, _ = F.alloc_outputs(db.n, 0, dev)
        ap = F.make_params(b.subst, **b.scoring)
        if not tuned:  # setup, untimed: the antidiagonal kernels' shape costs
            ctx.autotune(ap)
            tuned = True

        def sr():
            rc = ctx.search_batch_ptr(sp, db.n, *db.ptrs(), out_s.data_ptr(), None, 0,
                                      stream=stream.cuda_stream)
            if rc != 0:
                raise F.FiltrError(rc, F.last_error())

        def ad():
            rc = ctx.align_batch_ptr(ap, db.n, *db.ptrs(), out_a.data_ptr(), None, 0,
                                     stream=stream.cuda_stream)
            if rc != 0:
                raise F.FiltrError(rc, F.last_error())

        t_sr, t_ad = timed(sr), timed(ad)
        rs, ra = F.results_to_numpy(out_s, db.n), F.results_to_numpy(out_a, db.n)
        assert np.array_equal(rs["score"], ra["score"]), "search and antidiagonal disagree"
        full = float((b.q_len.astype(np.float64) * b.r_len).sum())
        row = {"length": length, "divergence": div, "pairs": n,
               "search_ms": t_sr, "antidiagonal_ms": t_ad, "speedup": t_ad / t_sr,
               "paper_cpu_speedup": PAPER_SEARCH_SPEEDUP.get((length, div)),
               "search_pairs_per_s": n / (t_sr * 1e-3),
               "search_gcups_equiv": full / (t_sr * 1e-3) / 1e9,
               "antidiagonal_gcups": full / (t_ad * 1e-3) / 1e9,
               "mean_distance": float(-rs["score"].mean()),
               "wavefront_cells_per_pair": float(rs["cells"].mean())}
        if cpu:
            import oracle

            sub = synth.pack([b.pair(p)[0] for p in range(4)], [b.pair(p)[1] for p in range(4)],
                             4, b.subst)
            t0 = time.perf_counter()
            ores, _, _ = oracle.search_batch(sub, nthreads=1, traceback=False)
            row["oracle_ms_per_pair_1core"] = (time.perf_counter() - t0) * 1e3 / 4
            assert np.array_equal(-ores["distance"], rs["score"][:4])
        rows.append(row)
        del db, out_s, out_a
    return {"call": "filtr_search_batch (score only) vs filtr_align_batch (unit-cost global, "
                    "score only), same pairs",
            "l2": "flushed between timed steps", "steps": steps, "rows": rows}


# Sec. 9.5's transfer of X-drop to Nussinov folding: RNA lengths (its four
# classes span 76-500 bases), sequences per batch, thresholds.
FOLD_LENGTHS = ((76, 2048), (120, 2048), (300, 1024), (500, 1024))
FOLD_XS = (2, 8, 32)


def fold_table(F, ctx, steps, warmup, stream, flush, dev, cpu=True, lengths=None):
    """Fold one batch of structured synthetic RNAs per length unpruned and
    under X-drop (15-span warm-up): CUDA events on the stream, L2 flushed
    between steps; cells evaluated and agreement with the unpruned fold (pair
    count ratio and base-pair F1).  With cpu, the oracle on two sequences of
    each length (one core)."""
    import torch

    import synth

    def pairs_of(part, off, lens):
        out = []
        for p in range(len(lens)):
            a, n = int(off[p]), int(lens[p])
            pp = part[a:a + n]
            i = np.nonzero(pp > np.arange(n))[0]
            out.append(set(zip(i.tolist(), pp[i].tolist())))
        return out

    rows = []
    todo = FOLD_LENGTHS if not lengths else [tuple(int(v) for v in item.split(":"))
                                             for item in lengths.split(",")]
    for length, n in todo:
        seq, off, lens = synth.rna_structured(n, length, seed=7)
        seq_t = torch.from_numpy(seq).to(dev)
        off_t = torch.from_numpy(off.view(np.int64)).to(dev)
        len_t = torch.from_numpy(lens.view(np.int32)).to(dev)
        out_t = torch.empty(n * F.FOLD_RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        part_t = torch.empty(len(seq), dtype=torch.int32, device=dev)
        row = {"length": length, "sequences": n}
        ref = None
        for X in (None,) + FOLD_XS:
            prm = F.make_fold_params(min_loop=3, xdrop=X, warmup=15, traceback=True)

            def run():
                rc = ctx.fold_batch_ptr(prm, n, seq_t.data_ptr(), off_t.data_ptr(),
                                        len_t.data_ptr(), out_t.data_ptr(), part_t.data_ptr(),
                                        stream=stream.cuda_stream)
                if rc != 0:
                    raise F.FiltrError(rc, F.last_error())

            for _ in range(max(warmup, 1)):
                run()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for k in range(steps):
                flush.fill_((k + 5) & 0xFF)
                ev[k][0].record(stream)
                run()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)[steps // 2]
            res = out_t.cpu().numpy().view(F.FOLD_RESULT_DTYPE).copy()
            pairs = pairs_of(part_t.cpu().numpy(), off, lens)
            key = "unpruned" if X is None else f"x{X}"
            entry = {"ms": ms, "sequences_per_s": n / (ms * 1e-3),
                     "cells": int(res["cells"].sum()), "mean_pairs": float(res["score"].mean()),
                     "dropped": int((res["status"] != 0).sum())}
            if ref is None:
                ref = (res, pairs)
            else:
                f1 = []
                for a, b in zip(ref[1], pairs):
                    tp = len(a & b)
                    f1.append(1.0 if not a and not b else 2 * tp / max(len(a) + len(b), 1))
                entry.update(speedup=row["unpruned"]["ms"] / ms,
                             cells_fraction=entry["cells"] / row["unpruned"]["cells"],
                             pair_ratio=float(res["score"].sum() / max(ref[0]["score"].sum(), 1)),
                             pair_f1=float(np.mean(f1)))
            row[key] = entry
        if cpu:
            import oracle

            t0 = time.perf_counter()
            ores, _ = oracle.fold_batch(seq[: 2 * length], off[:2], lens[:2], nthreads=1,
                                        min_loop=3)
            row["oracle_ms_per_sequence_1core"] = (time.perf_counter() - t0) * 1e3 / 2
            assert np.array_equal(ores["score"], ref[0]["score"][:2].astype(np.int64))
        rows.append(row)
    return {"call": "filtr_fold_batch, traceback on, min_loop 3, warm-up 15 spans",
            "l2": "flushed between timed steps", "steps": steps, "rows": rows}


def workload_batch(synth, wl, pairs, seed_off, lmin=0, lmax=0):
    if wl == "protein-sw-100k":
        return synth.protein_pairs(n=pairs or 100_000, seed=2 + seed_off)
    if wl == "short-dna-1k":
        return synth.short_dna_pairs(n=pairs or 1000, seed=1 + seed_off)
    if wl in ("long-reads-10k", "long-reads-10k-zdrop"):
        return synth.long_reads(n=pairs or 10_000, lmin=lmin or 10_000, lmax=lmax or 50_000,
                                seed=3 + seed_off)
    return synth.long_pair(seed=5 + seed_off)


# per workload: pairs of the plain one-launch-per-pair sample, of the
# whole-GPU-per-pair (filtr_align_long) sample, and of the oracle's parity /
# timing samples (pairs, pairs timed, runs)
PLAIN_SAMPLE = {"protein-sw-100k": 3000, "short-dna-1k": 1000, "long-reads-10k": 20,
                "long-reads-10k-zdrop": 20}
LONG_SAMPLE = {"protein-sw-100k": 300, "short-dna-1k": 300, "long-reads-10k": 4,
               "long-reads-10k-zdrop": 4}
CPU_SAMPLE = {"protein-sw-100k": (5000, 1000, 10), "short-dna-1k": (1000, 1000, 10),
              "long-reads-10k": (160, 160, 1), "long-reads-10k-zdrop": (64, 64, 1)}


def roofline_of(wl, cells, cells_packed, fwd_ms, probe, traffic_per_cell):
    """ALU roofline of the forward kernels.  Work = cells x 9 integer operations
    (an add and a max count as two).  Peak: the time the cells would take at
    the measured rate of their cell width -- int32 cells at the two-pipe
    add/max rate, int16x2 cells at the packed DPX add-max rate (two cells per
    lane instruction, two operations each) -- so the fraction follows the mix."""
    i32 = probe["int_ops"] if probe else None
    pk = 2.0 * probe["viaddmax_s16x2_lanes"] if probe else None
    achieved = cells * OPS_PER_CELL / (fwd_ms * 1e-3) / 1e12
    peak = None
    if i32:
        t_min = (cells - cells_packed) * OPS_PER_CELL / i32 + cells_packed * OPS_PER_CELL / pk
        peak = cells * OPS_PER_CELL / t_min / 1e12 if t_min > 0 else None
    xd = wl in ("long-reads-10k", "long-pair-1m", "long-reads-10k-zdrop")
    kern = "k_xdrop (antidiagonal sweep)" if xd else "k_full + k_pack (tiled forward, all waves)"
    return {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": (achieved / peak) if peak else None, "ops_per_cell": OPS_PER_CELL,
            "cells": {"i32": cells - cells_packed, "i16x2": cells_packed},
            "peak_per_width": {"i32": i32 / 1e12 if i32 else None,
                               "i16x2": pk / 1e12 if pk else None},
            "forward_ms": fwd_ms, "forward_gcups": cells / (fwd_ms * 1e-3) / 1e9,
            "traffic": (traffic_per_cell * cells) if traffic_per_cell else None,
            "traffic_unit": "DRAM bytes per step (ncu dram__bytes_read+write per cell x cells)",
            "algorithmic_bytes": 0.5 * cells,
            "peak_source": "filtr_probe_int_peak: int32 add+max two-pipe rate; "
                           "__viaddmax_s16x2 lane rate x 2 ops (measured on this GPU, 'of measured')",
            "probe": probe}


def plain_long_per_pair(F, ctx, params, batch, nsample, stream, dev, res):
    """The whole-GPU-per-pair form: one filtr_align_long call (the intra-pair
    kernel across every SM) per pair, on a sample; results must equal the
    batched call's."""
    import torch

    ns = min(nsample, batch.n)
    tot_ms, cells = 0.0, 0
    cap = int(max(batch.q_len[:ns].max() + batch.r_len[:ns].max(), 1)) + 1
    dout = torch.empty(F.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    dcig = torch.empty(cap, dtype=torch.int32, device=dev)
    for p in range(ns):
        q, r = batch.pair(p)
        dq = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
        dr = torch.from_numpy(np.ascontiguousarray(r)).to(dev)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = ctx.align_long_ptr(params, dq.data_ptr(), len(q), dr.data_ptr(), len(r), dout.data_ptr(),
                                dcig.data_ptr(), cap, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())
        got = F.results_to_numpy(dout, 1)[0]
        for f in ("score", "q_end", "r_end", "status", "cells"):
            assert int(got[f]) == int(res[p][f]), "filtr_align_long and the batched call differ"
        tot_ms += a.elapsed_time(b)
        cells += int(got["cells"])
    return {"pairs": ns, "gcups": cells / (tot_ms * 1e-3) / 1e9, "ms_total": tot_ms,
            "call": "filtr_align_long per pair (intra-pair kernel on every SM)"}


def measure_workload(F, ctx, synth, wl, args, steps, warmup, stream, flush, dev, rank, world, dist,
                     probe):
    """One workload: untimed setup and warm-up, `steps` timed steps (CUDA events,
    L2 flushed between steps, clocks sampled), then on rank 0 the end-to-end
    call through the host-buffer entry point, the plain forms and the roofline.
    Returns (record, batch, scoring, results, cigar tensor)."""
    import torch

    seed_off = 1000 * rank
    own = wl == args.workload
    batch = workload_batch(synth, wl, args.pairs if own else 0, seed_off,
                           args.lmin if own else 0, args.lmax if own else 0)
    sc = dict(batch.scoring)
    if wl == "long-reads-10k-zdrop":
        sc.update(xdrop=None, zdrop=400)
    prec = {"auto": F.PREC_AUTO, "i32": F.PREC_I32, "i16x2": F.PREC_I16X2}[args.precision]
    params = F.make_params(batch.subst, **dict(sc, precision=prec))
    db = F.DeviceBatch(batch, dev)
    out_t, cig_t = F.alloc_outputs(db.n, db.cigar_upper, dev)
    is_long = wl == "long-pair-1m"
    tb_on = bool(sc.get("traceback"))

    def step():
        if is_long:
            rc = ctx.align_long_ptr(params, db.q_seq.data_ptr(), int(batch.q_len[0]),
                                    db.r_seq.data_ptr(), int(batch.r_len[0]), out_t.data_ptr(),
                                    cig_t.data_ptr(), db.cigar_upper, stream=stream.cuda_stream)
        else:
            rc = ctx.align_batch_ptr(params, db.n, *db.ptrs(), out_t.data_ptr(),
                                     cig_t.data_ptr() if tb_on else None,
                                     db.cigar_upper if tb_on else 0, stream=stream.cuda_stream)
        if rc != 0:
            raise F.FiltrError(rc, F.last_error())

    tune = None
    if not args.no_autotune:
        # one-time setup, outside every timed region
        if args.tune_load and wl == args.workload:
            with open(args.tune_load) as f:
                tune = json.load(f)
            ctx.tune_apply(params, tune)
        else:
            tune = ctx.autotune(params)
            if args.tune_save and wl == args.workload:
                with open(args.tune_save, "w") as f:
                    json.dump(tune, f)
    ctx.set_timing(True)
    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    res = F.results_to_numpy(out_t, db.n)
    cells = int(res["cells"].sum())
    if wl in ("protein-sw-100k", "short-dna-1k"):
        assert cells == batch.cells_full()

    sampler = ClockSampler(dev.index or 0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    fwd_ms, walk_ms, launches, other_ms = [], [], [], {}
    packed = cells_packed = 0
    xd16 = (0, 0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.fill_(k & 0xFF)  # evict L2 between timed steps (outside the events)
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select these launches
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        torch.cuda.nvtx.range_pop()
        st = ctx.last_stats()  # waits for the step; device-side phase times
        fwd_ms.append(st["ms_forward"])
        walk_ms.append(st["ms_walk"])
        for key in ("ms_validate", "ms_place", "ms_total", "ms_host_wait", "ms_host_plan"):
            other_ms.setdefault(key[3:], []).append(st[key])
        launches.append(st["launches"])
        packed = st.get("pairs_i16x2", 0)
        cells_packed = st.get("cells_i16x2", 0)
        xd16 = (st.get("pairs_xd16", 0), st.get("pairs_xd16_rerun", 0))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms, total_cells = reduce_over_ranks(ms, float(cells), dist, dev)
    value = total_cells / (ms * 1e-3) / 1e9
    rec = None
    if rank == 0:
        plain = plain_long = None
        if is_long:
            e2e = long_pair_e2e(F, ctx, params, batch, steps, res, stream, dev)
        else:
            e2e = host_entry_e2e(F, ctx, params, batch, db, res, cells, steps, tb_on)
            if not args.no_plain:
                ns = args.plain_sample if wl == args.workload and args.plain_sample else PLAIN_SAMPLE[wl]
                plain = plain_per_pair(F, ctx, params, batch, ns, stream, dev, tb_on)
                plain_long = plain_long_per_pair(F, ctx, params, batch, LONG_SAMPLE[wl], stream, dev,
                                                 res)
        fwd = statistics.median(fwd_ms)
        # the committed capture covers the tiled kernels on the protein workload only
        traffic_per_cell = ncu_traffic() if wl == "protein-sw-100k" else None
        # the antidiagonal sweep's cells count as packed when every pair ran in
        # the int16x2 sweep (pairs rerun in int32 are counted as int32 cells)
        if xd16[0] and not cells_packed:
            cells_packed = int(cells * max(xd16[0] - xd16[1], 0) / max(batch.n, 1))
        roof = roofline_of(wl, cells, cells_packed, fwd, probe, traffic_per_cell)
        rec = {
            "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32|i16x2 (exact integer)" if cells_packed else "i32 (exact integer)",
            "data": "synthetic",
            "config": {"workload": wl, "pairs": batch.n, "cells_per_step": cells,
                       "mode": WORKLOAD_DESC[wl],
                       "precision": args.precision, "pairs_i16x2": packed,
                       "pairs_sweep_i16x2": xd16[0], "pairs_sweep_rerun_i32": xd16[1],
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"replica x{world}"},
            "plain_per_pair": plain,
            "plain_long_per_pair": plain_long,
            "step_ms": step_ms,
            "phases_ms": {"forward": fwd, "walk": statistics.median(walk_ms), "step": ms,
                          **{k: statistics.median(v) for k, v in other_ms.items()}},
            "autotune_ns_per_warp_step": tune,
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": int(statistics.median(launches)),
            "clocks": clocks,
            "wall_s_timed": wall,
        }
    return rec, batch, sc, res, cig_t, params, db, (out_t, cig_t)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2607_06225_gb300 as F
    import synth
    from paper_2607_06225_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if not os.path.exists(F._lib.LIB_PATH):
        B.build()
    ctx = F.Context(local_rank, int(args.workspace_gb * (1 << 30)))
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    if args.fold_only:
        if rank == 0:
            tab = fold_table(F, ctx, args.steps, args.warmup, stream, flush, dev,
                             cpu=not args.no_cpu_baseline, lengths=args.fold_lengths)
            print(json.dumps({"fold_table": tab}), flush=True)
        ctx.close()
        return
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": serve_bench(F, ctx, args.serve_seconds, args.serve_load, 40.0,
                                                     args.serve_lanes)}), flush=True)
        ctx.close()
        return
    if args.search_only:
        if rank == 0:
            tab = search_table(F, ctx, args.steps, args.warmup, stream, flush, dev,
                               cpu=not args.no_cpu_baseline, cells=args.search_cells)
            print(json.dumps({"search_table": tab}), flush=True)
        ctx.close()
        return
    # weak scaling: every rank aligns its own batch (independent problems)
    wl = args.workload
    probe = ctx.probe() if rank == 0 else None
    line, batch, sc, res, cig_t, params, db, outs = measure_workload(
        F, ctx, synth, wl, args, args.steps, args.warmup, stream, flush, dev, rank, world, dist, probe)
    tb_on = bool(sc.get("traceback"))
    if rank == 0:
        cells = int(res["cells"].sum())
        if wl in ("protein-sw-100k", "short-dna-1k") and not args.no_graph:
            line["graph"] = graph_bench(F, ctx, params, batch, db, res, cells, args.steps,
                                        args.warmup, stream, flush, dev, tb_on,
                                        args.graph_workspace_gb)
        if not args.no_search and wl == "protein-sw-100k":
            line["search"] = search_table(F, ctx, 3, 1, stream, flush, dev,
                                          cpu=not args.no_cpu_baseline)
        if not args.no_fold and wl == "protein-sw-100k":
            line["fold"] = fold_table(F, ctx, 3, 1, stream, flush, dev,
                                      cpu=not args.no_cpu_baseline)
        if not args.no_serve and wl == "protein-sw-100k":
            line["serving"] = serve_bench(F, ctx, args.serve_seconds, args.serve_load, 40.0,
                                          args.serve_lanes)
        if not args.no_cpu_baseline and wl != "long-pair-1m":
            npairs, tpairs, runs = CPU_SAMPLE[wl]
            if args.cpu_sample != CPU_SAMPLE_PAIRS:
                npairs = tpairs = args.cpu_sample
            line["cpu_baseline"] = cpu_baseline(batch, sc, res, cig_t, npairs, tpairs, runs)
    del db, outs, cig_t
    torch.cuda.empty_cache()
    # the other configurations, each timed the same way (a sub-record each)
    if args.configs and wl == "protein-sw-100k":
        subs = {}
        for other in ("short-dna-1k", "long-reads-10k", "long-pair-1m"):
            # enough steps for the clock sampler (200 ms period) to see the short workload
            k_steps = {"long-pair-1m": 2, "long-reads-10k": 3, "short-dna-1k": 2000}[other]
            rec, ob, osc, ores, ocig, _, odb, oouts = measure_workload(
                F, ctx, synth, other, args, k_steps, 3, stream, flush, dev, rank, world, dist, probe)
            if rank == 0:
                if not args.no_cpu_baseline and other != "long-pair-1m":
                    npairs, tpairs, runs = CPU_SAMPLE[other]
                    rec["cpu_baseline"] = cpu_baseline(ob, osc, ores, ocig, npairs, tpairs, runs)
                elif other == "long-pair-1m":
                    rec["cpu_baseline"] = {
                        "value": None, "kind": "oracle",
                        "note": "not timed here: the oracle keeps every evaluated cell (848 M cells, "
                                "about 35 GB) and takes about 40 s; its result is stored in "
                                "tests/golden/long_pair_1mbp.json and the GPU test compares against it"}
                subs[other] = rec
            del odb, oouts, ocig
            torch.cuda.empty_cache()
        if rank == 0:
            line["configs"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()
