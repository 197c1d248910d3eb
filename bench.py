"""Throughput benchmark of the JABBA symbolization path on GB300.

Metric: series points symbolized per second (Gpts/s) through the whole
forward path (domains, Eq. 1 compression, normalisation, per-domain greedy
aggregation, global merge, label propagation), with the input resident in HBM
(`value`), and end to end through the same C-ABI calls with the input copied
from pinned host memory and the symbols + dictionary read back inside the
timed region (`e2e`).  Workload: the scale-stress collection (100,000 series,
log-uniform lengths in [100, 100,000], ~1.44e9 points, 11.5 GB of float64 --
far larger than L2, so no flush is needed between steps).

Forms timed: "batched" = the whole step captured once in a CUDA graph and
replayed (persistent work-stealing kernels, autotuned launch configuration);
"plain" = the unbatched form, one compression launch and one Stage I launch
per domain issued eagerly, timed on a bounded sample of the same workload
(the first --plain-series series) next to the batched form on that sample.  The CPU oracle is timed on a bounded sample of the same
workload on the host cores (`cpu_baseline`); `--impl reference` times only
that oracle, as the reference arm.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the
workload (the path is timed per GPU; replicas only), the max time over ranks
is taken and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "series points symbolized/sec (Gpts/s) and % of HBM roofline, batched vs plain, 1 GB300"
WORKLOAD_DESC = {
    "scale": "scale stress: 100,000 series, lengths log-uniform [100, 100,000], walk/sinusoid+AR(1)/level-shift "
             "generators, z-normalised, FIXED_LEN 4,096-interval domains, tol=0.1 alpha=0.1 scl=1",
    "uneven": "uneven batch: 10,000 series, lengths U[500, 50,000], walk + level shifts, FIXED_LEN 1,000, "
              "tol=alpha=0.05",
    "multivar": "multivariate: 64 channels x 2^20, 3 sinusoids + AR(1), 1,024 equal domains per channel, "
                "tol=0.1 alpha=0.2",
    "diff": "1,024 x 10,000 walk + sinusoid, 4 equal domains, tol=alpha=0.1",
    "small": "16 x 2,000 walk + sinusoid, 4 equal domains, tol=alpha=0.1",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle (CPU) timing
def oracle_step(x, off, cfg, threads):
    import oracle
    t0 = time.perf_counter()
    oracle.pipeline(x, off, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"], cfg["domain_value"],
                    threads=threads, with_reconstruct=False)
    return time.perf_counter() - t0


def cpu_sample(workload, sample_series):
    import synth
    x, off, cfg = synth.make(workload, max_series=sample_series)
    return x, off, cfg


def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle (the paper's multicore design:
    parallel compression over domains, serial digitization) on a bounded
    sample of the same workload per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    x, off, cfg = cpu_sample(args.workload, args.cpu_series)
    for _ in range(args.warmup):
        oracle_step(x, off, cfg, threads)
    t = 0.0
    for _ in range(args.steps):
        t += oracle_step(x, off, cfg, threads)
    n = len(x)
    value = n * args.steps / t / 1e9
    sample = f"first {args.cpu_series} series of the workload ({n} points) per step"
    line = dict(metric=METRIC, value=value, unit="Gpts/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * t / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD_DESC[args.workload], sample=sample),
                cpu_baseline=dict(value=value, unit="Gpts/s", cores=threads, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="Gpts/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def roofline_table(workload, n, N, G, D, comp_ms, loc_ms, rnd_ms, rounds_name, peak, peak_kind):
    """Roofline entries of the three largest stages (lists of per-step
    milliseconds in) and the dominant one (largest time) as the `roofline`
    object.  Algorithmic bytes per launch, per unit processed:
      k_compress: 8 B per point read + 12 B per piece written (len, end value);
      local aggregation (tile kernels + routing + group offsets): 12 B per
        piece read (len, inc) + 4 B per piece written (label) + 48 B per group
        record + 12 B per domain (group count and offset);
      merge rounds (k_mrounds1, or k_mrounds in the two-barrier form): 12.125 B
        per local group (its FP32 centre and key-order position, 12 B, and its
        coverage bit, each read once).
    DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) is known for
    the scale workload from ncu captures of its first 10,000 series
    (143,804,766 points, 17,479,524 pieces): k_compress 1,184.6 MB read and
    212.7 MB written, scaled to a launch by its points; the five Stage I tile
    launches of a step 222.6 MB read and 60.7 MB written, scaled by the
    pieces (both stream their inputs once, so the traffic grows with them).
    The rounds kernel's traffic is not scaled (the sample's working set fits
    in L2, the full one does not): null there and for other workloads."""
    scale = workload == "scale"
    comp_traffic = 1397.301728e6 / 143804766 * n if scale else None
    local_traffic = 283.246592e6 / 17479524 * N if scale else None
    cand = [("k_compress", comp_ms, 8.0 * n + 12.0 * N, comp_traffic),
            ("local aggregation (k_local_tile x5, k_local_classify, k_local_warp, scan)", loc_ms,
             16.0 * N + 48.0 * G + 12.0 * D, local_traffic),
            (rounds_name, rnd_ms, 12.125 * G, None)]
    by_kernel = []
    for name, ms_list, alg, traffic in cand:
        t = float(np.mean(ms_list))
        ach = alg / (t * 1e-3) / 1e9
        by_kernel.append(dict(kernel=name, ms_per_launch=t, algorithmic_bytes_per_launch=alg, achieved=ach,
                              frac=ach / peak, traffic=traffic))
    dom = max(by_kernel, key=lambda r: r["ms_per_launch"])
    return dict(bound="hbm", achieved=dom["achieved"], peak=peak, unit="GB/s", frac=dom["frac"],
                traffic=dom["traffic"], kernel=dom["kernel"], peak_source=peak_kind,
                algorithmic_bytes_per_launch=dom["algorithmic_bytes_per_launch"],
                ms_per_launch=dom["ms_per_launch"], by_kernel=by_kernel)


def run_ours(args, ws, rank, local):
    import torch

    import paper_2401_00109_gb300 as jb
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    S, n = synth.sizes(args.workload, args.max_series)
    # pinned host input (the e2e leg copies it every step)
    x_host = torch.empty(n, dtype=torch.float64, pin_memory=True)
    t_gen = time.perf_counter()
    _, off_np, cfg = synth.make(args.workload, max_series=args.max_series, out=x_host.numpy())
    t_gen = time.perf_counter() - t_gen
    off_host = torch.from_numpy(off_np).pin_memory()
    p = jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                  domain_value=cfg["domain_value"])
    ctx = jb.Context(local)
    # size the group table from one sizing pass (capacity = 1.25 x observed)
    pl = jb.Pipeline(ctx, off_np, n, p, group_capacity=max(1 << 16, n // 16))
    pl.x.copy_(x_host, non_blocking=True)
    pl.enqueue()
    try:
        ctx.sync_status(where="sizing step")
        need = int(pl.b["n_groups"][0].item())
    except jb.JabbaError as e:
        if e.code != jb.ERR_CAPACITY:
            raise
        need = int(pl.b["n_groups"][0].item())
    gcap = int(need * 1.25) + 1024
    if gcap > pl.gcap or gcap < pl.gcap // 4:
        del pl
        torch.cuda.empty_cache()
        pl = jb.Pipeline(ctx, off_np, n, p, group_capacity=gcap)
        pl.x.copy_(x_host, non_blocking=True)
    st = torch.cuda.current_stream()

    # ---- autotuned launch configuration (native autotuner: each stage times
    # its candidate configurations on this collection)
    tuning = pl.tune() if not args.no_tune else ctx.tuning()

    # ---- batched: graph capture of the whole step; one graph per timed step
    # so each keeps its own event pair around the compression kernel
    pl.enqueue()
    ctx.sync_status(where="eager step")
    graphs = []
    for i in range(args.warmup + args.steps):
        ctx.profile_slot(i if i < 256 else -1)
        graphs.append(pl.capture())
    ctx.profile_slot(-1)
    kernels_per_step = jb.graph_kernel_nodes(pl.capture(keep_graph=True))
    for i in range(args.warmup):
        graphs[i].replay()
    torch.cuda.synchronize()
    ctx.sync_status(where="warm-up")
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(args.steps):
        graphs[args.warmup + i].replay()
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ctx.sync_status(where="timed steps")
    ms_all = max_over_ranks(ms, ws)
    comp_ms = [ctx.profile_elapsed(args.warmup + i, 0) for i in range(args.steps)]
    fin_ms = [ctx.profile_elapsed(args.warmup + i, 1) for i in range(args.steps)]
    loc_ms = [ctx.profile_elapsed(args.warmup + i, 2) for i in range(args.steps)]
    mrg_ms = [ctx.profile_elapsed(args.warmup + i, 3) for i in range(args.steps)]
    sym_ms = [ctx.profile_elapsed(args.warmup + i, 4) for i in range(args.steps)]
    rnd_ms = [ctx.profile_elapsed(args.warmup + i, 5) for i in range(args.steps)]
    res = pl.results()
    diag = ctx.diagnostics()
    N, G, k = res["n_pieces"], res["n_groups"], res["k"]
    value = ws * n / (ms_all * 1e-3) / 1e9

    # ---- two batches in flight: a second pipeline (own context and buffers,
    # same input) so that one step's compression and Stage I overlap the
    # other step's merge (whose rounds kernel leaves most SMs idle)
    inflight = None
    pl2 = None
    if args.inflight > 1:
        ctx2 = jb.Context(local)
        ctx2.set_tuning(ctx.tuning())
        pl2 = jb.Pipeline(ctx2, off_np, n, p, group_capacity=pl.gcap)
        pl2.x.copy_(x_host, non_blocking=True)
        pl2.enqueue()
        ctx2.sync_status(where="second pipeline")
        if args.no_tune:
            fl = jb.InFlight([pl, pl2])
            inflight_tuning = ctx.tuning()
        else:
            inflight_tuning, _, fl = jb.tune_inflight([pl, pl2], ctx.tuning())
        for _ in range(2 * args.warmup):
            fl.step()
        fl.join()
        torch.cuda.synchronize()
        ctx.sync_status(where="in-flight warm-up")
        ctx2.sync_status(where="in-flight warm-up")
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(st)
        fl.fork(st)
        for _ in range(args.steps):
            fl.step()
        fl.join(st)
        e1.record(st)
        torch.cuda.synchronize()
        barrier(ws)
        ims = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
        ctx.sync_status(where="in-flight steps")
        ctx2.sync_status(where="in-flight steps")
        inflight = dict(value=ws * n / (ims * 1e-3) / 1e9, unit="Gpts/s", ms_per_step=ims, batches_in_flight=2,
                        tuning=inflight_tuning)
    # clocks sampled over both timed regions (one batch, two in flight)
    clocks = sampler.stop()

    # ---- e2e: H2D of the series from pinned memory, the step, D2H of the
    # symbols and dictionary, all inside the timed region
    e2e = None
    if not args.no_e2e:
        sym_host = torch.empty(max(N, 1), dtype=torch.int32, pin_memory=True)
        dl_host = torch.empty(max(k, 1), dtype=torch.float64, pin_memory=True)
        di_host = torch.empty(max(k, 1), dtype=torch.float64, pin_memory=True)
        dc_host = torch.empty(max(k, 1), dtype=torch.int64, pin_memory=True)

        def e2e_step():
            pl.x.copy_(x_host, non_blocking=True)
            pl.series_off.copy_(off_host, non_blocking=True)
            graphs[-1].replay()
            sym_host[:N].copy_(pl.b["symbol"][:N], non_blocking=True)
            dl_host[:k].copy_(pl.b["dict_len"][:k], non_blocking=True)
            di_host[:k].copy_(pl.b["dict_inc"][:k], non_blocking=True)
            dc_host[:k].copy_(pl.b["dict_count"][:k], non_blocking=True)

        e2e_tuning = tuning
        if inflight is not None:
            # the same two pipelines: the host->device copies run back to back
            # on a copy stream of their own (the copy of a step waits only
            # until the front half of the step two before it, on the same
            # pipeline, has read its input), each step waits for its copy,
            # runs, and copies its symbols and dictionary out on its stream,
            # so the link stays busy while the kernels of the steps overlap.
            # The steps run in the single-batch configuration: the link sets
            # the pace, and the copies, not the other batch's kernels, fill
            # the time beside each step, so each step's own latency counts
            # (the in-flight caps lengthen it).
            for q in (pl, pl2):
                q.ctx.set_tuning(tuning)
            fl = jb.InFlight([pl, pl2])
            syms = [sym_host, torch.empty_like(sym_host).pin_memory()]
            dicts = [(dl_host, di_host, dc_host),
                     tuple(torch.empty_like(t).pin_memory() for t in (dl_host, di_host, dc_host))]
            pls = [pl, pl2]
            cs = torch.cuda.Stream()
            copied = [torch.cuda.Event() for _ in pls]
            issued = [0, 0]

            def h2d_issue():
                i = fl.next_index()
                with torch.cuda.stream(cs):
                    if issued[i]:
                        cs.wait_event(fl.front_done[i])
                    pls[i].x.copy_(x_host, non_blocking=True)
                    pls[i].series_off.copy_(off_host, non_blocking=True)
                    copied[i].record(cs)
                issued[i] += 1

            def wait_copy(i, s):
                s.wait_event(copied[i])

            def d2h(i, s):
                b = pls[i].b
                syms[i][:N].copy_(b["symbol"][:N], non_blocking=True)
                for dst, key in zip(dicts[i], ("dict_len", "dict_inc", "dict_count")):
                    dst[:k].copy_(b[key][:k], non_blocking=True)

            def e2e_steps(n_steps):
                for _ in range(n_steps):
                    h2d_issue()
                    fl.step(wait_copy, d2h)

            cs.wait_stream(st)
            # two untimed steps per pipeline (a trace of this leg showed the
            # copies right after the first step of each pipeline running at
            # half the link rate once, then at full rate)
            e2e_steps(4)
            fl.join()
            torch.cuda.synchronize()
            barrier(ws)
            e0.record(st)
            fl.fork(st)
            cs.wait_stream(st)
            e2e_steps(args.steps)
            fl.join(st)
            st.wait_stream(cs)
            e1.record(st)
        else:
            e2e_step()
            torch.cuda.synchronize()
            barrier(ws)
            e0.record(st)
            for _ in range(args.steps):
                e2e_step()
            e1.record(st)
        torch.cuda.synchronize()
        barrier(ws)
        ems = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
        bi = 8 * n + 8 * (S + 1)
        bo = 4 * N + 24 * k
        e2e = dict(value=ws * n / (ems * 1e-3) / 1e9, unit="Gpts/s", h2d_bytes_per_step=bi, d2h_bytes_per_step=bo,
                   ms_per_step=ems, batches_in_flight=2 if inflight is not None else 1, tuning=e2e_tuning)
        ctx.sync_status(where="e2e steps")

    # ---- plain: the unbatched form (one compression launch and one Stage I
    # launch per domain, eager, no graph) on a bounded sample of the same
    # workload, next to the batched form on that sample
    plain = None
    if not args.no_plain:
        plain = plain_form(jb, synth, args, local, ws)

    # ---- rooflines (HBM; nothing here is a dense contraction): the three
    # largest stages and the dominant one (roofline_table)
    peak, peak_kind = peaks()
    roofline = roofline_table(args.workload, n, N, G, pl.D, comp_ms, loc_ms, rnd_ms,
                              "k_mrounds1" if ctx.tuning()["merge_form"] == 1 else "k_mrounds", peak, peak_kind)
    roofline["path_frac_of_point_roofline"] = value / ws / (peak / 8.0)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        xs, offs, cfgs = cpu_sample(args.workload, args.cpu_series)
        tcpu = oracle_step(xs, offs, cfgs, threads)
        cpu = dict(value=len(xs) / tcpu / 1e9, unit="Gpts/s", cores=threads, kind="oracle",
                   sample=f"first {args.cpu_series} series of the workload ({len(xs)} points), one pass; "
                          f"compression on {threads} threads, digitization serial")

    flips = None
    if rank == 0 and not args.no_cpu_baseline:
        flips = flip_count(pl, x_host.numpy(), cfg, args.cpu_series)

    if args.verify and rank == 0:
        verify_sample(pl, x_host.numpy(), off_np, cfg, args.verify)
    sweep = partition_sweep(jb, synth, local) if args.partition_sweep and rank == 0 else None

    # ---- the full-reassignment variant (Alg. 1 Digitize, the O(N k) argmin
    # pass that label propagation replaces): its time on this workload and the
    # SSE of both assignments (Table 2's comparison)
    reassign = None
    if not args.no_reassign:
        res = pl.as_result()
        ctx.reassign(res, p)
        ctx.sync_status(where="reassignment warm-up")
        e0.record(st)
        sym_re = ctx.reassign(res, p)
        e1.record(st)
        torch.cuda.synchronize()
        ra_ms = e0.elapsed_time(e1)
        s_two = float(ctx.sse(res, p, res["symbol"]).item())
        s_re = float(ctx.sse(res, p, sym_re).item())
        changed = float((sym_re != res["symbol"]).double().mean().item())
        ctx.sync_status(where="reassignment")
        reassign = dict(ms=ra_ms, sse_label_propagation=s_two, sse_reassigned=s_re,
                        sse_ratio=s_two / s_re if s_re > 0 else None, pieces_changed=changed)

    # ---- the block form of Sec. 5 (one global sort of the pieces, contiguous
    # sorted blocks, Stage II over the starting points) on the same batch, as
    # many blocks as domains: its dictionary and SSE beside the per-domain
    # form's (one eager pass, own context; timed end to end with its syncs)
    block = None
    if not args.no_block_form and rank == 0:
        res = pl.as_result()
        cbx = jb.Context(local)
        cbx.set_tuning(dict(ctx.tuning(), per_domain_launch=0))
        torch.cuda.synchronize()
        t0b = time.perf_counter()
        bo = cbx.symbolize_blocks(pl.x, pl.series_off, p, series_off_host=off_np)
        torch.cuda.synchronize()
        t_blk = time.perf_counter() - t0b
        s_blk = float(cbx.sse(bo, p, bo["symbol"]).item())
        s_dom = float(ctx.sse(res, p, res["symbol"]).item())
        cbx.sync_status(where="block form")
        block = dict(seconds_eager=t_blk, n_blocks=bo["n_blocks"], local_groups=bo["n_groups_host"],
                     dictionary=bo["k_host"], sse=s_blk, per_domain=dict(local_groups=G, dictionary=k, sse=s_dom),
                     sse_ratio_block_to_domain=s_blk / s_dom if s_dom > 0 else None)
        del bo, cbx
        torch.cuda.empty_cache()

    if rank == 0:
        single = dict(value=value, unit="Gpts/s", ms_per_step=ms_all, tuning=tuning,
                      form="one batch at a time: CUDA-graph replay of the whole step")
        head_value, head_ms = (inflight["value"], inflight["ms_per_step"]) if inflight else (value, ms_all)
        form = ("batched, two batches in flight: two pipelines on two streams, each step one CUDA-graph replay "
                "of compression + Stage I and one of merge + labels; merges ordered one after the other"
                if inflight else "batched: CUDA-graph replay of the whole step")
        roofline["path_frac_of_point_roofline"] = head_value / ws / (peak / 8.0)
        line = dict(metric=METRIC, value=head_value, unit="Gpts/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
                    ms_per_step=head_ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                    data="synthetic",
                    config=dict(workload=WORKLOAD_DESC[args.workload], n_series=S, n_points=n, pieces=N,
                                local_groups=G, dictionary=k, parallelism=f"replicas x{ws}",
                                l2="input 8 B/point >> L2 (no flush needed)" if 8 * n > 2e9 else "input fits L2",
                                form=form, tuning=inflight["tuning"] if inflight else tuning),
                    roofline=roofline, cpu_baseline=cpu, e2e=e2e, plain=plain, single_batch=single, clocks=clocks,
                    breakpoint_flips=flips,
                    gpu_launches=kernels_per_step * args.steps,
                    stage_ms=dict(compress=float(np.mean(comp_ms)), finish=float(np.mean(fin_ms)),
                                  local=float(np.mean(loc_ms)), merge=float(np.mean(mrg_ms)),
                                  merge_rounds_kernel=float(np.mean(rnd_ms)), symbolize=float(np.mean(sym_ms))),
                    diagnostics=diag, input_gen_s=t_gen)
        if sweep is not None:
            line["partition_sweep"] = sweep
        if block is not None:
            line["block_form"] = block
        if reassign is not None:
            line["reassignment"] = reassign
        print(json.dumps(line), flush=True)


def plain_form(jb, synth, args, local, ws):
    import torch
    xs, offs, cfgs = synth.make(args.workload, max_series=args.plain_series)
    p = jb.Params(tol=cfgs["tol"], alpha=cfgs["alpha"], scl=cfgs["scl"], domain_mode=cfgs["domain_mode"],
                  domain_value=cfgs["domain_value"])
    n = len(xs)
    out = {}
    for form in ("plain", "batched"):
        c = jb.Context(local)
        c.set_tuning(dict(per_domain_launch=1 if form == "plain" else 0))
        pl = jb.Pipeline(c, offs, n, p, group_capacity=max(1 << 12, n // 4))
        pl.x.copy_(torch.from_numpy(xs))
        pl.enqueue()
        c.sync_status(where=form + " sample")
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if form == "plain":
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(args.plain_steps):
                pl.enqueue()
            e1.record(st)
        else:
            g = pl.capture()
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(args.plain_steps):
                g.replay()
            e1.record(st)
        torch.cuda.synchronize()
        c.sync_status(where=form + " sample steps")
        ms = max_over_ranks(e0.elapsed_time(e1) / args.plain_steps, ws)
        out[form] = dict(value=ws * n / (ms * 1e-3) / 1e9, ms_per_step=ms)
        del pl, c
    pl_ = out["plain"]
    return dict(value=pl_["value"], unit="Gpts/s", ms_per_step=pl_["ms_per_step"],
                sample=f"first {args.plain_series} series of the workload ({n} points, "
                       f"{jb.Context.plan(offs, p)[0]} domains)",
                form="per-domain launches: one compression launch and one Stage I launch per domain, "
                     "issued eagerly (no CUDA graph); normalisation, merge and label propagation as single launches",
                batched_same_sample=dict(value=out["batched"]["value"], unit="Gpts/s",
                                         ms_per_step=out["batched"]["ms_per_step"]))


def partition_sweep(jb, synth, local, steps=20):
    """Sec. 7.3's experiment on the GPU path: one series of 100,000 N(0, 1)
    draws (tol = 0.01, alpha = 0.05) cut into M equal domains; per M the
    pieces, local groups, dictionary size, reconstruction MSE and the
    CUDA-event time of the whole forward step (median of graph replays), and
    the oracle's single-thread time on the same input."""
    import torch
    import oracle
    oracle.build()
    x_np, off_np, cfg = synth.make("noise")
    x = torch.from_numpy(x_np).cuda()
    off = torch.from_numpy(off_np).cuda()
    rows = []
    for M in (1, 2, 4, 8, 16, 32, 64, 128, 256):
        p = jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                      domain_value=M)
        c = jb.Context(local)
        out = c.symbolize(x, off, p, series_off_host=off_np)
        _, xhat = c.reconstruct(x, off, out, p)
        mse = float(c.mse(x, xhat).item())
        pl = jb.Pipeline(c, off_np, len(x_np), p, group_capacity=max(out["n_groups_host"] + 1024, 4096))
        pl.x.copy_(x)
        pl.enqueue()
        c.sync_status(where=f"sweep M={M}")
        g = pl.capture()
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        c.sync_status(where=f"sweep M={M} replays")
        t0 = time.perf_counter()
        oracle.pipeline(x_np, off_np, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"], M, threads=1,
                        with_reconstruct=False)
        t_cpu = time.perf_counter() - t0
        rows.append(dict(M=M, pieces=out["n_pieces"], local_groups=out["n_groups_host"], symbols=out["k_host"],
                         mse=mse, gpu_ms=float(np.median(ts)), oracle_1thread_ms=1e3 * t_cpu))
        del pl, g, c
    return rows


def flip_count(pl, x, cfg, n_series):
    """Breakpoint flips of the GPU's pieces against Eq. 1 read literally (the
    plain sequential sum of squared residuals, oracle) on the domains of the
    first n_series series: the library decides Eq. 1 in its L^2-scaled exact
    form, and the two may differ only where the error lies within rounding of
    the bound.  Counts the flips and the largest |err - bound| / bound."""
    import oracle
    b = pl.b
    S = min(n_series, pl.S)
    Ds = int(b["series_dom_off"][S].item())
    db = b["dom_begin"][:Ds].cpu().numpy()
    de = b["dom_end"][:Ds].cpu().numpy()
    so = b["dom_slot_off"][:Ds].cpu().numpy()
    cnt = b["dom_piece_cnt"][:Ds].cpu().numpy().astype(np.int64)
    end = int(so[-1] + cnt[-1]) if Ds else 0
    plen = b["piece_len"][:end].cpu().numpy()
    ln = np.concatenate([plen[so[d]:so[d] + cnt[d]] for d in range(Ds)]) if Ds else np.zeros(0, np.int32)
    po = np.concatenate([[0], np.cumsum(cnt)])
    r = oracle.breakpoint_flips(x, db, de, ln, po, cfg["tol"], threads=os.cpu_count() or 1)
    gaps = [abs(err - bound) / bound for _, _, err, bound in r["flips"] if bound > 0]
    return dict(flips=len(r["flips"]), pieces_checked=r["pieces"], max_rel_gap=max(gaps) if gaps else None,
                rule="|err - bound| < 1e-12 bound at every flip",
                rule_holds=all(g < 1e-12 for g in gaps) and all(bd > 0 for _, _, _, bd in r["flips"]),
                sample=f"domains of the first {S} series ({Ds} domains)")


def verify_sample(pl, x, off, cfg, n_dom):
    """Full-size parity on a sample: the oracle compresses n_dom domains drawn
    at random and must reproduce their pieces bit for bit."""
    import oracle
    b = pl.b
    D = pl.D
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(D, min(n_dom, D), replace=False))
    db = b["dom_begin"].cpu().numpy()
    de = b["dom_end"].cpu().numpy()
    so = b["dom_slot_off"].cpu().numpy()
    cnt = b["dom_piece_cnt"][:D].cpu().numpy()
    plen = b["piece_len"].cpu().numpy()
    pinc = b["piece_inc"].cpu().numpy()
    bad = 0
    for d in pick:
        ln, inc, _ = oracle.compress(x, db[d:d + 1], de[d:d + 1], cfg["tol"])
        g_ln = plen[so[d]:so[d] + cnt[d]]
        g_inc = pinc[so[d]:so[d] + cnt[d]]
        if not (np.array_equal(ln, g_ln) and np.array_equal(inc, g_inc)):
            bad += 1
    print(json.dumps(dict(verify_domains=len(pick), mismatched=bad)), file=sys.stderr, flush=True)
    if bad:
        raise SystemExit(f"parity failure on {bad} of {len(pick)} sampled domains")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_DESC), default="scale")
    ap.add_argument("--max-series", type=int, default=None)
    ap.add_argument("--cpu-series", type=int, default=2000)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain-series", type=int, default=300, help="series in the plain-form sample")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--no-reassign", action="store_true", help="skip the full-reassignment comparison")
    ap.add_argument("--no-block-form", action="store_true", help="skip the block-form (Sec. 5 as stated) comparison")
    ap.add_argument("--partition-sweep", action="store_true",
                    help="add the Gaussian-noise partition sweep (Sec. 7.3) to the JSON line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--inflight", type=int, default=2, choices=[1, 2],
                    help="batches in flight (2: two pipelines on two streams)")
    ap.add_argument("--verify", type=int, default=0, help="oracle-check this many sampled domains")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
