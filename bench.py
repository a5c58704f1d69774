#!/usr/bin/env python
"""Device-resident decode benchmark (one JSON line on stdout).

Workload (default): the chr1-shaped synthetic genome of 253,935,557 B
(seed 0; 15,499 blocks of 16 KiB), encoded by the library encoder with the
4-entry distance history; one step = one full device-resident decode
(rANS of the four streams + parse + match copy) from the archive in HBM to
the output in HBM, through aceapex_decode_all.

Metric: decoded GB/s (decompressed bytes / device time), with the roofline of
the dominant kernel, the whole-path HBM fraction, an end-to-end number
through aceapex_decode_host (host archive -> host output, copies inside the
timed region), and the CPU oracle timed on the host as the baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--corpus dna|text] [--encoding history|no_rep] [--variant fast|plain]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

GENOME = synth.GENOME_CHR1_SIZE
TEXT = 200 * 1024 * 1024
L2_FLUSH = 256 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="single", choices=["single", "batch", "serve", "depth", "serve-encode"],
                   help="single: one archive (--corpus); batch: the 96-archive mixed batch; serve: region server; "
                        "depth: the encoder's chain-depth statistics of the corpus (host only, no GPU); "
                        "serve-encode: write the serving archive to the cache (host only)")
    p.add_argument("--corpus", default="dna", choices=["dna", "text"])
    p.add_argument("--size", type=int, default=0)
    p.add_argument("--encoding", default="history", choices=["history", "no_rep"])
    p.add_argument("--variant", default="fast", choices=["fast", "plain", "fused"],
                   help="fast: entropy stage, local pass, cross-block pass; plain: the serial history-bound "
                        "decoder; fused: entropy stage and local pass in one kernel (single-archive decodes)")
    p.add_argument("--lanes", type=int, default=32)
    p.add_argument("--wait-ns", type=int, default=0,
                   help="decoder: first cross-block round's wait per piece (0: library default)")
    p.add_argument("--shard", action="store_true",
                   help="N GPUs split the output blocks (each decodes its range's closure) instead of replicas")
    p.add_argument("--max-depth", type=int, default=0,
                   help="encoder chain-depth cap (0: the library default of 16)")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the comparison measurements (plain decoder, history-free, text, serving)")
    p.add_argument("--no-serve", action="store_true", help="skip the serving measurement among the comparisons")
    p.add_argument("--levels", type=int, default=0,
                   help="1: encode with level bodies (the cross-block pass may take pieces in level order); "
                        "0: without")
    p.add_argument("--no-graph", action="store_true", help="batch: plain launches instead of a graph replay")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="batch: keep the default lane cap and launch shapes")
    p.add_argument("--serve-gib", type=int, default=16, help="serve: genome size in GiB (256 MiB chromosomes)")
    p.add_argument("--serve-rate", type=float, default=20000.0, help="serve: Poisson arrivals per second")
    p.add_argument("--serve-seconds", type=float, default=10.0, help="serve: measured seconds (after 2 s warm-up)")
    p.add_argument("--cache-gib", type=float, default=4.0, help="serve: decoded-block cache in GiB")
    p.add_argument("--serve-streams", type=int, default=2, help="serve: tick lanes (streams)")
    p.add_argument("--cache-dir", default=os.environ.get("ACEAPEX_CACHE", "/tmp/aceapex_bench_cache"))
    return p.parse_args()


def workload(args):
    size = args.size or (GENOME if args.corpus == "dna" else TEXT)
    name = (f"chr1-shaped synthetic genome {size:,} B" if args.corpus == "dna" and size == GENOME
            else f"synthetic {args.corpus} {size:,} B")
    return size, name


def encoder_key():
    h = hashlib.sha256()
    for f in ("encode.cpp", "internal.h", "plan.h"):
        h.update(open(os.path.join(ROOT, "paper_2608_10188_gb300", "csrc", f), "rb").read())
    h.update(open(os.path.join(ROOT, "synth", "synth.c"), "rb").read())
    return h.hexdigest()[:16]


def get_archive(args, acx):
    """Generate the corpus and encode it with the library encoder (cached on
    the local disk between runs of the same source version)."""
    size, _ = workload(args)
    data = synth.corpus(args.corpus, size, 0)
    key = (f"{args.corpus}-{size}-s0-{args.encoding}-k{args.lanes}-d{args.max_depth}-lv{args.levels}-"
           f"{encoder_key()}.acx")
    path = os.path.join(args.cache_dir, key)
    arc = None
    if os.path.exists(path):
        arc = open(path, "rb").read()
    if arc is None:
        arc = acx.encode(data, no_rep=args.encoding == "no_rep", max_lanes=args.lanes, max_depth=args.max_depth,
                         levels=bool(args.levels))
        try:
            os.makedirs(args.cache_dir, exist_ok=True)
            tmp = path + f".{os.getpid()}"
            with open(tmp, "wb") as f:
                f.write(arc)
            os.replace(tmp, path)
        except OSError:
            pass
    return data, arc


def cached_encode(args, acx, data, key, **kw):
    path = os.path.join(args.cache_dir, key)
    if os.path.exists(path):
        return open(path, "rb").read()
    arc = acx.encode(data, **kw)
    try:
        os.makedirs(args.cache_dir, exist_ok=True)
        tmp = path + f".{os.getpid()}.{threading.get_ident()}"
        with open(tmp, "wb") as f:
            f.write(arc)
        os.replace(tmp, path)
    except OSError:
        pass
    return arc


def tune_lanes(args, acx, torch, ctx, device):
    """The encode-side tuning lever: the rANS lane cap.  Samples of both
    corpora (8 MiB each, seeds 4000/4001) are encoded with every cap and
    decoded as one batch; the cap with the fastest decode is used."""
    from concurrent.futures import ThreadPoolExecutor
    samples = [synth.dna(8 << 20, 4000), synth.text(8 << 20, 4001)]
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=device)
    sh = torch.cuda.current_stream().cuda_stream
    res = {}
    for K in (8, 16, 32, 64, 128):
        with ThreadPoolExecutor(max_workers=2) as ex:
            arcs = list(ex.map(lambda d: acx.encode(d, max_lanes=K, threads=1), samples))
        keep, archives, outs = [], [], []
        for a in arcs:
            h = np.frombuffer(a, np.uint8).copy()
            d = torch.from_numpy(h).to(device)
            keep.append(d)
            A = acx.Archive(ctx, d.data_ptr(), h, h.size)
            archives.append(A)
            outs.append(torch.empty(A.total, dtype=torch.uint8, device=device))
        b = acx.Batch(ctx, [(A, o.data_ptr(), A.total) for A, o in zip(archives, outs)], graph=False)
        ms = []
        for r in range(6):
            flush.fill_(1)
            rc, _, st = b.run(sh, stats=True)
            if rc != 0:
                raise RuntimeError(f"lane tuning decode failed: {rc}")
            if r:
                ms.append(st["ms_total"])
        b.close()
        for A in archives:
            A.close()
        res[K] = statistics.median(ms)
    return min(res, key=res.get), res


def batch_archives(args, acx):
    """The mixed batch workload: 96 archives, sizes log-uniform in
    [64 KiB, 64 MiB] (seed 4), archive i from seed 1000+i, DNA for even i and
    text for odd i, history-free encoding for i mod 4 in {2, 3}.  Archives are
    encoded in parallel (one encoder thread each)."""
    from concurrent.futures import ThreadPoolExecutor
    specs = synth.batch_specs()
    ek = encoder_key()

    def one(s):
        data = synth.corpus(s["kind"], s["size"], s["seed"])
        key = f"batch-{s['kind']}-{s['size']}-s{s['seed']}-{int(s['no_rep'])}-k{args.lanes}-{ek}.acx"
        arc = cached_encode(args, acx, data, key, no_rep=s["no_rep"], max_lanes=args.lanes, threads=1)
        return data, arc

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, sorted(specs, key=lambda s: -s["size"])))
    order = sorted(range(len(specs)), key=lambda i: -specs[i]["size"])
    out = [None] * len(specs)
    for k, i in enumerate(order):
        out[i] = res[k]
    return specs, out


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling every 100 ms and wait (up to 3 s) for the first
        sample, so that sampling runs before the timed region begins."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        """Stop after one more sample (up to 0.5 s): short timed regions fall
        between two samples, one taken before and one after them."""
        if not self.proc:
            return None
        n0, t0 = len(self.lines), time.perf_counter()
        while len(self.lines) == n0 and time.perf_counter() - t0 < 0.5 and self.proc.poll() is None:
            time.sleep(0.005)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def cpu_oracle_baseline(arc, data, repeats=3):
    import oracle
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        out = oracle.decode(arc, verify=False)
        times.append(time.perf_counter() - t)
    if not np.array_equal(out, data):
        raise RuntimeError("oracle decode mismatch")
    med = statistics.median(times)
    return {"value": round(data.size / med / 1e9, 4), "unit": "GB/s", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"whole archive ({data.size:,} B decoded), single-threaded C oracle, median of {repeats}"}


def timed_decode(acx, torch, dev, flush, sh, data, arc, steps, warmup, **ctx_kw):
    """One archive decoded `steps` times after `warmup` warm-ups, the L2
    flushed between steps and every step timed with CUDA events on the
    stream, after a correctness gate against the input; clocks sampled over
    the timed steps."""
    device = f"cuda:{dev}"
    ctx = acx.Context(dev, **ctx_kw)
    h = np.frombuffer(arc, np.uint8).copy()
    d = torch.from_numpy(h).to(device)
    A = acx.Archive(ctx, d.data_ptr(), h, h.size)
    out = torch.empty(max(data.size, 1), dtype=torch.uint8, device=device)
    rc = acx.decode_all(ctx, A, out.data_ptr(), data.size, sh)
    if rc != 0:
        raise RuntimeError(f"decode failed: {rc} {ctx.last_error()}")
    if not torch.equal(out[:data.size], torch.from_numpy(data).to(device)):
        raise RuntimeError("GPU decode differs from the input")
    for _ in range(warmup):
        flush.fill_(1)
        acx.decode_all(ctx, A, out.data_ptr(), data.size, sh)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    rows, st = [], {}
    for _ in range(steps):
        flush.fill_(1)
        r, st = acx.decode_all(ctx, A, out.data_ptr(), data.size, sh, stats=True)
        if r != 0:
            raise RuntimeError(f"decode failed: {r} {ctx.last_error()}")
        rows.append((st["ms_total"], st["ms_ans"], st["ms_parse"], st["ms_copy"]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot = sum(r[0] for r in rows)
    res = {"value": round(data.size * steps / (tot / 1e3) / 1e9, 3), "unit": "GB/s",
           "ms_per_step": round(tot / steps, 4),
           "stage_ms": {"ans": round(statistics.mean(r[1] for r in rows), 4),
                        "local_parse_copy": round(statistics.mean(r[2] for r in rows), 4),
                        "cross_block": round(statistics.mean(r[3] for r in rows), 4)},
           "archive_bytes": len(arc), "ratio": round(data.size / len(arc), 4),
           "pending_pieces": st.get("pending_spans"), "rounds_after_first": st.get("wait_polls"),
           "verified": "decoded output equals the input", "clocks": clk}
    A.close()
    ctx.close()
    return res


def start_extra_encodes(args, acx, gdata):
    """Encode the archives of the comparison measurements on background
    threads while the headline runs: the genome history-free (level bodies
    as in the headline), and the 200 MiB text in both encodings with level
    bodies (its many pieces per lane are taken in level order)."""
    from concurrent.futures import ThreadPoolExecutor
    ex = ThreadPoolExecutor(max_workers=3)
    ek = encoder_key()
    tdata = synth.corpus("text", TEXT, 0)
    futs = {"text_data": tdata}
    futs["genome_history_free"] = ex.submit(
        cached_encode, args, acx, gdata, f"dna-{gdata.size}-s0-no_rep-k{args.lanes}-lv{args.levels}-{ek}.acx",
        no_rep=True, max_lanes=args.lanes, levels=bool(args.levels))
    for enc in ("history", "no_rep"):
        futs[f"text_{enc}"] = ex.submit(
            cached_encode, args, acx, tdata, f"text-{TEXT}-s0-{enc}-k{args.lanes}-lv1-{ek}.acx",
            no_rep=enc == "no_rep", max_lanes=args.lanes, levels=True)
    futs["pool"] = ex
    return futs


def comparison_extras(args, acx, torch, dev, flush, sh, gdata, garc, futs):
    """The comparisons the headline is read against, measured in the same
    process on the same GPU: the plain history-bound decoder on the headline
    archive, the history-free genome, the 200 MiB text in both encodings,
    and the region server under load."""
    steps, warm = max(5, args.steps // 2), 3
    out = {}
    out["plain"] = dict(workload="the headline archive, plain decoder (serial parse with the history, "
                                 "byte-serial copies)",
                        **timed_decode(acx, torch, dev, flush, sh, gdata, garc, steps, warm,
                                       variant=acx.lib.VARIANT_PLAIN))
    out["history_free"] = dict(workload=f"the same genome encoded history-free ({gdata.size:,} B)",
                               **timed_decode(acx, torch, dev, flush, sh, gdata,
                                              futs["genome_history_free"].result(), steps, warm))
    tdata = futs["text_data"]
    out["text"] = {"workload": f"synthetic Zipf text {tdata.size:,} B (50k-word vocabulary, s = 1.1), "
                               "level bodies"}
    for enc, key in (("history", "text_history"), ("history_free", "text_no_rep")):
        out["text"][enc] = timed_decode(acx, torch, dev, flush, sh, tdata, futs[key].result(), steps, warm)
    futs["pool"].shutdown()
    hist, hfree = out["text"]["history"], out["text"]["history_free"]
    out["history_free_vs_plain"] = round(out["history_free"]["value"] / out["plain"]["value"], 2)
    out["text"]["history_free_vs_history"] = round(hfree["value"] / hist["value"], 3)
    if not args.no_serve:
        out["serve"] = serve_measure(args, dev)
    return out


def run_reference(args, dist):
    """The oracle timed on the host cores (bench --impl reference)."""
    rank = dist["rank"]
    if rank != 0:
        return
    import oracle
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    data, arc = get_archive(args, acx)
    size, wname = workload(args)
    for _ in range(args.warmup):
        oracle.decode(arc, verify=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = oracle.decode(arc, verify=False)
    el = time.perf_counter() - t0
    if not np.array_equal(out, data):
        raise RuntimeError("oracle decode mismatch")
    value = size * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": "device-resident decode GB/s", "value": round(value, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": wname, "encoding": args.encoding, "block_size": 16384},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": f"whole archive per step ({size:,} B), single-threaded C oracle"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, dist):
    """The mixed batch workload: 96 archives decoded by one graph-replayed
    batch per step (aceapex_batch_run), against the same archives decoded by
    one aceapex_decode_all_async per archive."""
    import torch

    import paper_2608_10188_gb300 as acx
    acx.build.build()
    dev = dist["local"]
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    variant = acx.lib.VARIANT_PLAIN if args.variant == "plain" else acx.lib.VARIANT_FAST
    ctx = acx.Context(dev, variant=variant, wait_ns=args.wait_ns)
    lanes_ms = None
    if args.autotune:
        args.lanes, lanes_ms = tune_lanes(args, acx, torch, ctx, device)
    specs, pairs = batch_archives(args, acx)
    d_arcs, archives, outs = [], [], []
    for data, arc in pairs:
        h = np.frombuffer(arc, dtype=np.uint8).copy()
        d = torch.from_numpy(h).to(device)
        d_arcs.append(d)
        A = acx.Archive(ctx, d.data_ptr(), h, h.size)
        archives.append(A)
        outs.append(torch.empty(max(A.total, 1), dtype=torch.uint8, device=device))
    total = sum(A.total for A in archives)
    arc_total = sum(len(a) for _, a in pairs)
    entries = [(A, o.data_ptr(), A.total) for A, o in zip(archives, outs)]
    tuned = None
    if args.autotune:
        tuned = acx.tune.tuned_params(ctx, entries, f"batch96-k{args.lanes}-{encoder_key()}",
                                      os.path.join(args.cache_dir, "autotune.json"), reps=3, device=dev)
    graph = not args.no_graph
    B = acx.Batch(ctx, entries, graph=graph)
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=device)
    sh = torch.cuda.current_stream().cuda_stream

    def check(tag):
        for (data, _), A, o in zip(pairs, archives, outs):
            if not torch.equal(o[:A.total], torch.from_numpy(data).to(device)):
                raise RuntimeError(f"{tag}: GPU decode differs from the input")

    rc, per = B.run(sh)
    if rc != 0 or any(per):
        raise RuntimeError(f"batch decode failed: {rc} {per} {ctx.last_error()}")
    check("batch")
    for _ in range(args.warmup):
        flush.fill_(1)
        B.run(sh)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ms = []
    st = {}
    for _ in range(args.steps):
        flush.fill_(1)
        rc, per, st = B.run(sh, stats=True)
        if rc != 0:
            raise RuntimeError(f"batch decode failed: {rc} {ctx.last_error()}")
        ms.append(st["ms_total"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = statistics.median(ms)
    value = total / (ms_step / 1e3) / 1e9

    # stage split from the same batch without a graph (events between the launches)
    Bs = acx.Batch(ctx, entries, graph=False)
    sa, sl, sx, sst = [], [], [], {}
    for _ in range(max(3, min(args.steps, 5))):
        flush.fill_(1)
        rc, per, sst = Bs.run(sh, stats=True)
        sa.append(sst["ms_ans"])
        sl.append(sst["ms_parse"])
        sx.append(sst["ms_copy"])
    Bs.close()
    pb = {"payload": 0, "decoded": 0}
    for _, a in pairs:
        q = stream_bytes(a)
        pb["payload"] += q["payload"]
        pb["decoded"] += q["decoded"]
    n_blocks = sum(A.info["n_blocks"] for A in archives)
    roof, path_roof = rooflines({"ans": statistics.median(sa), "local": statistics.median(sl),
                                 "cross": statistics.median(sx)}, pb, total, arc_total, sst, n_blocks,
                                args.variant, ms_step)

    # the same archives, one decode launch sequence per archive
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_ms = []
    for it in range(args.warmup + max(3, min(args.steps, 10))):
        flush.fill_(1)
        e0.record()
        for A, o in zip(archives, outs):
            acx.decode_all_async(ctx, A, o.data_ptr(), A.total, sh)
        e1.record()
        if ctx.sync(sh) != 0:
            raise RuntimeError(f"per-archive decode failed: {ctx.last_error()}")
        if it >= args.warmup:
            per_ms.append(e0.elapsed_time(e1))
    check("per-archive")
    per_gbs = total / (statistics.median(per_ms) / 1e3) / 1e9

    cpu = None
    if dist["rank"] == 0 and not args.no_cpu_baseline:
        import oracle
        small = sorted(range(len(specs)), key=lambda i: specs[i]["size"])[: len(specs) // 2]
        t = time.perf_counter()
        nb = 0
        for i in small:
            oracle.decode(pairs[i][1], verify=False)
            nb += specs[i]["size"]
        el = time.perf_counter() - t
        cpu = {"value": round(nb / el / 1e9, 4), "unit": "GB/s", "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"the {len(small)} smallest archives of the batch ({nb:,} B), single-threaded C oracle"}
    if dist["rank"] == 0:
        kinds = {k: sum(1 for s in specs if s["kind"] == k) for k in ("dna", "text")}
        line = {
            "metric": "device-resident decode GB/s", "value": round(value, 3), "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded generators)",
            "config": {"workload": f"batch of {len(specs)} archives, {total:,} B (log-uniform 64 KiB-64 MiB; "
                                   f"{kinds['dna']} DNA, {kinds['text']} text; history-free for i mod 4 in {{2,3}})",
                       "launch": "one CUDA graph replay per step" if graph else "one launch sequence per step",
                       "autotuned": None if tuned is None else {
                           "rans_lanes_ms": {str(k): round(v, 4) for k, v in lanes_ms.items()},
                           "ctas_per_sm": tuned["ctas_per_sm"], "rans_ctas_per_sm": tuned["rans_ctas_per_sm"],
                           "queue_chunk": tuned["queue_chunk"], "cached": tuned["cached"]},
                       "variant": args.variant, "rans_lanes": args.lanes, "blocks": n_blocks,
                       "archive_bytes": arc_total, "ratio": round(total / arc_total, 4),
                       "l2": "256 MiB buffer written between steps; per-step CUDA events exclude it"},
            "per_archive_launches": {"value": round(per_gbs, 3), "unit": "GB/s",
                                     "ms_per_step": round(statistics.median(per_ms), 4),
                                     "launches_per_step": 4 * len(specs)},
            "stage_ms": {"ans": round(statistics.median(sa), 4), "local_parse_copy": round(statistics.median(sl), 4),
                         "cross_block": round(statistics.median(sx), 4)},
            "cross_block_stats": {"pending_pieces": sst.get("pending_spans"), "pending_bytes": sst.get("pending_bytes"),
                                  "rounds_after_first": sst.get("wait_polls")},
            "roofline": roof, "path_roofline": path_roof, "e2e": None, "cpu_baseline": cpu,
            "gpu_launches": 4 * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    B.close()
    for A in archives:
        A.close()
    ctx.close()


def serve_data(args):
    """The serving workload's input: a synthetic genome of serve_gib GiB made
    of 256 MiB chromosomes (chromosome i from seed 5000+i, generated in
    parallel)."""
    from concurrent.futures import ThreadPoolExecutor
    chrom = 256 << 20
    size = args.serve_gib << 30
    n_chrom = (size + chrom - 1) // chrom
    data = np.empty(size, dtype=np.uint8)

    def gen(i):
        n = min(chrom, size - i * chrom)
        synth.dna(n, 5000 + i, out=data[i * chrom:i * chrom + n])

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(gen, range(n_chrom)))
    key = f"serve-{size}-chrom{chrom}-k{args.lanes}-{encoder_key()}.acx"
    return data, key, chrom


def run_serve_encode(args):
    """Encode the serving archive into the cache (the 4-entry history, one
    parse per chromosome) and exit."""
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    data, key, chrom = serve_data(args)
    cached_encode(args, acx, data, key, max_lanes=args.lanes, segment=chrom, threads=os.cpu_count() or 4)


def serve_archive(args, acx):
    """The serving workload's input and archive.  An archive not yet cached is
    encoded by a child process, and the dirty pages are flushed before the
    measurement: after an encode of this size in the measuring process the
    server sustained about 7,500 of the 20,000 requests/s offered, against
    all of them when the archive came from the cache."""
    data, key, chrom = serve_data(args)
    path = os.path.join(args.cache_dir, key)
    if not os.path.exists(path):
        subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", "serve-encode",
                        "--serve-gib", str(args.serve_gib), "--lanes", str(args.lanes), "--cache-dir", args.cache_dir],
                       check=False)
        os.sync()
    arc = cached_encode(args, acx, data, key, max_lanes=args.lanes, segment=chrom, threads=os.cpu_count() or 4)
    return data, arc


def host_memory_gib():
    """MemTotal and MemAvailable of the host, GiB (None where /proc is absent)."""
    try:
        kv = {}
        for line in open("/proc/meminfo"):
            k, v = line.split(":", 1)
            kv[k] = int(v.split()[0]) / (1 << 20)
        return {"total": round(kv["MemTotal"], 1), "available": round(kv["MemAvailable"], 1)}
    except (OSError, KeyError, ValueError):
        return None


def run_serve(args, dist):
    line = serve_measure(args, dist["local"])
    print(json.dumps(line), flush=True)


def serve_measure(args, dev):
    """Region serving under open-loop Poisson load: requests with lognormal
    lengths (median 16 KiB, sigma 1, clipped to [4 KiB, 1 MiB]) at uniform
    starts arrive at serve_rate per second for 2 s of warm-up plus
    serve_seconds measured; each is decoded through its byte-level closure
    minus the device cache.  Latency = arrival -> completion seen by the
    server; the line reports p50/p99 of the measured window."""
    import torch

    import paper_2608_10188_gb300 as acx
    acx.build.build()
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    t_setup = time.perf_counter()
    data, arc = serve_archive(args, acx)
    total = data.size
    ctx = acx.Context(dev)
    h_arc = np.frombuffer(arc, dtype=np.uint8).copy()
    d_arc = torch.from_numpy(h_arc).to(device)
    A = acx.Archive(ctx, d_arc.data_ptr(), h_arc, h_arc.size)
    t = time.perf_counter()
    A.build_index()
    index_s = time.perf_counter() - t
    srv = acx.Server(ctx, A, cache_bytes=int(args.cache_gib * (1 << 30)), streams=args.serve_streams)
    warm = 2.0
    rng = np.random.default_rng(55)
    horizon = warm + args.serve_seconds
    n_req = int(args.serve_rate * horizon * 1.2) + 16
    at = np.cumsum(rng.exponential(1.0 / args.serve_rate, n_req))
    at = at[at < horizon]
    n_req = at.size
    lens = np.clip(rng.lognormal(np.log(16384), 1.0, n_req), 4096, 1 << 20).astype(np.int64)
    starts = (rng.random(n_req) * (total - lens + 1)).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)])
    arena = torch.empty(int(offs[-1]), dtype=torch.uint8, device=device)
    ptrs = (arena.data_ptr() + offs[:-1]).astype(np.uint64)
    setup_s = time.perf_counter() - t_setup
    clocks = ClockSampler(dev)
    clocks.start()
    t0 = srv.now_ns() + 50_000_000
    at_ns = (t0 + at * 1e9).astype(np.int64)
    ids = srv.submit_many(starts.astype(np.uint64), lens.astype(np.uint64), ptrs, at_ns)
    rc = srv.drain(int((horizon + 120) * 1000))
    clk = clocks.stop()
    if rc != 0:
        raise RuntimeError(f"server drain: {rc} {srv.last_error()}")
    comps = srv.poll(n_req + 16)
    st_all = srv.stats()
    by_id = {c["id"]: c for c in comps}
    idx = {int(i): k for k, i in enumerate(ids)}
    lat, win_bytes, closure, t_last = [], 0, [], 0.0
    served, dec_blocks = [], []
    bad = [c for c in comps if c["status"] != 0]
    if bad:
        raise RuntimeError(f"{len(bad)} requests failed, first status {bad[0]['status']}")
    for c in comps:
        k = idx[c["id"]]
        if at[k] >= warm:
            lat.append(c["latency_us"])
            win_bytes += int(lens[k])
            closure.append(c["closure_blocks"])
            served.append(c["latency_us"] - c["queue_us"])
            dec_blocks.append(c["decoded_blocks"])
            t_last = max(t_last, at[k] + c["latency_us"] / 1e6)
    lat = np.array(lat)
    # service time (admission -> completion) against the blocks a request
    # added to its tick's decode: fixed cost + cost per block, the form of
    # the paper's single-seek model (a launch-bound fixed part plus a part
    # that scales with work); meaningful when ticks hold one request each
    if len(set(dec_blocks)) > 1:
        slope, fixed = np.polyfit(np.array(dec_blocks, float), np.array(served, float), 1)
        fit = {"fixed_us": round(float(fixed), 1), "us_per_decoded_block": round(float(slope), 3),
               "requests": len(served)}
    else:
        fit = None
    # correctness: a sample of the requests against the generator's bytes
    smp = rng.choice(n_req, size=min(2000, n_req), replace=False)
    for k in smp:
        o, s, l = int(offs[k]), int(starts[k]), int(lens[k])
        if not np.array_equal(arena[o:o + l].cpu().numpy(), data[s:s + l]):
            raise RuntimeError(f"request {k} differs from the input")
    window = t_last - warm
    gbs = win_bytes / window / 1e9 if window > 0 else 0.0
    line = {
        "metric": "p99 region latency under load", "value": round(float(np.percentile(lat, 99)), 1), "unit": "us",
        "n_gpus": 1, "steps": int(lat.size), "warmup": int(n_req - lat.size),
        "ms_per_step": round(float(np.mean(lat)) / 1e3, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded generator; 256 MiB chromosomes)",
        "config": {"workload": f"region server over a {args.serve_gib} GiB synthetic genome ({total:,} B, "
                               f"{len(arc):,} B compressed, held on the device), {args.cache_gib:g} GiB decoded-block "
                               f"cache; Poisson {args.serve_rate:g} requests/s, 2 s warm-up + {args.serve_seconds:g} s",
                   "request_lengths": "lognormal median 16 KiB, sigma 1, clipped to [4 KiB, 1 MiB]; uniform starts",
                   "closure": "byte-level (match index built in %.2f s)" % index_s, "setup_s": round(setup_s, 1),
                   "host_mem_gib": host_memory_gib()},
        "latency_us": {"p50": round(float(np.percentile(lat, 50)), 1), "p90": round(float(np.percentile(lat, 90)), 1),
                       "p99": round(float(np.percentile(lat, 99)), 1), "max": round(float(lat.max()), 1),
                       "mean": round(float(lat.mean()), 1)},
        "throughput": {"value": round(gbs, 3), "unit": "GB/s", "requests_per_s": round(lat.size / window, 1)},
        "closure_blocks": {"mean": round(float(np.mean(closure)), 1), "p50": float(np.percentile(closure, 50)),
                           "p99": float(np.percentile(closure, 99))},
        "decoded_blocks": {"mean": round(float(np.mean(dec_blocks)), 1),
                           "p50": float(np.percentile(dec_blocks, 50)), "p99": float(np.percentile(dec_blocks, 99))},
        "service_us": {"p50": round(float(np.percentile(served, 50)), 1),
                       "p99": round(float(np.percentile(served, 99)), 1), "fit": fit},
        "server": {"ticks": st_all["ticks"], "blocks_decoded": st_all["blocks_decoded"],
                   "blocks_hit": st_all["blocks_hit"],
                   "hit_rate": round(st_all["blocks_hit"] / max(1, st_all["blocks_hit"] + st_all["blocks_decoded"]), 4),
                   "refused": st_all["refused"], "streams": args.serve_streams,
                   "tick_overlaps": st_all["tick_overlaps"], "tick_waits": st_all["tick_waits"],
                   "host_ms_per_tick": round(st_all["tick_host_ms"] / max(1, st_all["ticks"]), 4),
                   "walk_ms_per_tick": round(st_all["walk_ms"] / max(1, st_all["ticks"]), 4),
                   "launch_ms_per_tick": round(st_all["launch_ms"] / max(1, st_all["ticks"]), 4)},
        "verified": f"{smp.size} sampled requests equal the generator's bytes",
        "clocks": clk,
    }
    srv.close()
    A.close()
    ctx.close()
    del arena, d_arc
    torch.cuda.empty_cache()
    return line


def init_dist(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    d = {"rank": rank, "world": world, "local": local, "pg": None}
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        d["pg"] = tdist
    return d


def run_depth(args):
    """Chain-depth statistics of the corpus as the library encoder parses it
    (paper, Depth Does Not Govern Latency): the per-block maximum depth, its
    median and tail, and the depth of the matches.  Host-only work."""
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    size, wname = workload(args)
    data = synth.corpus(args.corpus, size, 0)
    st = {}
    t = time.perf_counter()
    arc = acx.encode(data, no_rep=args.encoding == "no_rep", max_lanes=args.lanes, max_depth=args.max_depth,
                     stats=st)
    enc_s = time.perf_counter() - t
    bm = np.array(st["block_max_depth"], np.int64)
    md = np.array(st["match_depth"], np.int64)
    ml = np.array(st["match_level"], np.int64)
    lb = np.array(st["level_bytes"], np.int64)

    def rank(h, q):  # the element of rank floor(q * (count - 1)) of the sorted values
        c = np.cumsum(h)
        return int(np.searchsorted(c, int(q * (c[-1] - 1)), side="right"))

    line = {
        "metric": "chain depth", "workload": wname, "encoding": args.encoding,
        "max_depth": "none" if args.max_depth == 0xFFFFFFFF else (args.max_depth or 16),
        "ratio": round(size / len(arc), 4), "archive_bytes": len(arc), "blocks": st["blocks"],
        "matches": st["matches"], "encode_s": round(enc_s, 1),
        "block_max_depth": {"median": rank(bm, 0.5), "p90": rank(bm, 0.9), "p99": rank(bm, 0.99),
                            "max": int(np.nonzero(bm)[0].max()),
                            "blocks_with_matches": int(bm[1:].sum())},
        "match_depth": {"median": rank(md, 0.5), "p99": rank(md, 0.99), "max": int(np.nonzero(md)[0].max()),
                        "share_depth_1": round(float(md[1] / max(md.sum(), 1)), 4),
                        "mean": round(float((md * np.arange(256)).sum() / max(md.sum(), 1)), 3)},
        # cross-block levels: level 0 is finished by the local pass; a pass
        # taking the levels in order needs one round per level above 0
        "cross_block_level": {"max": int(np.nonzero(ml)[0].max()) if ml.any() else 0,
                              "matches": {str(l): int(ml[l]) for l in np.nonzero(ml)[0]},
                              "bytes": {str(l): int(lb[l]) for l in np.nonzero(lb)[0]}},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == "depth":
        run_depth(args)
        return
    if args.workload == "serve-encode":
        run_serve_encode(args)
        return
    dist = init_dist(args)
    if args.impl == "reference":
        run_reference(args, dist)
        if dist["pg"]:
            dist["pg"].barrier()
        return
    if args.workload == "batch":
        run_batch(args, dist)
        return
    if args.workload == "serve":
        if dist["rank"] == 0:
            run_serve(args, dist)
        return
    import torch

    import paper_2608_10188_gb300 as acx
    acx.build.build()
    dev = dist["local"]
    torch.cuda.set_device(dev)
    size, wname = workload(args)
    data, arc = get_archive(args, acx)
    world = dist["world"]
    # the comparisons of the default run (one GPU): their archives are encoded
    # on host threads while the headline is measured
    extras = (world == 1 and not args.no_extras and args.corpus == "dna" and not args.size
              and args.encoding == "history" and args.variant == "fast" and not args.shard)
    futs = start_extra_encodes(args, acx, data) if extras else None
    variant = {"plain": acx.lib.VARIANT_PLAIN, "fused": acx.lib.VARIANT_FUSED}.get(args.variant, acx.lib.VARIANT_FAST)
    ctx = acx.Context(dev, variant=variant, wait_ns=args.wait_ns)
    h_arc = np.frombuffer(arc, dtype=np.uint8).copy()
    d_arc = torch.from_numpy(h_arc).to(f"cuda:{dev}")
    A = acx.Archive(ctx, d_arc.data_ptr(), h_arc, h_arc.size)
    info = A.info
    out = torch.empty(size, dtype=torch.uint8, device=f"cuda:{dev}")
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    # --shard: this rank decodes its block-aligned range through the range's
    # byte-level closure (strong scaling); otherwise every rank decodes its
    # own replica of the whole archive (weak scaling)
    if args.shard:
        A.build_index()
        s0, ln = acx.shard_range(size, world, dist["rank"])

        def one(stats=False):
            return acx.decode_range(ctx, A, s0, ln, out.data_ptr() + s0, sh, stats=stats)
    else:
        s0, ln = 0, size

        def one(stats=False):
            return acx.decode_all(ctx, A, out.data_ptr(), size, sh, stats=stats)

    # correctness gate: the timed configuration must reproduce the input exactly
    rc = one()
    if rc != 0:
        raise RuntimeError(f"decode failed: {rc} {ctx.last_error()}")
    if not torch.equal(out[s0:s0 + ln], torch.from_numpy(data[s0:s0 + ln]).to(out.device)):
        raise RuntimeError("GPU decode differs from the input")

    for _ in range(args.warmup):
        flush.fill_(1)
        one()
    torch.cuda.synchronize()
    if dist["pg"]:
        dist["pg"].barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ms_total, ms_ans, ms_asm, ms_ext = [], [], [], []
    last_stats = {}
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)  # write 256 MiB > L2 between steps
        r, st = one(stats=True)
        if r != 0:
            raise RuntimeError(f"decode failed: {r} {ctx.last_error()}")
        ms_total.append(st["ms_total"])
        ms_ans.append(st["ms_ans"])
        ms_asm.append(st["ms_parse"])
        ms_ext.append(st["ms_copy"])
        last_stats = st
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist["pg"]:
        dist["pg"].barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    # the last timed decode's cross-block rounds: (round, list size, start µs)
    trace = ctx.round_trace() if not args.shard else None

    dev_ms = sum(ms_total)
    if dist["pg"]:
        t = torch.tensor([dev_ms], device=out.device, dtype=torch.float64)
        dist["pg"].all_reduce(t, op=dist["pg"].ReduceOp.MAX)
        dev_ms = float(t.item())
    value = (1 if args.shard else world) * size * args.steps / (dev_ms / 1e3) / 1e9
    ms_step = dev_ms / args.steps

    # roofline of the dominant kernel and of the whole path
    a_ms = statistics.mean(ms_ans)
    s_ms = statistics.mean(ms_asm)
    x_ms = statistics.mean(ms_ext)
    roof, path_roof = rooflines({"ans": a_ms, "local": s_ms, "cross": x_ms}, stream_bytes(arc), size, len(arc),
                                last_stats, info["n_blocks"], args.variant, ms_step,
                                wname if args.encoding == "history" and args.variant == "fast"
                                and not args.max_depth and args.lanes == 32 else "")

    # end to end through the C ABI from pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        h_in = torch.from_numpy(h_arc).pin_memory()
        h_out = torch.empty(size, dtype=torch.uint8).pin_memory()
        hin_np, hout_np = h_in.numpy(), h_out.numpy()
        for _ in range(2):
            acx.decode_host(ctx, A, hin_np, hout_np, sh)
        e_ms = []
        for _ in range(args.e2e_steps):
            r, st = acx.decode_host(ctx, A, hin_np, hout_np, sh, stats=True)
            if r != 0:
                raise RuntimeError(f"decode_host failed: {r} {ctx.last_error()}")
            e_ms.append(st["ms_total"])
        if not np.array_equal(hout_np, data):
            raise RuntimeError("decode_host output differs from the input")
        # the host link is shared with other jobs on the machine: a step can
        # stall on their traffic, so the value is the median step (the mean
        # and the spread are reported beside it)
        e_med, e_mean = statistics.median(e_ms), statistics.mean(e_ms)
        scale = (1 if args.shard else world) * size / 1e9
        e2e = {"value": round(scale / (e_med / 1e3), 3), "unit": "GB/s",
               "h2d_bytes_per_step": len(arc), "d2h_bytes_per_step": size, "steps": len(e_ms),
               "of": "median step", "mean_value": round(scale / (e_mean / 1e3), 3),
               "step_ms": {"median": round(e_med, 4), "min": round(min(e_ms), 4), "max": round(max(e_ms), 4)}}

    # parse statistics of the archive from the device's parse-only pass
    # (after the timed region): the repeat-coded share and the
    # dependency-free runs between repeat-coded tokens
    ps = A.parse_stats()
    n_rep = sum(ps["rep_matches"])
    parse = {"tokens": ps["tokens"], "repeat_coded": n_rep,
             "repeat_coded_share": round(n_rep / max(ps["tokens"], 1), 5),
             "multibyte_value_share": round(ps["multibyte_values"] / max(ps["values"], 1), 5),
             "runs": ps["runs"], "median_run": ps["median_run"],
             "mean_run": round(ps["run_len_sum"] / max(ps["runs"], 1), 2), "max_run": ps["max_run"],
             "external_matches": ps["external_matches"], "overlap_matches": ps["overlap_matches"]}

    cpu = None
    if dist["rank"] == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_baseline(arc, data)

    comps = None
    if extras:
        comps = comparison_extras(args, acx, torch, dev, flush, sh, data, arc, futs)

    if dist["rank"] == 0:
        line = {
            "metric": "device-resident decode GB/s", "value": round(value, 3), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic (seeded generator; stands in for chr1 hg38)",
            "config": {"workload": wname, "encoding": args.encoding, "variant": args.variant,
                       "levels": "level bodies, level-ordered cross-block rounds" if args.levels else "none",
                       "max_depth": args.max_depth or 16,
                       "rans_lanes": args.lanes, "block_size": 16384, "blocks": info["n_blocks"],
                       "tokens": info["tokens"], "archive_bytes": len(arc),
                       "ratio": round(size / len(arc), 4),
                       "l2": "256 MiB buffer written between steps; per-step CUDA events exclude it"},
            "step_ms": {"median": round(statistics.median(ms_total), 4), "min": round(min(ms_total), 4),
                        "max": round(max(ms_total), 4),
                        "spread": round((max(ms_total) - min(ms_total)) / statistics.median(ms_total), 4)},
            "stage_ms": {"ans": round(a_ms, 4), "local_parse_copy": round(s_ms, 4), "cross_block": round(x_ms, 4)},
            "cross_block_stats": {"pending_pieces": last_stats.get("pending_spans"),
                                  "pending_bytes": last_stats.get("pending_bytes"),
                                  "rounds_after_first": last_stats.get("wait_polls"),
                                  "round_trace": trace},
            "parse_stats": parse,
            "roofline": roof,
            "path_roofline": path_roof,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": (3 if args.variant == "fused" else 6 if args.levels and args.variant == "fast" else 4)
            * args.steps,
            "gpu_launches_note": "prologue, entropy stage, local pass, [level scan, level fill,] cross-block pass",
            "clocks": clk,
            "wall_s": round(wall, 3),
            "comparisons": comps,
        }
        print(json.dumps(line), flush=True)
    A.close()
    ctx.close()
    if dist["pg"]:
        dist["pg"].barrier()
        dist["pg"].destroy_process_group()


def kernel_source_key():
    """Hash of the files that make up the decode kernels and of the encoder
    that writes the measured archives: profiler counters taken on other
    kernels, or on other archives, do not describe these."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2608_10188_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")) or f in ("internal.h", "encode.cpp"):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# Counters from one-kernel ncu captures of the full-size workload, per launch,
# keyed by (kernel source key, workload, kernel): DRAM bytes read + written,
# and warp-instructions per decoded symbol of the entropy stage.  A key that
# does not match the running sources gives null: the counters were taken on
# other kernels.
_GENOME = "chr1-shaped synthetic genome 253,935,557 B"
CAPTURED_DRAM = {
    ("98fdae1c5dff3c38", _GENOME, "k_rans"): 93797632 + 227070208,
    ("98fdae1c5dff3c38", _GENOME, "k_local"): 223956992 + 246156288,
    ("98fdae1c5dff3c38", _GENOME, "k_external"): 140977664 + 39984640,
}
CAPTURED_RANS_INSTR_PER_SYMBOL = {
    ("98fdae1c5dff3c38", _GENOME): 195824333 / 221024708,
}
ISSUE_PEAK = 152 * 4 * 2.07e9  # warp-instructions per second: 4 schedulers x 152 SMs x 2070 MHz


def rooflines(stage, pb, size, arc_len, st, n_blocks, variant, ms_step, wname=""):
    """HBM roofline of the decode (the paper's "Memory Floor" accounting):
    the algorithmic bytes of one decode are the archive read
    plus the output written; `achieved` divides them by the CUDA-event time of
    the dominant (slowest) kernel of the step, `frac` by the measured HBM copy
    peak.  Each kernel's own traffic by design (the decoded streams it writes
    or reads, the pending pieces) is reported beside it, not as algorithmic."""
    peak, peak_kind = measured_peaks()
    src = kernel_source_key()
    pend_b = int(st.get("pending_bytes") or 0)
    pend_n = int(st.get("pending_spans") or 0)
    local = "k_plain" if variant == "plain" else "k_local"
    path_bytes = arc_len + size
    kern = {
        # payload read + decoded streams written
        "k_rans": (stage["ans"], pb["payload"] + pb["decoded"]),
        # decoded streams read + output written
        local: (stage["local"], pb["decoded"] + size),
    } if variant != "fused" else {
        # one kernel: payload read + output written (the streams stay on chip)
        "k_fused": (stage["local"], pb["payload"] + size),
    }
    kern.update({
        # source bytes read + destination bytes written + 16 B per piece record + 4 B count per block
        "k_external": (stage["cross"], 2 * pend_b + 16 * pend_n + 4 * n_blocks),
    })
    per = {}
    for k, (ms, b) in kern.items():
        per[k] = {"ms": round(ms, 4), "design_bytes": int(b),
                  "design_gbs": round(b / (ms / 1e3) / 1e9, 1) if ms > 0 else None,
                  "traffic": CAPTURED_DRAM.get((src, wname, k)), "traffic_source": "ncu one-kernel capture"}
    instr = CAPTURED_RANS_INSTR_PER_SYMBOL.get((src, wname))
    if instr and stage["ans"] > 0:
        rate = instr * pb["decoded"] / (stage["ans"] / 1e3)
        per["k_rans"]["alu"] = {"bound": "alu", "instr_per_symbol": round(instr, 4), "source": "ncu capture",
                                "achieved": round(rate / 1e12, 4), "peak": round(ISSUE_PEAK / 1e12, 4),
                                "unit": "T warp-instr/s", "frac": round(rate / ISSUE_PEAK, 4)}
    dom = max(kern, key=lambda k: kern[k][0])
    ms = kern[dom][0]
    achieved = path_bytes / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": CAPTURED_DRAM.get((src, wname, dom)),
            "peak_kind": peak_kind + " hbm_gbs", "algorithmic_bytes": int(path_bytes),
            "algorithmic": "archive bytes read + output bytes written (1 + 1/ratio per output byte)",
            "kernel_source": src, "kernels": per}
    path_gbs = path_bytes / (ms_step / 1e3) / 1e9
    path = {"bytes": path_bytes, "achieved": round(path_gbs, 1), "peak": peak, "frac": round(path_gbs / peak, 4),
            "frac_nominal_8tbs": round(path_gbs / 8000, 4)}
    return roof, path


def stream_bytes(arc: bytes) -> dict:
    """Payload bytes and decoded stream bytes of an archive (from its index
    and block descriptors)."""
    import struct
    nb = struct.unpack_from("<I", arc, 24)[0]
    off_idx = struct.unpack_from("<Q", arc, 40)[0]
    payload = 0
    decoded = 0
    for b in range(nb):
        poff, plen = struct.unpack_from("<QI", arc, off_idx + 40 * b)
        payload += plen
        for s in range(4):
            decoded += struct.unpack_from("<I", arc, poff + 12 * s)[0]
    return {"payload": payload, "decoded": decoded}



if __name__ == "__main__":
    main()
