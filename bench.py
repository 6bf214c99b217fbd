#!/usr/bin/env python3
"""Benchmark of the IBIP hot path on one GB300 (or N replicas).

One step = the whole path on one synthetic image held in HBM:
  squared EDT -> rank + invasion (sequence image, radius per step)
  -> trapping (outlet face) -> saturation / Pc curve -> morphological-opening
  drainage at 40 radii.
Workload (default): 512^3 anisotropic blobs (noise smoothed with sigma
(4, 8, 4) voxels, porosity 0.60, seed 3), inlet x=0, outlet x=511, voxel
5 um, sigma 0.072 N/m, theta 180 deg -- the largest single-image
configuration, standing in for the 250^3 60 %-porosity blobs of the paper's
Fig. 4.  --config spheres200 / blobs48 select the smaller images.  Results
are bit-exact with the CPU oracle (tests/).

value  = voxels per second through the whole path (device-resident inputs);
e2e    = the same through the public API with the image copied from pinned
         host memory and seq_out + Pc curve copied back inside the timing;
roofline = the dominant kernel class (the invasion: a latency-bound loop on
         one CTA, whose figure of merit is its step latency), with
         roofline.hbm_kernels giving every HBM-bound class (EDT, rank sort,
         widest path, trapped mask, Pc, opening dilation) as algorithmic
         bytes / live CUDA-event time / measured HBM copy bandwidth;
cpu_baseline = the plain C oracle on this host's cores (rank 0, N=1), on a
         bounded sample when a full pass would take minutes.

Multi-GPU: one process per GPU (torchrun), each an independent replica of
the same workload (the invasion is serial per image and does not shard);
no collective on the data path; value = total voxels / max time over ranks.

--impl reference runs the oracle as the reference arm on the same workload.
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
# hardware work queues for the server's streams (see ibip_server_create);
# must be set before the CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

L2_BYTES = 129 * 1024 * 1024
CLASS_NAMES = ["edt", "rank", "invade", "maximin", "trap", "pc", "dilate"]

# DRAM traffic per voxel and launch of each kernel class, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum summed over the class's
# kernels in one launch on the named workload, divided by its voxels; the
# profiles/ summary named in "capture" gives the command and the figures).
# "src" lists the sources the counters were taken on with the first 16 hex
# digits of their SHA-256: when one has changed since, or the line runs
# another workload, the class reports traffic null.
NCU_TRAFFIC = {
    "edt": {"bytes_per_voxel": 15.699, "src": {"paper_2101_03240_gb300/csrc/edt.cu": "1dad9f25dc064510"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "rank": {"bytes_per_voxel": 45.067, "src": {"paper_2101_03240_gb300/csrc/invade.cu": "0f50d49a6694434e", "paper_2101_03240_gb300/csrc/scan.cu": "7ae2dbb22ecb3ed4"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "maximin": {"bytes_per_voxel": 300.551, "src": {"paper_2101_03240_gb300/csrc/maximin.cu": "2a905a8c9742daf6"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "maximin_trim": {"bytes_per_voxel": 105.892, "src": {"paper_2101_03240_gb300/csrc/maximin.cu": "2a905a8c9742daf6"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "trap": {"bytes_per_voxel": 12.615, "src": {"paper_2101_03240_gb300/csrc/pc.cu": "eb392979ed4ea0da"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "pc": {"bytes_per_voxel": 4.631, "src": {"paper_2101_03240_gb300/csrc/pc.cu": "eb392979ed4ea0da", "paper_2101_03240_gb300/csrc/scan.cu": "7ae2dbb22ecb3ed4"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "dilate": {"bytes_per_voxel": 14.721, "src": {"paper_2101_03240_gb300/csrc/edt.cu": "1dad9f25dc064510"},
             "workload": "blobs512", "capture": "profiles/traffic_blobs512.md"},
    "invade": {"bytes_per_voxel": 38.414, "src": {"paper_2101_03240_gb300/csrc/invade.cu": "0f50d49a6694434e"},
               "workload": "blobs512", "capture": "profiles/k_invade_blobs512_traffic.md"},
}


def source_sha16(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_per_launch(cls, units, workload="blobs512"):
    """ncu DRAM bytes of one launch of class `cls` on `units` voxels of
    `workload`, or None when not captured on that workload or captured on
    sources that changed since."""
    t = NCU_TRAFFIC.get(cls)
    if not t or t.get("workload") != workload:
        return None
    try:
        if any(source_sha16(f) != h for f, h in t["src"].items()):
            return None
    except OSError:
        return None
    return t["bytes_per_voxel"] * units


def max_over_ranks(x, world, device):
    """The largest x over all ranks: a replica job takes as long as its
    slowest rank.  Works on any process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` independent replicas that each
    processed `units_per_rank` units, the slowest in `seconds`."""
    return world * units_per_rank / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["spheres200", "blobs48", "blobs512", "blobs256", "batch256", "serve"],
                    default="blobs512")
    ap.add_argument("--requests", type=int, default=600, help="serve: requests in the Poisson stream")
    ap.add_argument("--budget-gb", type=float, default=20.0,
                    help="serve: device arena of the server (20 GB: below the stream's peak demand, so admission binds)")
    ap.add_argument("--slots", type=int, default=16,
                    help="serve: worker slots (the stream keeps ~6 jobs in flight on average; 16 slots keep the "
                         "jobs' kernels from crowding each other's one-CTA invasions)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rule", choices=["frontier", "paper"], default="frontier",
                    help="invasion rule: the frontier rule, or Section 2.1 as printed (all ties, trunc radius)")
    ap.add_argument("--mio-levels", type=int, default=40)
    ap.add_argument("--autotune", action="store_true",
                    help="tune the EDT tile shapes on the first call of each shape class (before warm-up)")
    ap.add_argument("--no-extra", action="store_true",
                    help="single-image lines at N=1: skip the short batch256 and serve measurements added as "
                         "extra keys")
    return ap.parse_args()


def workload(name):
    from paper_2101_03240_gb300 import synth
    return {"spheres200": synth.c2_spheres200, "blobs48": synth.c1_blobs48,
            "blobs512": synth.c3_blobs512, "blobs256": synth.c3_blobs256}[name]()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        text = open(self.f.name).read()
        os.unlink(self.f.name)
        return parse_clock_samples(text)


def parse_clock_samples(text):
    """Median SM clock, the largest max clock and the throttle reasons seen
    in nvidia-smi CSV samples (fields as in Clocks.Q, no header or units);
    None when no sample parses."""
    rows = [l.split(",") for l in text.strip().splitlines() if l.strip()]
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        r = [x.strip() for x in r]
        try:
            sm.append(float(r[1]))
            mx = max(mx, float(r[2]))
        except (ValueError, IndexError):
            continue
        for n, v in zip(names, r[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- batched ----

def run_batch(args, rank, world):
    """256 uneven images (32^3..160^3, half blobs, half sphere packs), EDT +
    invasion + trapping + Pc each: images/s of the batched call, with the
    plain per-image calls on the same images for comparison."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2101_03240_gb300 import ibip, synth

    imgs_h = batch_images(256)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nimg = len(imgs_h)
    nvox_total = sum(a.size for a in imgs_h)
    imgs = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in imgs_h]
    ctx = ibip.Context(local)
    if args.autotune:
        ctx.set_autotune(True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    paper = args.rule == "paper"

    def batched(images=imgs):
        if paper:   # EDT + the paper-literal invasion, one thread-block cluster per image
            res, cs = ctx.invade_literal_batched(images, 0)
            batched.cluster = cs
            return res
        return ctx.invade_batched(images, 0, 1, trapping=True, curve=True)

    def single():
        out = []
        for im in imgs:
            d = ctx.edt(im)
            if paper:
                out.append(ctx.invade_literal(im, d, inlet=0)[4])
                continue
            s_, r2, cen, K, st = ctx.invade(im, d, inlet=0)
            tr, so = ctx.trapping(s_, 1)
            Sa, Pc, _ = ctx.pc_curve(so, r2)
            out.append(K)
        return out

    for _ in range(max(1, args.warmup)):
        batched()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local) if rank == 0 else None
    ctx.profile(True)
    l0 = ctx.launches
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = batched()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    launches = (ctx.launches - l0) // max(args.steps, 1)
    prof = {CLASS_NAMES[c]: ctx.profile_read(c) for c in range(len(CLASS_NAMES))}
    ctx.profile(False)
    ck = clocks.stop() if clocks else None
    ms_step = sum(ms) / len(ms)
    ms_step = max_over_ranks(ms_step, world, dev)
    # plain per-image path, one pass (same outputs)
    single()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ks = single()
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    assert Ks == [r["K"] for r in res]
    # end to end: host images in, seq_out out.  The caller keeps the batch
    # packed back to back in one pinned buffer, so one copy brings it in
    # (the device images are views of one buffer) and one copy takes the
    # packed sequence images back (gathered on the device first).
    offs = np.concatenate([[0], np.cumsum([a.size for a in imgs_h])]).astype(np.int64)
    pin_in = torch.from_numpy(np.concatenate([a.reshape(-1) for a in imgs_h])).pin_memory()
    pin_out = torch.empty(nvox_total, dtype=torch.int32).pin_memory()
    dev_in = torch.empty(nvox_total, dtype=torch.uint8, device=dev)
    views = [dev_in[int(offs[i]):int(offs[i + 1])].view(a.shape) for i, a in enumerate(imgs_h)]
    e2e_ms = []
    torch.cuda.synchronize()
    for _ in range(max(args.steps, 1)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dev_in.copy_(pin_in, non_blocking=True)
        res = batched(views)
        packed = torch.cat([(r["seq"] if paper else r["seq_out"]).reshape(-1) for r in res])
        pin_out.copy_(packed, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    if not np.array_equal(pin_out.numpy(), packed.cpu().numpy()):
        raise RuntimeError("batch e2e: the copied-back results differ from the device results")
    e2e_s = max_over_ranks(sum(e2e_ms) / len(e2e_ms) * 1e-3, world, dev)
    if rank != 0:
        return None
    tot = sum(v[0] for v in prof.values()) or 1.0
    kinfo = {c: {"ms_per_step": v[0] / args.steps, "share": v[0] / tot, "spans": v[1] // max(args.steps, 1)}
             for c, v in prof.items() if v[1]}
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    steps_total = sum(r["K"] for r in res)
    inv_ms = prof["invade"][0] / max(prof["invade"][1], 1)
    alg = 8 * nvox_total + 8 * steps_total
    achieved = alg / (inv_ms * 1e-3) / 1e9
    out = {
        "metric": ("batched images/s (EDT+paper-literal invasion per image on its own thread-block cluster, "
                   "bit-exact vs oracle)") if paper else
                  "batched images/s (EDT+rank+invasion+trapping+Pc per image, bit-exact vs oracle)",
        "value": job_rate(nimg, world, ms_step * 1e-3), "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "batch256_paper_rule" if paper else "batch256", "images": nimg, "voxels": nvox_total,
                   "edge": "32..160 log-uniform", "cluster_ctas_per_image": getattr(batched, "cluster", None),
                   "mix": "half blobs, half sphere packs", "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas%d" % world},
        "per_image_path_images_per_s": nimg / single_s,
        "batched_over_per_image": (nimg / (ms_step * 1e-3)) / (nimg / single_s),
        "invasion_steps": steps_total,
        "e2e": {"value": job_rate(nimg, world, e2e_s), "unit": "images/s", "h2d_bytes_per_step": int(nvox_total),
                "d2h_bytes_per_step": int(4 * nvox_total)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "invade (batched)", "achieved": round(achieved, 3), "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                     "peak_source": "measured" if pk else "fallback",
                     "note": "one latency-bound CTA per image; bytes are the algorithmic minimum"},
        "kernels": kinfo, "clocks": ck,
        "gpu": torch.cuda.get_device_name(dev), "host_cores": os.cpu_count(), "seed": 4,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        sample = imgs_h[:16]
        t0 = time.perf_counter()
        for a in sample:
            dd = O.edt(a)
            if paper:
                O.invade_literal(a, dd, 0)
                continue
            sq = O.invade(a, dd, inlet=0)
            so = O.trapping(sq[0], 1)[1]
            O.pc_curve(so, sq[1])
        t = time.perf_counter() - t0
        mean_vox = nvox_total / nimg
        out["cpu_baseline"] = {"value": sum(a.size for a in sample) / t / mean_vox, "unit": "images/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "the first 16 images of the batch, whole path each; images/s = their "
                                         "voxels/s / the batch's mean voxels per image"}
    return out


# -------------------------------------------------------------- serve ----

def _batch_image(i):
    from paper_2101_03240_gb300 import synth
    return synth.mixed_image(i, 4000, 32, 160)


def batch_images(n):
    """The 256-image batch (synth.c4_batch: image i is mixed_image(i) of the
    32^3..160^3 mix), generated by a spawn pool."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(n, os.cpu_count() or 1)) as pool:
        return pool.map(_batch_image, range(n))


def _request_image(j):
    from paper_2101_03240_gb300 import synth
    return synth.mixed_image(j, 5000, 64, 384)


def serve_images(which):
    """The request stream's images (image j is mixed_image(j) of the
    64^3..384^3 stream) for the request indices `which`, generated by a
    spawn pool before any GPU call."""
    import multiprocessing as mp
    which = list(which)
    if not which:
        return []
    with mp.get_context("spawn").Pool(min(len(which), os.cpu_count() or 1)) as pool:
        return pool.map(_request_image, which)


def serve_stream(srv, imgs, arrivals, keep=(), host=None, stage=None):
    """Submits imgs[i] at time arrivals[i] (seconds from now, ascending) and
    waits for all of them.  Results are dropped once seen complete (their
    device buffers freed), except those of the indices in `keep`.  With
    `host` (pinned host images), request i's image is first copied from
    host[i] into a fresh device buffer, and with `stage` (a pinned int32
    buffer) every result's seq_out is copied back into it when seen
    complete.  Returns (records, kept): per request (submit ns, end ns, K,
    status)."""
    import collections

    import torch
    t0 = time.monotonic()
    out = [None] * len(imgs)
    kept = {}
    pending = collections.deque()

    def collect(i, r):
        out[i] = (r["t_submit_ns"], r["t_end_ns"], r["K"], r["status"])
        if stage is not None:
            stage[:r["seq_out"].numel()].copy_(r["seq_out"].view(-1))
        if i in keep:
            kept[i] = r

    for i, (im, ta) in enumerate(zip(imgs, arrivals)):
        d = t0 + ta - time.monotonic()
        if d > 0:
            time.sleep(d)
        if host is not None:
            im = torch.empty(host[i].shape, dtype=torch.uint8, device=im.device)
            im.copy_(host[i], non_blocking=True)
        pending.append((i, srv.submit(im, inlet=0, outlet=1)))
        while pending:   # drop what has completed, in arrival order
            r = srv.poll(pending[0][1])
            if r is None:
                break
            collect(pending[0][0], r)
            pending.popleft()
    for i, t in pending:
        collect(i, srv.wait(t))
    return out, kept


def run_serve(args, rank, world):
    """Poisson request stream (20 requests/s, 64^3..384^3, half blobs, half
    sphere packs; 600 requests by default), each request EDT + invasion +
    trapping + Pc, through the continuous-batching server.  One timed step
    is the whole stream: every request submitted at its arrival time;
    value = requests / (last completion - first arrival), and p50/p99 of
    (completion - arrival) over all requests.  Under torchrun the stream is
    split over the ranks by ibip.route_requests (fewest routed voxels, the
    same split computed on every rank, no messages)."""
    import numpy as np
    from paper_2101_03240_gb300 import synth
    reqs = synth.c5_requests(n=args.requests)
    n_all = len(reqs)
    from paper_2101_03240_gb300 import ibip
    assign = ibip.route_requests([L ** 3 for _, L, _ in reqs], world) if world > 1 else [0] * n_all
    mine = [j for j in range(n_all) if assign[j] == rank]
    imgs_h = serve_images(mine)
    import torch
    import torch.distributed as dist

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nvox_mine = sum(a.size for a in imgs_h)
    imgs = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in imgs_h]
    arrivals = [reqs[j][0] for j in mine]
    ctx = ibip.Context(local)
    if args.autotune:
        ctx.set_autotune(True)
    budget = int(args.budget_gb * (1 << 30))
    srv = ibip.Server(ctx, budget, max_slots=args.slots)
    torch.cuda.synchronize()
    sample = list(range(min(8, len(imgs))))   # kept for the bit-exactness check

    for _ in range(max(1, args.warmup)):
        serve_stream(srv, imgs[:8], [0.0] * min(8, len(imgs)))
    if world > 1:
        dist.barrier()
    clocks = Clocks(local) if rank == 0 else None
    l0 = srv.stats()["launches"]
    spans, recs, kept = [], None, None
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        recs, kept = serve_stream(srv, imgs, arrivals, keep=set(sample))
        spans.append((max(r[1] for r in recs) - min(r[0] for r in recs)) * 1e-9)
    ck = clocks.stop() if clocks else None
    st = srv.stats()
    launches = (st["launches"] - l0) // max(args.steps, 1)
    assert all(r[3] == 0 for r in recs)
    span = max(spans)
    # end to end through the same stream: every request's image copied in
    # from pinned host memory at its arrival time, its seq_out copied back
    # to pinned host memory when it completes
    pins = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in imgs_h]
    stage = torch.empty(max(a.size for a in imgs_h), dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    erecs, _ = serve_stream(srv, imgs, arrivals, host=pins, stage=stage)
    e2e_s = (max(r[1] for r in erecs) - min(r[0] for r in erecs)) * 1e-9
    del pins
    srv.close()
    # bit-exactness of served results against the one-image calls (sample)
    alone_s, exact = [], 0
    for i in sample:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dd = ctx.edt(imgs[i])
        s_, r2, cen, K, st_ = ctx.invade(imgs[i], dd, inlet=0)
        tr, so = ctx.trapping(s_, 1)
        S_, P_, _ = ctx.pc_curve(so, r2)
        torch.cuda.synchronize()
        alone_s.append(time.perf_counter() - t1)
        r = kept[i]
        exact += int(K == r["K"] and torch.equal(s_, r["seq"]) and torch.equal(so, r["seq_out"]) and
                     torch.equal(tr, r["trapped"]) and torch.equal(P_, r["Pc"]) and torch.equal(S_, r["S"]))
    # gather every rank's records
    if world > 1:
        allrec = [None] * world
        dist.all_gather_object(allrec, recs)
        recs_all = [r for part in allrec for r in part]
        span = max_over_ranks(span, world, dev)
        e2e_s = max_over_ranks(e2e_s, world, dev)
    else:
        recs_all = recs
    if rank != 0:
        return None
    lat_all = np.array([(r[1] - r[0]) * 1e-6 for r in recs_all])
    n = len(recs_all)
    out = {
        "metric": "served images/s and p50/p99 latency (EDT+rank+invasion+trapping+Pc per request, bit-exact)",
        "value": n / span, "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": span * 1e3, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serve", "requests": n_all, "rate_per_s": 20.0,
                   "edge": "64..384 log-uniform", "mix": "half blobs, half sphere packs",
                   "budget_bytes": budget, "slots": args.slots,
                   "l2": "inputs larger than L2 (whole stream resident)", "parallelism": "replicas%d" % world,
                   "routing": "least routed voxels per rank" if world > 1 else None,
                   "timing": "host clock: one step = the whole Poisson stream, first arrival to last completion"},
        "latency_ms": {"p50": float(np.percentile(lat_all, 50)), "p99": float(np.percentile(lat_all, 99)),
                       "max": float(lat_all.max()), "mean": float(lat_all.mean())},
        "offered_images_per_s": n_all / reqs[-1][0],
        "server": st,
        "bit_exact_sample": "%d of %d served results equal the one-image calls" % (exact, len(sample)),
        "sample_alone_s": alone_s,
        "invasion_steps": int(sum(r[2] for r in recs_all)),
        "e2e": {"value": n / e2e_s, "unit": "images/s",
                "h2d_bytes_per_step": int(nvox_mine), "d2h_bytes_per_step": int(4 * nvox_mine),
                "note": "the same stream with each image copied in from pinned host memory at its arrival "
                        "and its seq_out copied back when complete (per rank's share)"},
        "gpu_launches": int(launches),
        "clocks": ck,
        "gpu": torch.cuda.get_device_name(dev), "host_cores": os.cpu_count(), "seed": 5,
    }
    assert exact == len(sample), out["bit_exact_sample"]
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        small = sorted(imgs_h, key=lambda a: a.size)[:4]
        t = time.perf_counter()
        for a in small:
            dd = O.edt(a)
            sq = O.invade(a, dd, inlet=0)
            so = O.trapping(sq[0], 1)[1]
            O.pc_curve(so, sq[1])
        t = time.perf_counter() - t
        mean_vox = sum(L ** 3 for _, L, _ in reqs) / n_all
        out["cpu_baseline"] = {"value": sum(a.size for a in small) / t / mean_vox, "unit": "images/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "the 4 smallest request images, whole path each; images/s = their "
                                         "voxels/s / the stream's mean voxels per image"}
    return out


# --------------------------------------------------------------- ours ----

R2_CLASSES = [("r=1", 1, 1), ("1<r<=2", 2, 4), ("2<r<=4", 5, 16), ("4<r<=8", 17, 64), ("r>8", 65, 1 << 62)]


def step_time_stats(rec, r2, K, span_cycles, span_ns):
    """Device time per invasion step, p50/p99 per radius class.  `rec` holds
    one row per batch (first step, steps, SM cycles, loop); each step of a
    batch is charged the batch's cycles over its steps, and cycles become
    microseconds by the kernel's own cycles-per-nanosecond ratio."""
    import numpy as np
    rec = np.asarray(rec, dtype=np.int64)
    rec = rec.reshape(len(rec), -1)[:, :4] if len(rec) else rec.reshape(0, 4)
    first, n, cyc = rec[:, 0], rec[:, 1], rec[:, 2]
    if len(rec) == 0 or int(n.sum()) != K or first[0] != 0 or np.any(first[1:] != np.cumsum(n)[:-1]):
        return None   # batches must tile steps 0..K-1 in order
    mhz = span_cycles / max(span_ns, 1) * 1e3
    us = np.repeat(cyc / np.maximum(n, 1) / mhz, n)
    r2 = np.asarray(r2[:K], dtype=np.int64)

    def pct(x):
        return {"steps": int(len(x)), "p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                "mean_us": float(x.mean())} if len(x) else {"steps": 0}

    classes = {name: pct(us[(r2 >= lo) & (r2 <= hi)]) for name, lo, hi in R2_CLASSES}
    busy = cyc.sum() / mhz
    return {"sm_mhz_in_kernel": mhz, "batches": int(len(rec)),
            "batches_single_voxel_loop": int((rec[:, 3] == 1).sum()),
            "batch_us": {"p50": float(np.percentile(cyc / mhz, 50)), "p99": float(np.percentile(cyc / mhz, 99))},
            "all": pct(us), "by_radius": classes,
            "traced_fraction_of_kernel": float(busy / (span_ns * 1e-3)) if span_ns else None,
            "note": "amortised: a batch's device time over the steps it committed, from one untimed "
                    "traced invasion (ibip_invade_trace)"}


def invasion_step_times(ctx, img_d, w):
    import torch
    d = ctx.edt(img_d)
    npore = int((img_d > 0).sum().item())
    buf = torch.zeros((npore + 1, 8), dtype=torch.int32, device=img_d.device)
    ctx.invade_trace(buf)
    try:
        _, r2, _, K, _ = ctx.invade(img_d, d, inlet=w.inlet)
    finally:
        ctx.invade_trace(None)
    s = ctx.invade_stats()
    nrec = min(s["trace_batches"], buf.shape[0])
    return step_time_stats(buf[:nrec].cpu().numpy(), r2.cpu().numpy(), K, s["span_cycles"], s["span_ns"])


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2101_03240_gb300 import ibip, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.config)
    img_h = np.ascontiguousarray(w.image)
    N = img_h.size
    ctx = ibip.Context(local)
    if args.autotune:
        ctx.set_autotune(True)
    img_d = torch.from_numpy(img_h).to(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    # opening radii: a workload parameter fixed once per image (A9 levels)
    d0 = ctx.edt(img_d)
    maxd = int(d0[img_d.bool()].max().item()) if bool(img_d.any()) else 1
    levels = synth.mio_levels(maxd, args.mio_levels)

    seq = torch.empty(img_d.shape, dtype=torch.int32, device=dev)
    r2 = torch.empty(N, dtype=torch.int32, device=dev)
    cen = torch.empty(N, dtype=torch.int32, device=dev)
    dt2 = torch.empty(img_d.shape, dtype=torch.int32, device=dev)

    # The opening needs only the image and dt2, not the invasion, whose one
    # CTA leaves the other SMs idle for most of the step: it runs on a second
    # context (shared-device mode: no cooperative grid beside the running
    # invasion) on a low-priority stream, driven from a worker thread while
    # this thread waits on the invasion; the rest of the path runs on a
    # high-priority stream.  The opening is joined as soon as the invasion
    # returns, so trapping's cooperative grid never starts beside it.
    from concurrent.futures import ThreadPoolExecutor
    ctx_open = ibip.Context(local)
    ctx_open.set_shared_device(True)
    if args.autotune:
        ctx_open.set_autotune(True)
    main_stream = torch.cuda.Stream(device=dev, priority=-1)
    open_stream = torch.cuda.Stream(device=dev, priority=0)
    pool = ThreadPoolExecutor(1, initializer=torch.cuda.set_device, initargs=(local,))

    def opening(image, d, ready):
        open_stream.wait_event(ready)
        with torch.cuda.stream(open_stream):
            lev, cnt = ctx_open.morph_drainage(image, d, levels, inlet=w.inlet)
            done = torch.cuda.Event()
            done.record()
        return lev, cnt, done

    eq = [None, None, None]

    def step(image, copy_back=None):
        """One pass of the whole path on the current stream, the opening
        beside it; copy_back(src, which) (the end-to-end run) is called for
        seq_out and for the Pc curve as soon as each exists."""
        d = ctx.edt(image, out=dt2)
        ready = torch.cuda.Event()
        ready.record()
        fut = pool.submit(opening, image, d, ready)
        try:
            if args.rule == "paper":
                s, _, rr, _, K, st = ctx.invade_literal(image, d, inlet=w.inlet)
            else:
                s, rr, cc, K, st = ctx.invade(image, d, inlet=w.inlet, seq=seq, step_r2=r2, step_centre=cen)
        finally:
            lev, cnt, done = fut.result()
        torch.cuda.current_stream().wait_event(done)
        so = ctx.trapping(s, w.outlet)[1] if w.outlet is not None else s
        if copy_back:
            copy_back(so, "seq")
        S, P, _ = ctx.pc_curve(so, rr, w.voxel_m, w.sigma, w.theta_deg)
        if copy_back:
            copy_back(P, "pc")
        eq[:] = ctx.equal_saturation(s, lev, K, len(levels))   # Section 3.1.1 check, by counts
        return K, so, S, P

    with torch.cuda.stream(main_stream):
        for _ in range(args.warmup):
            K, *_ = step(img_d)
    torch.cuda.synchronize()

    # ---- device-resident timing
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    ctx.profile(True)
    ctx_open.profile(True)
    l0, l1 = ctx.launches, ctx_open.launches
    t_wall = time.perf_counter()
    with torch.cuda.stream(main_stream):
        for i in range(args.steps):
            flush.zero_()                       # evict L2 between steps (untimed)
            ev[i][0].record()
            K, *_ = step(img_d)
            ev[i][1].record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = (ctx.launches - l0 + ctx_open.launches - l1) // max(args.steps, 1)
    prof, prof_open = {}, {}
    for c in range(len(CLASS_NAMES)):
        (m0, n0), (m1, n1) = ctx.profile_read(c), ctx_open.profile_read(c)
        prof[CLASS_NAMES[c]] = (m0 + m1, n0 + n1)
        prof_open[CLASS_NAMES[c]] = (m1, n1)
    # the widest path runs twice: trapping on the critical path (one
    # cooperative grid) and the opening's trim beside the invasion
    mm_trap = (prof["maximin"][0] - prof_open["maximin"][0], prof["maximin"][1] - prof_open["maximin"][1])
    ctx.profile(False)
    ctx_open.profile(False)
    ck = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = sum(ms) / len(ms)
    ms_step = max_over_ranks(ms_step, world, dev)
    if world > 1:
        dist.barrier()

    # ---- end to end through the public API (host image in, seq_out + Pc out).
    # seq_out is final once trapping returns and the Pc curve once it is
    # computed: each is copied back on a side stream as soon as it exists,
    # overlapping the work that follows (a copy issued after a long
    # device-only phase pays a start-up cost of ~20 ms at 512^3 when it is
    # not overlapped).  The step ends when both copies have landed.
    img_pin = torch.from_numpy(img_h).pin_memory()
    out_seq = torch.empty(img_d.shape, dtype=torch.int32).pin_memory()
    out_pc = torch.empty(N, dtype=torch.float32).pin_memory()
    image_dev = torch.empty_like(img_d)
    copy_stream = torch.cuda.Stream(device=dev)

    def copy_back(src, which):
        ready = torch.cuda.Event()
        ready.record()
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            (out_seq if which == "seq" else out_pc[:src.numel()]).copy_(src, non_blocking=True)

    e2e_ms = []
    torch.cuda.synchronize()
    with torch.cuda.stream(main_stream):
        for i in range(max(args.steps, 1)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            image_dev.copy_(img_pin, non_blocking=True)
            K2, so, S, P = step(image_dev, copy_back)
            torch.cuda.current_stream().wait_stream(copy_stream)
            b.record()
            torch.cuda.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    pool.shutdown()
    if not (np.array_equal(out_seq.numpy(), so.cpu().numpy()) and
            np.array_equal(out_pc[:K2].numpy(), P.cpu().numpy())):
        raise RuntimeError("e2e: the copied-back results differ from the device results")
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    e2e_step = max_over_ranks(e2e_step, world, dev)

    # ---- trapped wetting phase, invasion vs opening (Figure 9), once, untimed
    trap_cmp = None
    if w.outlet is not None:
        d_ = ctx.edt(img_d)
        if args.rule == "paper":
            s_ = ctx.invade_literal(img_d, d_, inlet=w.inlet)[0]
        else:
            s_ = ctx.invade(img_d, d_, inlet=w.inlet)[0]
        lev_, _ = ctx.morph_drainage(img_d, d_, levels, inlet=w.inlet)
        npore_ = int((img_d > 0).sum().item())
        t_ibip = int(ctx.trapping(s_, w.outlet)[0].sum().item())
        t_mio = int(ctx.trapping(lev_, w.outlet)[0].sum().item())
        trap_cmp = {"trapped_frac_invasion": t_ibip / npore_, "trapped_frac_opening": t_mio / npore_,
                    "note": "pore voxels trapped (defending phase cut from the outlet) after the invasion and "
                            "after the opening's last level, the opening's levels read as a sequence"}

    # ---- Section 3.1.1 / Fig. 8 and the Pc envelope (Sections 2.2.2, 3.1.1),
    # once, untimed: each invasion rule against the opening with its own
    # structuring element, by integer counts over all pore voxels
    rules_vs_opening = None
    if w.outlet is not None:
        npore_ = int((img_d > 0).sum().item())
        d_ = ctx.edt(img_d)
        s_f, r2_f, _, K_f, _ = ctx.invade(img_d, d_, inlet=w.inlet)
        s_p, _, r2_p, _, K_p, _ = ctx.invade_literal(img_d, d_, inlet=w.inlet)
        lev_o, cnt_o = ctx.morph_drainage(img_d, d_, levels, inlet=w.inlet)
        Te, Td = synth.integer_radius_levels(maxd)
        lev_m, cnt_m = ctx.morph_drainage(img_d, d_, Te, inlet=w.inlet, dilate_levels=Td)

        def compare(seq_, r2_, K_, lev_, cnt_, T_):
            _, diff, _ = ctx.equal_saturation(seq_, lev_, K_, len(T_))
            _, n_env = ctx.pc_envelope(seq_, r2_, T_)
            env = [abs(a - b) for a, b in zip(n_env, cnt_)]
            return {"levels": len(T_), "equal_saturation_max": max(diff) / npore_,
                    "equal_saturation_mean": sum(diff) / len(diff) / npore_,
                    "envelope_max": max(env) / npore_, "envelope_mean": sum(env) / len(env) / npore_}

        rules_vs_opening = {
            "frontier_rule_vs_opening": compare(s_f, r2_f, K_f, lev_o, cnt_o, levels),
            "paper_rule_vs_closed_ball_opening": compare(s_p, r2_p, K_p, lev_m, cnt_m, Te),
            "paper_rule_vs_opening": compare(s_p, r2_p, K_p, lev_o, cnt_o, levels),
            "frontier_rule_vs_closed_ball_opening": compare(s_f, r2_f, K_f, lev_m, cnt_m, Te),
            "note": "fractions of the pore voxels: equal_saturation = voxels in exactly one of the opening's set "
                    "and the invasion's set of the same count; envelope = |voxels invaded before the running "
                    "minimum sphere drops below the level - the opening's count at that level|.  The opening "
                    "erodes at T and dilates by d^2 < T at the A9 radii; the closed-ball opening erodes at R^2 "
                    "and dilates by d^2 <= R^2 at every integer R, the sphere of the paper-literal rule"}

    # ---- time per invasion step by radius class, once, untimed
    step_times = invasion_step_times(ctx, img_d, w) if args.rule == "frontier" else None

    if rank != 0:
        return None

    # ---- roofline of the dominant kernel class, and of every HBM-bound one
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    tot = sum(v[0] for v in prof.values()) or 1.0
    dom = max(prof, key=lambda c: prof[c][0])
    npore = int(img_h.astype(bool).sum())
    # algorithmic bytes per launch (one profiled span) of each class: the
    # minimum each must move
    alg = {
        "edt": 5 * N,                                   # read image, write dt2
        "invade": 8 * N + 8 * K,                        # read dt2, write seq, r2+centre per step
        "rank": 4 * N + 4 * N + 8 * npore,              # read dt2, write rank, write (idx, dt2) by rank
        "maximin": 8 * N,                               # read values, write widest-path field
        "trap": 4 * N + 4 * N + 1 * N + 4 * N,          # read seq, M; write mask, seq_out
        "pc": 4 * N + 12 * K,                           # histogram of seq; S, Pc, r2 per step
        "dilate": (4 + 4 + 4) * N,                      # per level: read W, read/write level
    }
    kinfo = {}
    for c, (tms, spans) in prof.items():
        if spans == 0:
            continue
        per = tms / spans
        kinfo[c] = {"ms_per_step": tms / args.steps, "share": tms / tot, "spans": spans // args.steps,
                    "ms_per_span": per, "algorithmic_GBps": alg[c] / (per * 1e-3) / 1e9}
    hbm_kernels = {}
    spans_of = {c: prof[c] for c in ("edt", "rank", "trap", "pc", "dilate")}
    spans_of["maximin"] = mm_trap
    spans_of["maximin_trim"] = prof_open["maximin"]
    alg["maximin_trim"] = alg["maximin"]
    for c in ("edt", "rank", "maximin", "maximin_trim", "trap", "pc", "dilate"):
        tms, spans = spans_of[c]
        if spans == 0:
            continue
        per = tms / spans
        ach = alg[c] / (per * 1e-3) / 1e9
        hbm_kernels[c] = {"bound": "hbm", "achieved": round(ach, 3), "peak": hbm_peak, "unit": "GB/s",
                          "frac": ach / hbm_peak, "traffic": traffic_per_launch(c, N, w.name),
                          "algorithmic_bytes_per_launch": int(alg[c]),
                          "ms_per_launch": per, "launches_per_step": spans // max(args.steps, 1)}
    hbm_kernels["maximin"]["note"] = "trapping's widest path: one cooperative grid on the critical path"
    if "maximin_trim" in hbm_kernels:
        hbm_kernels["maximin_trim"]["note"] = ("the opening's trim: the same propagation in shared-device mode "
                                               "(one launch per round), overlapped with the invasion")
    per_launch = prof[dom][0] / max(prof[dom][1], 1)
    achieved = alg[dom] / (per_launch * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 3), "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic_per_launch(dom, N, w.name),
                "peak_source": "measured" if pk else "fallback",
                "note": "the invasion is a serial, latency-bound loop on one CTA: achieved counts its "
                        "algorithmic bytes (dt2 read + seq write + step arrays), traffic is ncu's DRAM bytes per "
                        "launch (lines re-read between overlapping balls); its figure of merit is the step "
                        "latency (invasion_step_times, invasion_us_per_step); hbm_kernels holds the HBM-bound "
                        "classes against the measured copy bandwidth",
                "hbm_kernels": hbm_kernels}
    us_per_step = prof["invade"][0] / max(args.steps, 1) * 1e3 / max(K, 1)

    value = job_rate(N, world, ms_step * 1e-3)
    out = {
        "metric": "invasion voxels/s (EDT+rank+invasion+trapping+Pc+opening, bit-exact vs oracle)",
        "value": value,
        "unit": "voxels/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": w.name if args.rule == "frontier" else w.name + "_paper_rule",
                   "shape": list(img_h.shape), "porosity": float(npore / N),
                   "inlet": "x0", "outlet": "x1" if w.outlet is not None else None, "mio_levels": len(levels),
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas%d" % world,
                   "edt_tiles": list(ctx.edt_tiles(img_h.shape)), "autotune": bool(args.autotune)},
        "invasion_steps": K,
        "equal_saturation": {"levels": len(levels), "max_diff_frac": max(eq[1]) / npore,
                             "mean_diff_frac": sum(eq[1]) / len(eq[1]) / npore,
                             "note": "voxels in exactly one of the opening's level set and the invasion's "
                                     "matched-count set, over all pore voxels (Section 3.1.1)"},
        "trapping_vs_opening": trap_cmp,
        "rules_vs_opening": rules_vs_opening,
        "invasion_steps_per_s": K / (prof["invade"][0] / args.steps * 1e-3) if prof["invade"][1] else None,
        "invasion_us_per_step": us_per_step,
        "invasion_step_times": step_times,
        "e2e": {"value": job_rate(N, world, e2e_step * 1e-3), "unit": "voxels/s",
                "h2d_bytes_per_step": int(img_h.nbytes),
                "d2h_bytes_per_step": int(out_seq.numel() * 4 + K * 4)},
        "step_ms": {"min": min(ms), "median": sorted(ms)[len(ms) // 2], "max": max(ms)},
        "e2e_step_ms": {"min": min(e2e_ms), "median": sorted(e2e_ms)[len(e2e_ms) // 2], "max": max(e2e_ms)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernels": kinfo,
        "clocks": ck,
        "wall_s_timed": t_wall,
        "gpu": torch.cuda.get_device_name(dev),
        "host_cores": os.cpu_count(),
        "seed": {"spheres200": 2, "blobs48": 1, "blobs512": 3, "blobs256": 3}.get(w.name),
        "paper_context": "about 5 steps/s for the first 3,000 steps of a 250^3 blob image on a laptop CPU "
                         "(Python/SciPy, Fig. 4 caption); context, not a target",
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, w, args.mio_levels)
    return out


# ------------------------------------------------------------ oracle ----

def oracle_pass(w, levels, rule="frontier"):
    import oracle as O
    d = O.edt(w.image)
    if rule == "paper":
        seq, _, r2, _, st, K = O.invade_literal(w.image, d, inlet=w.inlet)
    else:
        seq, r2, cen, st, K = O.invade(w.image, d, inlet=w.inlet)
    so = O.trapping(seq, w.outlet)[1] if w.outlet is not None else seq
    O.pc_curve(so, r2, w.voxel_m, w.sigma, w.theta_deg)
    O.morph_drainage(w.image, d, levels, inlet=w.inlet)
    return K


# a full oracle pass over more voxels than this takes minutes: time a cube
# cut from the image's corner instead (same generator, same statistics)
ORACLE_FULL_MAX_VOXELS = 32 * 1024 * 1024
ORACLE_CROP_EDGE = 128


def oracle_sample(w, n_levels):
    """(workload, opening radii, description) of the oracle's timed sample:
    the whole image when small enough, else its corner cube [0, 128)^3 with
    the same faces; the radii (A9) come from the sample's own largest
    squared distance."""
    import numpy as np

    import oracle as O
    from paper_2101_03240_gb300 import synth
    if w.image.size <= ORACLE_FULL_MAX_VOXELS:
        img, name, desc = w.image, w.name, "one full pass of the %s workload" % w.name
    else:
        e = ORACLE_CROP_EDGE
        img = np.ascontiguousarray(w.image[:e, :e, :e])
        name = "%s_corner%d" % (w.name, e)
        desc = ("one pass over the corner cube [0,%d)^3 of the %s image (%d voxels, its own opening radii); "
                "a full pass over all %d voxels takes minutes" % (e, w.name, img.size, w.image.size))
    sw = synth.Workload(name, img, w.inlet, w.outlet, w.mio_levels, w.voxel_m, w.sigma, w.theta_deg)
    d = O.edt(img)
    maxd = int(d[img > 0].max()) if img.any() else 1
    return sw, synth.mio_levels(maxd, n_levels), desc


def cpu_baseline(args, w, mio_levels):
    """The oracle as it stands on the host cores: passes over the bounded
    sample until at least 10 s of work (at least one pass)."""
    sw, levels, desc = oracle_sample(w, mio_levels)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle_pass(sw, levels, args.rule)
        n += 1
        t = time.perf_counter() - t0
        if t >= 10.0:
            break
    return {"value": sw.image.size * n / t, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%s, %d time(s) (EDT-sep, %s, trap-UF, Pc, opening by EDT at %d radii); the invasion and "
                      "trap-UF are single-threaded, the EDT passes use OpenMP on all cores"
                      % (desc, n, "literal-queue" if args.rule == "paper" else "invade-heap", len(levels)),
            "seconds": t}


def run_reference_images(args, world):
    """The oracle on a bounded sample of the batch / request-stream images:
    whole path per image (EDT, invasion, trapping, Pc), images/s."""
    import oracle as O
    from paper_2101_03240_gb300 import synth
    if args.config == "batch256":
        imgs = [synth.mixed_image(i, 4000, 32, 160) for i in range(8)]
        mean_vox = sum(synth.mixed_edge(i, 4000, 32, 160) ** 3 for i in range(256)) / 256
        sample = "the first 8 images of the 256-image batch, whole path each"
        cfg = {"workload": "batch256", "images": 256, "edge": "32..160 log-uniform",
               "mix": "half blobs, half sphere packs"}
        metric = "batched images/s (EDT+rank+invasion+trapping+Pc per image, bit-exact vs oracle)"
    else:
        reqs = synth.c5_requests(n=args.requests)
        small = sorted(range(min(32, len(reqs))), key=lambda j: reqs[j][1])[:4]
        imgs = [synth.mixed_image(j, 5000, 64, 384) for j in small]
        mean_vox = sum(r[1] ** 3 for r in reqs) / len(reqs)
        sample = "the 4 smallest of the first 32 requests, whole path each"
        cfg = {"workload": "serve", "requests": len(reqs), "rate_per_s": 20.0, "edge": "64..384 log-uniform",
               "mix": "half blobs, half sphere packs"}
        metric = "served images/s and p50/p99 latency (EDT+rank+invasion+trapping+Pc per request, bit-exact)"

    def one_pass():
        for a in imgs:
            d = O.edt(a)
            sq = O.invade(a, d, inlet=0)
            so = O.trapping(sq[0], 1)[1]
            O.pc_curve(so, sq[1])

    for _ in range(args.warmup):
        one_pass()
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        one_pass()
        ts.append(time.perf_counter() - t)
    s = sum(ts) / len(ts)
    # the sample's voxel rate scaled to the workload's mean image size
    v = sum(a.size for a in imgs) / s / mean_vox
    sample += "; images/s = the sample's voxels/s / the workload's mean voxels per image (%.0f)" % mean_vox
    return {"impl": "reference", "metric": metric, "value": v, "unit": "images/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "images/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if args.config in ("batch256", "serve"):
        return run_reference_images(args, world)
    w = workload(args.config)
    sw, levels, desc = oracle_sample(w, args.mio_levels)
    for _ in range(args.warmup):
        oracle_pass(sw, levels, args.rule)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        K = oracle_pass(sw, levels, args.rule)
        ts.append(time.perf_counter() - t)
    s = sum(ts) / len(ts)
    v = sw.image.size / s
    return {"impl": "reference", "metric": "invasion voxels/s (EDT+rank+invasion+trapping+Pc+opening, "
            "bit-exact vs oracle)", "value": v, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w.name if args.rule == "frontier" else w.name + "_paper_rule",
                       "shape": list(w.image.shape), "mio_levels": len(levels),
                       "sample_shape": list(sw.image.shape)},
            "invasion_steps": K,
            "cpu_baseline": {"value": v, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc + " per step"},
            "e2e": {"value": v, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def extra_lines(args):
    """The batched and served forms, measured briefly in the same run as the
    single-image line (same process, after it): batch256 (3 timed batches
    after 2 warm-up ones) and the first 200 requests of the Poisson stream
    (one pass), each without its CPU baseline.  Their own lines
    (--config batch256 | serve) give the full measurements."""
    import gc

    import torch
    gc.collect()
    torch.cuda.empty_cache()
    ab = argparse.Namespace(**vars(args))
    ab.steps, ab.warmup, ab.no_cpu_baseline, ab.rule = 3, 2, True, "frontier"
    b = run_batch(ab, 0, 1)
    gc.collect()
    torch.cuda.empty_cache()
    sv = argparse.Namespace(**vars(args))
    sv.steps, sv.warmup, sv.no_cpu_baseline, sv.requests = 1, 1, True, 200
    s = run_serve(sv, 0, 1)
    keep_b = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "per_image_path_images_per_s",
              "batched_over_per_image", "e2e", "gpu_launches", "clocks", "config")
    keep_s = ("metric", "value", "unit", "ms_per_step", "latency_ms", "offered_images_per_s", "bit_exact_sample",
              "e2e", "gpu_launches", "clocks", "config")
    return {"batch256": {k: b[k] for k in keep_b if k in b}, "serve": {k: s[k] for k in keep_s if k in s}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        import torch.distributed as dist
        if world > 1:
            dist.init_process_group("nccl")
        import __graft_entry__
        if rank == 0 or world == 1:
            __graft_entry__.build()
        if world > 1:
            dist.barrier()
            __graft_entry__.build()
        if args.config == "batch256":
            out = run_batch(args, rank, world)
        elif args.config == "serve":
            out = run_serve(args, rank, world)
        else:
            out = run_ours(args, rank, world)
            if world == 1 and not args.no_extra and args.config == "blobs512":
                out.update(extra_lines(args))
        if world > 1:
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
