#!/usr/bin/env python
"""Benchmark: time to final image of the speculative progressive isosurface
raycaster (arXiv 2309.10212) on one GB300, with the CPU oracle beside it.

A step is one whole render -- ray generation and every pass (traverse with
speculation, entry grouping, LRU cache, decode, intersect, resolve) until no
ray is live -- of one camera pose from a cold block cache, on a volume that is
already resident in device memory.  Poses cycle through the workload's orbit.

Workloads (synthetic stand-ins for the paper's data sets, see synth/):
  paper (default)   2048x2048x1920 u8 mixing layer, 2 bits/value, iso 0.5,
                    1280x720, one pose, 4 GB cache, adaptive speculation (cap 64)
                    -- the configuration of the paper's R-M figure (Sec. 5.1)
  medium            512^3 u8 Gaussian blobs + 10% noise, 2 bits/value, iso 0.3,
                    1280x720, 16-pose orbit, cache 10% of the decoded size,
                    adaptive speculation capped at 16 (also reported as a
                    sub-object of the paper line unless --no-medium)
  small             64^3 float value noise, 8 bits/value, iso 0.5, 256x256,
                    cache 25% of the blocks, fixed k = 4

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to final image & per pass at 1280×720; decoded GB/s vs HBM peak; blocks decoded"

# Algorithmic bytes of the hot-path kernels per unit of work (the units come
# from the render's own per-pass counters):
#   traversal: per live ray, its ray (16 B) and iterator state (32 B) read and
#     the state written back (32 B), 4 B per speculated R_BID slot, and 8 B per
#     range-grid entry the walk visits (one per walk step);
#   decode: 8*rate bytes of bit stream read and 256 bytes of values written
#     per decoded block;
#   intersection: per visible block its 5^3 dual grid (125 x 4 B), per entry
#     the ray (16 B) and the 8-byte atomic on the pixel's key.
TRAV_BYTES_PER_RAY = 16 + 32 + 32
TRAV_BYTES_PER_SLOT = 4
TRAV_BYTES_PER_STEP = 8
ISECT_BYTES_PER_VISIBLE = 125 * 4
ISECT_BYTES_PER_ENTRY = 16 + 8


def decode_bytes_per_block(rate):
    return 8 * rate + 256


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of
# the same build of that kernel on the same workload: (kernel, dims, rate) ->
# (bytes, source).  Empty a line when the kernel changes.
MEASURED_TRAFFIC = {
    ("decode_sorted_kernel", (2048, 2048, 1920), 2): (
        110_352_640,
        "one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum: mean of the render's "
        "two launches (110.8 and 109.9 MB; the decoder also writes the slot assignment)"),
    ("traverse_kernel / traverse_seg_kernel", (2048, 2048, 1920), 2): (
        5_134_464,
        "one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum: mean of the render's two "
        "walking launches (traverse_kernel in pass 1: 5.81 MB; traverse_seg_kernel in pass 2: 4.46 MB)"),
}

WORKLOADS = {
    "medium": dict(field="blobs", dims=(512, 512, 512), rate=2, iso=0.3, W=1280, H=720, poses=16,
                   cache_bytes=int(0.10 * 512 ** 3 * 4), spec="adaptive", k=16,
                   name="medium: 512^3 u8 Gaussian blobs + 10% noise, 2 bits/value, iso 0.3, "
                        "1280x720, 16-pose orbit, cache 10% of decoded size, adaptive k<=16"),
    "paper": dict(field="mixing", dims=(2048, 2048, 1920), rate=2, iso=0.5, W=1280, H=720, poses=1,
                  cache_bytes=4 << 30, spec="adaptive", k=64,
                  name="paper-scale: 2048x2048x1920 u8 mixing layer, 2 bits/value, iso 0.5, "
                       "1280x720, cache 4 GB, adaptive k<=64"),
    "small": dict(field="noise", dims=(64, 64, 64), rate=8, iso=0.5, W=256, H=256, poses=1,
                  cache_bytes=1024 * 256, spec="fixed", k=4,
                  name="small: 64^3 value noise, 8 bits/value, iso 0.5, 256x256, "
                       "cache 25% of blocks, k=4"),
}


def replica_pose_index(rank: int, i: int) -> int:
    """Pose index of the i-th render of replica `rank`: every rank renders
    its own sequence (the path shards by image with no exchange), offset by
    1000 per rank so that no two ranks render the same pose."""
    return rank * 1000 + i


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest value over the ranks of the process group (the job's time
    is its slowest replica's); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2070.0), src="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


def pose(wl, i):
    import synth
    if wl["field"] == "noise":
        return synth.cameras.small_pose(wl["dims"], wl["W"], wl["H"])
    if wl["field"] == "mixing":
        return synth.cameras.paper_pose(wl["dims"], wl["W"], wl["H"])
    return synth.cameras.medium_pose(i % wl["poses"], wl["dims"], wl["W"], wl["H"])


def make_volume_u8_or_f32(wl, device):
    """The raw (uncompressed) volume as a torch tensor on `device` (small and
    medium workloads; the mixing layer is generated slab by slab)."""
    import synth
    dims = wl["dims"]
    if wl["field"] == "noise":
        return synth.volumes.value_noise(dims, seed=1, device=device)
    return synth.volumes.gaussian_blobs(dims, seed=2, device=device)


def is_mixing_layer(wl):
    return wl["field"] == "mixing"


def raw_slabs(wl, device):
    """The workload's raw volume as (z0, z1, tensor (z1-z0, Dy, Dx)) slabs,
    generated by synth (the seeded input generator both sides use) on
    `device`: 64-voxel slabs of the mixing layer, the other volumes whole."""
    import synth
    dims = wl["dims"]
    if is_mixing_layer(wl):
        Dz = dims[2]
        params = synth.volumes.mixing_layer_params(3, scale=Dz / 1920.0)
        for z0 in range(0, Dz, 64):
            z1 = min(Dz, z0 + 64)
            yield z0, z1, synth.volumes.mixing_layer_slab(dims, z0, z1, params, z_mid=Dz / 2.0,
                                                          device=device)
    else:
        yield 0, dims[2], make_volume_u8_or_f32(wl, device)


def compress_volume(wl, spr=None, torch=None, library=True, oracle_side=False):
    """Compress the workload's volume slab by slab (slabs of 4k voxels in z,
    so the per-slab streams concatenate to the whole volume's): with the
    library's encoder into a device stream (`library`) and/or with the
    oracle's own encoder into a host stream (`oracle_side`).  The raw slabs
    come from synth on the GPU when there is one.  Returns (device stream or
    None, host stream or None)."""
    import numpy as np
    if torch is None:
        import torch
    dims, rate = wl["dims"], wl["rate"]
    nb = [(d + 3) // 4 for d in dims]
    total = nb[0] * nb[1] * nb[2] * 8 * rate
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    out_dev = torch.empty(total, dtype=torch.uint8, device="cuda") if library else None
    out_host = np.empty(total, dtype=np.uint8) if oracle_side else None
    if oracle_side:
        import oracle
        oracle.build()
    for z0, z1, raw in raw_slabs(wl, dev):
        lo = nb[0] * nb[1] * (z0 // 4) * 8 * rate
        n = nb[0] * nb[1] * ((z1 - z0 + 3) // 4) * 8 * rate
        if library:
            if raw.dtype == torch.uint8:
                spr.spr_encode_u8(raw, rate, out=out_dev[lo:lo + n])
            else:
                spr.spr_encode_f32(raw, rate, out=out_dev[lo:lo + n])
        if oracle_side:
            host = raw.cpu().numpy()
            out_host[lo:lo + n] = oracle.encode_volume(host, (dims[0], dims[1], z1 - z0), rate)
        del raw
    return out_dev, out_host


def compressed_on_device(wl, spr, torch):
    """Generate the workload's volume on the GPU and compress it with the
    library's encoder; returns the block stream (device)."""
    return compress_volume(wl, spr, torch)[0]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to $SPR_CLOCKS_CSV (default: the temp directory)
        self.path = os.environ.get("SPR_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     "spr_clocks_bench.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          "--query-gpu=" + self.QUERY, "--format=csv,noheader",
                                          "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], 0.0, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx = max(mx, float(parts[2].split()[0]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sample_rows(H, bands, rows):
    """`bands` bands of `rows` consecutive pixel rows, spread evenly over an
    image of H rows: the oracle's timed sample (consecutive rows share
    blocks, as they do in a whole image)."""
    out = []
    for b in range(bands):
        c = int(round((b + 0.5) * H / bands)) - rows // 2
        c = max(0, min(H - rows, c))
        out.extend(range(c, c + rows))
    return sorted(set(out))


# Oracle samples (bands x rows): all host cores, and one core.  Sized for
# about 10-30 s of CPU work at paper scale on a 16-core host (about 1.5 s and
# 4 s of wall time).
ORACLE_SAMPLE = {"all": (16, 8), "one": (6, 3)}


def oracle_time(wl, comp_host, cam, rows, nthreads):
    """Render the pixel rows `rows` of one pose with the CPU oracle, blocks
    decoded on demand (Sec. 3.5) and memoised within the call, so the decode
    of every block the rays reach is counted.  Returns (ms per image
    extrapolated from the sample, details)."""
    import numpy as np

    import oracle
    dims, rate, W, H = wl["dims"], wl["rate"], wl["W"], wl["H"]
    ov = oracle.Volume.on_demand(comp_host, dims, rate)
    r = np.asarray(rows, dtype=np.int64)
    pixels = (r[:, None] * W + np.arange(W)[None, :]).reshape(-1)
    t0 = time.perf_counter()
    pix = oracle.render(ov, cam, W, H, wl["iso"], pixels=pixels, nthreads=nthreads)
    dt = time.perf_counter() - t0
    ms = 1e3 * dt * (W * H) / pixels.size
    return ms, dict(seconds=dt, pixels=int(pixels.size), rows=len(rows),
                    blocks_decoded=ov.last_decodes, hits=int(pix["hit"].sum()), threads=nthreads)


def cpu_baseline(wl, comp_host, cam, which=("all", "one")):
    """The oracle as it stands on the host cores: all cores (OpenMP over
    pixels) and one core, each on its bounded sample of pixel rows of the
    pose, extrapolated to the whole image."""
    ncores = os.cpu_count() or 1
    res = {}
    for key in which:
        bands, rows = ORACLE_SAMPLE[key]
        nt = ncores if key == "all" else 1
        ms, det = oracle_time(wl, comp_host, cam, sample_rows(wl["H"], bands, rows), nt)
        res[key] = dict(ms=ms, **det)
    return res


def describe_sample(d, W, H):
    return ("C oracle (FP64, %d thread%s, blocks decoded on demand and memoised per render, "
            "%d decoded): %d pixel rows (%d pixels, bands of consecutive rows spread over the "
            "image) of the %dx%d image in %.2f s, extrapolated to the whole image" %
            (d["threads"], "" if d["threads"] == 1 else "s", d["blocks_decoded"], d["rows"],
             d["pixels"], W, H, d["seconds"]))


def run_reference(args, wl):
    """The reference arm: the CPU oracle (the plain definition the GPU path is
    checked against) timed on the host cores on the workload's pose, each
    step a bounded sample of pixel rows.  Its input is the oracle's own
    encoding of the synth volume."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    _, comp = compress_volume(wl, library=False, oracle_side=True)
    cam = pose(wl, 0)
    bands, rows = ORACLE_SAMPLE["all"]
    sample = sample_rows(wl["H"], bands, rows)
    times, det = [], None
    for step in range(args.warmup + args.steps):
        ms, det = oracle_time(wl, comp, cam, sample, nthreads)
        if step >= args.warmup:
            times.append(ms)
    value = statistics.mean(times) if times else float("nan")
    print(json.dumps({
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(value, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "dims": list(wl["dims"]), "rate": wl["rate"],
                   "image": [wl["W"], wl["H"]], "iso": wl["iso"]},
        "cpu_baseline": {"value": round(value, 3), "unit": "ms", "cores": nthreads,
                         "kind": "oracle", "sample": describe_sample(det, wl["W"], wl["H"])},
        "e2e": {"value": round(value, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


def run_oracle_passes(args, wl):
    """The oracle's progressive replay on the host cores (the CPU counterpart
    of the renderer's pass structure): the plain raycaster over every pixel
    with each ray's visible-block list, then the pass simulator (speculation
    rule, LRU cache, overflow rule) from a cold cache, on pose 0.  Prints its
    times and the passes and decodes it counts."""
    import time

    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    _, comp = compress_volume(wl, library=False, oracle_side=True)
    cam = pose(wl, 0)
    W, H, dims = wl["W"], wl["H"], wl["dims"]
    ov = oracle.Volume.on_demand(comp, dims, wl["rate"], lazy_fine=True)
    t0 = time.perf_counter()
    pix, off, vis = oracle.render(ov, cam, W, H, wl["iso"], lists=True)
    t1 = time.perf_counter()
    if wl["spec"] == "fixed":
        spec = dict(spec_mode=oracle.SPEC_FIXED, k=wl["k"])
    else:
        spec = dict(spec_mode=oracle.SPEC_ADAPTIVE, k_max=wl["k"])
    st, _ = oracle.simulate(W, H, dims, pix, off, vis, n_slots=wl["cache_bytes"] // 256, **spec)
    t2 = time.perf_counter()
    print(json.dumps({
        "impl": "oracle_passes", "workload": wl["name"], "cores": nthreads,
        "render_with_lists_ms": round(1e3 * (t1 - t0), 1), "simulate_ms": round(1e3 * (t2 - t1), 1),
        "total_ms": round(1e3 * (t2 - t0), 1), "passes": int(len(st["n_active"])),
        "blocks_decoded": int(st["n_decoded"].sum()), "entries": int(st["n_entries"].sum()),
        "block_decodes_in_render": int(ov.last_decodes),
        "note": "C oracle, FP64, blocks decoded on demand (lazy fine ranges); the simulator replays "
                "the speculation rule, the LRU cache and the overflow rule on the rays' lists"}))
    return 0


def run_study(args, wl):
    """Speculation sweep (fixed k = 1..16, adaptive caps 16 and 64), resolution
    scaling (640x360, 1280x720, 1920x1080) and blocks decoded against the
    decode-every-active-block count of Sec. 5.3, on one workload.  Every
    render starts from an empty cache; times are CUDA events around the
    C-ABI calls, as in the bench line."""
    import ctypes

    import torch

    from paper_2309_10212_gb300 import build
    build.build()
    import paper_2309_10212_gb300 as spr
    from paper_2309_10212_gb300 import _lib
    L = _lib.load()
    stream = torch.cuda.Stream()
    out = {"workload": wl["name"], "iso": wl["iso"], "dims": list(wl["dims"]), "rate": wl["rate"],
           "cache_bytes": wl["cache_bytes"]}
    with torch.cuda.stream(stream):
        comp = compressed_on_device(wl, spr, torch)
        vol = spr.spr_create_volume(wl["dims"], wl["rate"], comp, stream=stream)
        act, need = spr.spr_count_active_blocks(vol, wl["iso"], stream=stream)
        out["active_blocks"], out["needed_blocks"] = act, need
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        f3 = ctypes.c_float * 3
        n_pose = min(wl["poses"], 16)

        def measure(W, H, spec, k):
            w2 = dict(wl, W=W, H=H)
            r = spr.spr_create_renderer(vol, W, H)
            spr.spr_set_cache_budget(r, wl["cache_bytes"])
            if spec == "fixed":
                spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=k)
            else:
                spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k)
            spr.spr_set_isovalue(r, wl["iso"])
            cams = [tuple(f3(*[float(v) for v in c[key]]) for key in ("eye", "p00", "du", "dv"))
                    for c in (pose(w2, i) for i in range(n_pose))]
            rows = []
            for rep in range(2):          # the first round warms up
                for i in range(n_pose):
                    flush.fill_(i & 255)
                    rs = _lib.RenderStats()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    _lib.check(L.spr_reset_cache(r.handle))
                    _lib.check(L.spr_set_camera(r.handle, *cams[i]))
                    _lib.check(L.spr_render_to_convergence(r.handle, ctypes.c_void_p(stream.cuda_stream),
                                                           4096, ctypes.byref(rs), None))
                    b.record(stream)
                    b.synchronize()
                    if rep:
                        d = rs.as_dict()
                        d["ms"] = a.elapsed_time(b)
                        rows.append(d)
            r.close()
            mean = lambda key: statistics.mean(x[key] for x in rows)   # noqa: E731
            return {"W": W, "H": H, "spec": spec, "k": k, "poses": n_pose,
                    "ms": round(mean("ms"), 4), "passes": round(mean("passes"), 2),
                    "ms_per_pass": round(mean("ms") / max(mean("passes"), 1e-9), 4),
                    "blocks_decoded": round(mean("blocks_decoded"), 1),
                    "decoded_vs_needed": round(mean("blocks_decoded") / max(need, 1), 4),
                    "entries": round(mean("entries"), 1),
                    "utilization_per_pass": round(mean("entries") / max(mean("passes"), 1e-9) / (W * H), 4)}

        # batched views: B orbit poses in one wavefront with a shared cache,
        # against the same poses rendered one by one
        if wl["poses"] >= 4:
            from paper_2309_10212_gb300 import tune
            out["batch"] = []
            for B in (1, 2, 4, 8, 16):
                r = spr.spr_create_renderer(vol, wl["W"], wl["H"])
                spr.spr_set_cache_budget(r, wl["cache_bytes"])
                spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=wl["k"])
                spr.spr_set_isovalue(r, wl["iso"])
                spr.spr_set_view_count(r, B)
                times, dec, npass, att = [], [], [], []
                for rep in range(3):
                    flush.fill_(rep & 255)
                    for v in range(B):          # (re)starts the render; host only
                        spr.spr_set_view(r, v, pose(wl, v), wl["iso"])
                    rs = _lib.RenderStats()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    _lib.check(L.spr_reset_cache(r.handle))
                    _lib.check(L.spr_render_to_convergence(r.handle, ctypes.c_void_p(stream.cuda_stream), 4096,
                                                           ctypes.byref(rs), None))
                    b.record(stream)
                    b.synchronize()
                    if rep:
                        times.append(a.elapsed_time(b))
                        dec.append(rs.blocks_decoded)
                        npass.append(rs.passes)
                        att.append(rs.kernel_launches)
                r.close()
                out["batch"].append({"views": B, "ms": round(statistics.mean(times), 4),
                                     "ms_per_view": round(statistics.mean(times) / B, 4),
                                     "blocks_decoded_per_view": round(statistics.mean(dec) / B, 1),
                                     "passes": round(statistics.mean(npass), 2),
                                     "kernel_launches": round(statistics.mean(att), 1)})
            # the autotuner on the first four poses
            r = spr.spr_create_renderer(vol, wl["W"], wl["H"])
            spr.spr_set_cache_budget(r, wl["cache_bytes"])
            spr.spr_set_isovalue(r, wl["iso"])
            spr.spr_set_camera(r, pose(wl, 0))
            res = tune.autotune(r, [pose(wl, i) for i in range(4)], k_max=(4, 8, 16, 32, 64),
                                warp_walk=(4096, 16384, 65536), stream=stream)
            r.close()
            out["autotune"] = res

        out["k_sweep"] = [measure(wl["W"], wl["H"], "fixed", k) for k in (1, 2, 4, 8, 16)]
        out["k_sweep"] += [measure(wl["W"], wl["H"], "adaptive", k) for k in (16, 64)]
        spec = wl["spec"]
        out["resolution"] = [measure(W, H, spec, wl["k"]) for W, H in ((640, 360), (1280, 720), (1920, 1080))]
        vol.close()
    with open(args.study, "w") as f:
        json.dump(out, f, indent=1)
    best = min(out["k_sweep"], key=lambda x: x["ms"])
    print(json.dumps({"study": args.study, "active_blocks": act, "needed_blocks": need,
                      "best": {k: best[k] for k in ("spec", "k", "ms", "passes", "blocks_decoded")}}))
    return 0


def run_learned(args, wl):
    """Learned speculation policy (config: the paper-scale volume, traces of
    the plain raycaster from 64 random poses with isovalues in [0.2, 0.8],
    evaluation on 32 held-out poses against the plain adaptive rule, every
    image required to be bit-identical).  Renders start from an empty
    cache; times are CUDA events around the C-ABI calls."""
    import ctypes

    import numpy as np
    import torch

    import synth
    from paper_2309_10212_gb300 import build
    build.build()
    import paper_2309_10212_gb300 as spr
    from paper_2309_10212_gb300 import _lib
    L = _lib.load()
    stream = torch.cuda.Stream()
    out = {"workload": wl["name"], "train_poses": args.learn_train, "eval_poses": args.learn_eval}
    rng = np.random.Generator(np.random.PCG64(21))
    dims, W, H = wl["dims"], wl["W"], wl["H"]

    def poses(n, seed0):
        res = []
        for i in range(n):
            cam = synth.cameras.random_pose(dims, seed=seed0 + i, W=W, H=H,
                                            distance_factor=float(rng.uniform(1.3, 2.0)))
            res.append((cam, float(np.float32(rng.uniform(0.2, 0.8)))))
        return res

    train, held = poses(args.learn_train, 2000), poses(args.learn_eval, 3000)
    f3 = ctypes.c_float * 3
    with torch.cuda.stream(stream):
        comp = compressed_on_device(wl, spr, torch)
        vol = spr.spr_create_volume(dims, wl["rate"], comp, stream=stream)
        del comp
        r = spr.spr_create_renderer(vol, W, H)
        spr.spr_set_cache_budget(r, wl["cache_bytes"])
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def one(cam, iso, keep=False):
            flush.fill_(1)
            rs = _lib.RenderStats()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            args_ = [f3(*[float(v) for v in cam[k]]) for k in ("eye", "p00", "du", "dv")]
            a.record(stream)
            _lib.check(L.spr_reset_cache(r.handle))
            _lib.check(L.spr_set_camera(r.handle, *args_))
            _lib.check(L.spr_set_isovalue(r.handle, ctypes.c_float(iso)))
            _lib.check(L.spr_render_to_convergence(r.handle, ctypes.c_void_p(stream.cuda_stream), 4096,
                                                   ctypes.byref(rs), None))
            b.record(stream)
            b.synchronize()
            d = rs.as_dict()
            d["ms"] = a.elapsed_time(b)
            if keep:
                fb = spr.spr_get_framebuffer(r)
                d["image"] = {k: fb[k].clone() for k in ("depth", "rgba", "block", "cell", "status")}
            return d

        # 1. traces of the plain raycaster
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=wl["k"])
        cap = args.learn_samples
        tr = spr.Trace(cap)
        spr.spr_set_trace(r, tr, args.learn_mod)
        t0 = time.perf_counter()
        for cam, iso in train:
            one(cam, iso)
            spr.spr_trace_labels(r, tr, stream=stream)
        spr.spr_set_trace(r, None)
        n = tr.n
        lab = tr.labels[:n].cpu().numpy()
        out["trace"] = {"samples": n, "sample_mod": args.learn_mod, "s": round(time.perf_counter() - t0, 2),
                        "label_mean": round(float(lab.mean()), 3),
                        "label_p50": int(np.percentile(lab, 50)), "label_p90": int(np.percentile(lab, 90))}
        # 2. training (hand-written kernels), seeded initial parameters
        init = np.concatenate([np.ravel(x) for x in _init_params(5)]).astype(np.float32)
        t0 = time.perf_counter()
        params, losses = spr.spr_policy_train(tr.features[:n], tr.labels[:n], init, epochs=args.learn_epochs,
                                              batch=8192, lr=2e-3, tau=0.9, seed=1, stream=stream)
        torch.cuda.synchronize()
        out["train"] = {"epochs": args.learn_epochs, "s": round(time.perf_counter() - t0, 3),
                        "mse_log2_per_epoch": [round(float(x), 4) for x in losses]}
        del tr
        # 3. the margin on the first training poses, with and without the
        # floor at the paper's uniform count
        tune = []
        for floor in ("all", "after_first", None):
            for m in (-1.0, -0.5, 0.0, 0.5, 1.0, 2.0):
                spr.spr_set_policy(r, params, m, floor=floor)
                spr.spr_set_speculation(r, spr.SPR_SPEC_LEARNED, k_max=wl["k"])
                for cam, iso in train[:2]:
                    one(cam, iso)                          # warm-up
                rows = [one(cam, iso) for cam, iso in train[:8]]
                tune.append({"floor": floor, "margin": m, "ms": round(statistics.mean(x["ms"] for x in rows), 4),
                             "passes": round(statistics.mean(x["passes"] for x in rows), 3),
                             "blocks_decoded": round(statistics.mean(x["blocks_decoded"] for x in rows), 1)})
        best = {f: min((t for t in tune if t["floor"] == f), key=lambda x: x["ms"])
                for f in ("all", "after_first", None)}
        fewest = min((t for t in tune if not t["floor"]), key=lambda x: x["blocks_decoded"])
        out["margin"] = {"table": tune, "fastest_floor": best["all"]["margin"],
                         "fastest_floor_after_first": best["after_first"]["margin"],
                         "fastest_no_floor": best[None]["margin"], "fewest_blocks_no_floor": fewest["margin"]}
        # 4. held-out poses: plain against learned, images compared
        arms = [("learned_floor", "all", best["all"]["margin"]),
                ("learned_floor_after_first", "after_first", best["after_first"]["margin"]),
                ("learned_fewest_blocks", None, fewest["margin"])]
        res = {"plain": []}
        res.update({a[0]: [] for a in arms})
        same = {a[0]: 0 for a in arms}
        for cam, iso in held:
            spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=wl["k"])
            one(cam, iso)
            a = one(cam, iso, keep=True)
            for name, floor, m in arms:
                spr.spr_set_policy(r, params, m, floor=floor)
                spr.spr_set_speculation(r, spr.SPR_SPEC_LEARNED, k_max=wl["k"])
                one(cam, iso)
                b = one(cam, iso, keep=True)
                same[name] += all(torch.equal(a["image"][k], b["image"][k]) for k in a["image"])
                del b["image"]
                res[name].append(b)
            del a["image"]
            res["plain"].append(a)

        def summ(rows):
            return {k: round(statistics.mean(x[k] for x in rows), 4)
                    for k in ("ms", "passes", "blocks_decoded", "entries")}
        out["plain"] = dict(summ(res["plain"]), rule="adaptive k<=%d" % wl["k"])
        for name, floor, m in arms:
            out[name] = dict(summ(res[name]), rule="learned count (<= 32, k_max %d)%s, margin %g" %
                             (wl["k"], {"all": ", floored at the adaptive count",
                                        "after_first": ", floored at the adaptive count from pass 2",
                                        None: ""}[floor], m),
                             identical_images="%d/%d" % (same[name], len(held)))
        out["identical_images"] = "%d/%d" % (min(same.values()), len(held))
        # the tensor-core MLP alone on one row per pixel (features in HBM)
        feats = torch.rand((W * H, 12), device="cuda")
        spr.spr_policy_forward(params, feats, stream=stream)
        ts = []
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            spr.spr_policy_forward(params, feats, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        out["mlp_forward"] = {"rows": W * H, "ms": round(statistics.median(ts), 4),
                              "tflops": round(2 * W * H * (16 * 64 + 64 * 64 + 64 * 16) / (statistics.median(ts) / 1e3) / 1e12, 2),
                              "timing": "median of 5 spr_policy_forward calls (includes its parameter copy and sync)"}
        r.close()
        vol.close()
    with open(args.learned, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"learned": args.learned, "plain": out["plain"], "learned_floor": out["learned_floor"],
                      "learned_floor_after_first": out["learned_floor_after_first"],
                      "learned_fewest_blocks": out["learned_fewest_blocks"],
                      "identical_images": out["identical_images"], "train": out["train"],
                      "mlp_forward": out["mlp_forward"]}))
    return 0


def _init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) layers of the 12-64-64-2
    policy, in the C ABI's order (W1, b1, W2, b2, W3, b3)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_out, fan_in in ((64, 12), (64, 64), (2, 64)):
        bound = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)))
        parts.append(rng.uniform(-bound, bound, size=fan_out))
    return parts


SERVE_VOLUMES = [
    # (name, dims, generator, cache bytes per view)
    ("256^3 u8 Gaussian blobs (100)", (256, 256, 256), "blobs256", int(0.10 * 256 ** 3 * 4)),
    ("1024^3 u8 Gaussian blobs (800)", (1024, 1024, 1024), "blobs1024", int(0.10 * 1024 ** 3 * 4)),
    ("2048x2048x1920 u8 mixing layer", (2048, 2048, 1920), "paper", 1 << 30),
]
SERVE_RES = [(640, 360), (1280, 720), (1920, 1080)]


def serve_trace(n, rate_hz, seed=11):
    """n requests: Poisson arrivals (mean rate_hz), a volume and a resolution
    uniform over the three, a random camera and an isovalue uniform in
    [0.2, 0.8] (rounded to float32)."""
    import numpy as np

    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        vi = int(rng.integers(0, len(SERVE_VOLUMES)))
        W, H = SERVE_RES[int(rng.integers(0, len(SERVE_RES)))]
        iso = float(np.float32(rng.uniform(0.2, 0.8)))
        dims = SERVE_VOLUMES[vi][1]
        cam = synth.cameras.random_pose(dims, seed=1000 + i, W=W, H=H,
                                        distance_factor=float(rng.uniform(1.3, 2.0)))
        out.append(dict(t=float(t[i]), vol=vi, W=W, H=H, iso=iso, cam=cam))
    return out


def serve_volumes(spr, torch):
    """The serving mix's three resident volumes at 2 bits/value, with their
    per-view cache budgets: [(volume, cache bytes per view)]."""
    import synth
    vols = []
    for name, dims, gen, cache in SERVE_VOLUMES:
        if gen == "paper":
            comp = compressed_on_device(WORKLOADS["paper"], spr, torch)
        else:
            n = 100 if dims[0] == 256 else 800
            u8 = synth.volumes.gaussian_blobs(dims, seed=6 if dims[0] == 256 else 7, n=n, device="cuda")
            comp = spr.spr_encode_u8(u8, 2)
            del u8
        vols.append((spr.spr_create_volume(dims, 2, comp), cache))
        del comp
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return vols


def run_batched(args):
    """Renders of several volumes in one graph launch (spr_batch_render)
    against the plain loop of one render at a time, on the serving mix:
    three resident volumes (256^3 and 1024^3 Gaussian blobs, the
    2048x2048x1920 mixing layer; 2 bits/value), resolutions 640x360 /
    1280x720 / 1920x1080, random cameras and isovalues in [0.2, 0.8], an
    8 GB cache budget.  A burst of requests is split in two: the first half
    tunes the batch's knobs (views per renderer, the cache split among the
    renderers, k_max) and the plain loop's k_max; the second half is timed
    in both forms (device time, cold caches), every image compared."""
    import torch

    from paper_2309_10212_gb300 import build
    build.build()
    import paper_2309_10212_gb300 as spr
    from paper_2309_10212_gb300 import tune
    t0 = time.perf_counter()
    vols = serve_volumes(spr, torch)
    setup_s = time.perf_counter() - t0
    trace = serve_trace(args.batch_requests, args.serve_rate)
    half = len(trace) // 2
    tune_set, eval_set = trace[:half], trace[half:]
    per_view = {i: c for i, (_, c) in enumerate(vols)}
    handles = [v for v, _ in vols]
    total = 8 << 30
    stream = torch.cuda.Stream()
    out = {"config": "serving mix: volumes " + ", ".join(v[0] for v in SERVE_VOLUMES) +
                     "; resolutions 640x360/1280x720/1920x1080; iso U[0.2,0.8]; 8 GB cache budget; "
                     "%d requests (%d tune, %d timed); cold caches" % (len(trace), half, len(eval_set)),
           "setup_s": round(setup_s, 1)}
    with torch.cuda.stream(stream):
        runner = tune.BatchRunner(handles, stream)
        best = tune.autotune_batch(runner, tune_set, total, per_view, views=(1, 2, 4, 8),
                                   splits=("per_view", "equal", "pixels"), k_max=(16, 64))
        out["autotune"] = {"chosen": {k: best[k] for k in ("views", "split", "k_max")},
                           "table": best["table"]}
        plain_tune = []
        for k in (16, 64):
            pool = {}
            tune.run_requests_plain(handles, tune_set, per_view, k, stream, pool)
            plain_tune.append(dict(k_max=k, **tune.run_requests_plain(handles, tune_set, per_view, k, stream, pool)))
            for r in pool.values():
                r.close()
        kp = min(plain_tune, key=lambda x: x["ms"])["k_max"]
        out["plain_autotune"] = {"chosen_k_max": kp, "table": plain_tune}
        # the timed half: plain loop (images kept), then the batched form
        imgs = {}

        def keep_plain(i, fb):
            imgs[i] = {k: fb[k].clone() for k in ("depth", "block", "status", "rgba")}
        pool = {}
        tune.run_requests_plain(handles, eval_set, per_view, kp, stream, pool)
        out["plain"] = tune.run_requests_plain(handles, eval_set, per_view, kp, stream, pool, keep=keep_plain)
        for r in pool.values():
            r.close()
        same = {"n": 0}

        def keep_batched(i, fb):
            same["n"] += all(torch.equal(fb[k], imgs[i][k]) for k in imgs[i])
        V, split, k = best["views"], best["split"], best["k_max"]
        runner.run(eval_set, V, split, total, per_view, k)
        out["batched"] = runner.run(eval_set, V, split, total, per_view, k)
        runner.run(eval_set, V, split, total, per_view, k, keep=keep_batched)
        out["batched"].update(views=V, split=split, k_max=k)
        runner.close()
        out["identical_images"] = "%d/%d" % (same["n"], len(eval_set))
        out["speedup_device"] = round(out["plain"]["ms"] / out["batched"]["ms"], 3)
        out["speedup_wall"] = round(out["plain"]["wall_ms"] / out["batched"]["wall_ms"], 3)
    for v, _ in vols:
        v.close()
    with open(args.batched, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"batched": args.batched, "plain": out["plain"], "batched_form": out["batched"],
                      "identical_images": out["identical_images"], "speedup_device": out["speedup_device"],
                      "speedup_wall": out["speedup_wall"]}))
    return 0


def run_serve(args):
    """The render service (config: 256 requests arriving as a Poisson process
    at 20/s over three resident volumes, resolutions 640x360 / 1280x720 /
    1920x1080, random cameras, isovalues in [0.2, 0.8], an 8 GB device
    memory budget for the pooled renderers).  Reports p50/p99 time to first
    pass and to final image, then the same requests as a burst (all queued at
    once) with and without overlap and batching."""
    import numpy as np
    import torch

    import synth
    from paper_2309_10212_gb300 import build
    build.build()
    import paper_2309_10212_gb300 as spr
    out = {"config": "256 requests, Poisson 20/s, volumes " + ", ".join(v[0] for v in SERVE_VOLUMES) +
                     ", resolutions 640x360/1280x720/1920x1080, iso U[0.2,0.8], 8 GB memory budget"}
    t0 = time.perf_counter()
    vols = serve_volumes(spr, torch)
    out["setup_s"] = round(time.perf_counter() - t0, 1)
    trace = serve_trace(args.serve_requests, args.serve_rate)

    def run(trace, max_inflight, max_batch, k_max, realtime, memory=8 << 30, server=None):
        srv = server or spr.spr_server_create(memory, max_inflight=max_inflight, max_batch=max_batch,
                                              k_max=k_max)
        if server is None:
            srv.ids = [spr.spr_server_add_volume(srv, v, c) for v, c in vols]
        res = {}
        info0 = spr.spr_server_info(srv)
        base = spr.spr_server_clock(srv)
        i = 0
        while len(res) < len(trace):
            now = spr.spr_server_clock(srv) - base
            while i < len(trace) and (not realtime or trace[i]["t"] <= now):
                q = trace[i]
                t_arr = base + q["t"] if realtime else -1.0
                spr.spr_server_submit(srv, srv.ids[q["vol"]], q["cam"], q["iso"], q["W"], q["H"],
                                      t_arrival=t_arr)
                i += 1
            for r_ in spr.spr_server_poll(srv):
                res[r_["id"]] = r_
        info = spr.spr_server_info(srv)
        rows = [res[k] for k in sorted(res)]
        assert all(r_["status"] == 0 for r_ in rows), [r_ for r_ in rows if r_["status"]][:3]
        ttfp = np.array([r_["t_first_pass"] - r_["t_arrival"] for r_ in rows]) * 1e3
        fin = np.array([r_["t_done"] - r_["t_arrival"] for r_ in rows]) * 1e3
        span = max(r_["t_done"] for r_ in rows) - min(r_["t_arrival"] for r_ in rows)
        # blocks decoded per request: a batch's count is shared by its requests
        dec = sum(r_["blocks_decoded"] / r_["batch"] for r_ in rows)
        return srv, {"max_inflight": max_inflight, "max_batch": max_batch, "k_max": k_max,
                     "requests": len(rows), "makespan_s": round(span, 4),
                     "requests_per_s": round(len(rows) / span, 2),
                     "ttfp_ms_p50": round(float(np.percentile(ttfp, 50)), 3),
                     "ttfp_ms_p99": round(float(np.percentile(ttfp, 99)), 3),
                     "final_ms_p50": round(float(np.percentile(fin, 50)), 3),
                     "final_ms_p99": round(float(np.percentile(fin, 99)), 3),
                     "mean_batch": round(float(np.mean([r_["batch"] for r_ in rows])), 2),
                     "blocks_decoded_per_request": round(dec / len(rows), 1),
                     "renders": info["renders"] - info0["renders"],
                     "renderers_created": info["renderers_created"] - info0["renderers_created"],
                     "renderers_destroyed": info["renderers_destroyed"] - info0["renderers_destroyed"],
                     "memory_used_gb": round(info["memory_used"] / 1e9, 2)}

    # autotune the speculation cap on a burst of the first 48 requests
    tune_rows = []
    for k_max in (16, 32, 64):
        srv, row = run(trace[:48], 4, 8, k_max, False)
        _, row = run(trace[:48], 4, 8, k_max, False, server=srv)   # warm pool
        srv.close()
        tune_rows.append(row)
    k_best = min(tune_rows, key=lambda r_: r_["makespan_s"])["k_max"]
    out["autotune_k_max"] = {"table": [{k: r_[k] for k in ("k_max", "makespan_s")} for r_ in tune_rows],
                             "chosen": k_best}
    # Poisson arrivals in real time on a pool reserved with one renderer per
    # (volume, resolution) and warmed by one request of each (renderer
    # creation and graph capture excluded)
    srv = spr.spr_server_create(8 << 30, max_inflight=4, max_batch=8, k_max=k_best)
    srv.ids = [spr.spr_server_add_volume(srv, v, c) for v, c in vols]
    warm = []
    for vi in range(len(vols)):
        for W, H in SERVE_RES:
            spr.spr_server_reserve(srv, srv.ids[vi], W, H, 1)
            q = next(x for x in trace if x["vol"] == vi)
            warm.append(dict(q, W=W, H=H, cam=dict(q["cam"]), t=0.0))
    for q in warm:   # cameras are resolution-specific: rebuild for this size
        q["cam"] = synth.cameras.random_pose(SERVE_VOLUMES[q["vol"]][1], seed=77, W=q["W"], H=q["H"])
    run(warm, 4, 8, k_best, False, server=srv)
    _, out["poisson"] = run(trace, 4, 8, k_best, True, server=srv)
    # the same requests queued at once on that pool: overlap and batching
    # (a batch uses a pooled renderer's view capacity, or a new renderer
    # when the budget has room)
    _, out["burst_batched"] = run(trace, 4, 8, k_best, False, server=srv)
    srv.close()
    srv, _ = run(trace, 1, 1, k_best, False)
    _, out["burst_plain"] = run(trace, 1, 1, k_best, False, server=srv)
    srv.close()
    srv, _ = run(trace, 4, 1, k_best, False)
    _, out["burst_overlap_only"] = run(trace, 4, 1, k_best, False, server=srv)
    srv.close()
    for v, _ in vols:
        v.close()
    with open(args.serve, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"serve": args.serve, "poisson": out["poisson"],
                      "burst_batched": out["burst_batched"], "burst_plain": out["burst_plain"]}))
    return 0


def run_decode_slab(args):
    """Decode rate of the blocks the paper-scale render decodes: a slab of the
    2048x2048x1920 mixing layer at its interface (z = 928..959, 2 bits/value,
    2,097,152 blocks), every block decoded in one call, timed with CUDA events
    (median of --steps calls, L2 written between them): the plain decoder
    (spr_decode_blocks, consecutive blocks per warp) and the renderer's
    decoder (spr_volume_decode_blocks, blocks grouped by parse length).
    Prints one JSON line."""
    import torch

    from paper_2309_10212_gb300 import build
    build.build()
    import paper_2309_10212_gb300 as spr
    import synth
    dims, z0, z1, rate = (2048, 2048, 1920), 928, 960, 2
    u8 = synth.volumes.mixing_layer_slab(dims, z0, z1, synth.volumes.mixing_layer_params(3, scale=1.0),
                                         z_mid=960.0, device="cuda")
    comp = spr.spr_encode_u8(u8, rate)
    del u8
    nb = comp.numel() // (8 * rate)
    vol = spr.spr_create_volume((dims[0], dims[1], z1 - z0), rate, comp)
    out = torch.empty((nb, 64), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(call):
        ts = []
        for i in range(args.warmup + args.steps):
            flush.fill_(i & 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            call()
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    pk = peaks()
    res = {}
    for name, call in (("plain", lambda: spr.spr_decode_blocks(comp, nb, rate, out=out)),
                       ("grouped", lambda: spr.spr_volume_decode_blocks(vol, out=out))):
        ms = timed(call)
        gbs = nb * (8 * rate + 256) / (ms / 1e3) / 1e9
        res[name] = {"ms": round(ms, 4), "gblocks_per_s": round(nb / ms / 1e6, 3), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / pk["hbm_gbs"], 4)}
    print(json.dumps({"decode_slab": "mixing layer 2048x2048x1920, z %d..%d, %d bits/value" % (z0, z1 - 1, rate),
                      "blocks": nb, "peak_gbs": pk["hbm_gbs"],
                      "plain": dict(res["plain"], kernel="decode_list_kernel", call="spr_decode_blocks"),
                      "grouped": dict(res["grouped"], kernel="decode_sorted_kernel",
                                      call="spr_volume_decode_blocks"),
                      "timing": "median of %d CUDA-event timed calls, L2 written before each" % args.steps}))
    return 0


def stage_rooflines(prof_stats, stage, rate, pk):
    """Algorithmic GB/s of the traversal, decode and intersection stages over
    the instrumented renders (per-pass counters x bytes per unit, over each
    stage's CUDA-event time), against the measured HBM copy peak."""
    per_pass = [p for _, ps in prof_stats for p in ps]
    trav = sum(p["n_processed"] * TRAV_BYTES_PER_RAY + p["n_entries_cap"] * TRAV_BYTES_PER_SLOT +
               p["n_steps"] * TRAV_BYTES_PER_STEP for p in per_pass)
    dec = sum(p["n_decoded"] * decode_bytes_per_block(rate) for p in per_pass)
    isect = sum(p["n_visible"] * ISECT_BYTES_PER_VISIBLE + p["n_entries"] * ISECT_BYTES_PER_ENTRY
                for p in per_pass)
    out = {}
    for name, kernel, nbytes, units in (
            ("traverse", "traverse_kernel / traverse_seg_kernel", trav,
             "live rays x %d B + speculated slots x %d B + walk steps x %d B" %
             (TRAV_BYTES_PER_RAY, TRAV_BYTES_PER_SLOT, TRAV_BYTES_PER_STEP)),
            ("decode", "decode_sorted_kernel", dec, "decoded blocks x %d B" % decode_bytes_per_block(rate)),
            ("intersect", "intersect_kernel", isect,
             "visible blocks x %d B + entries x %d B" % (ISECT_BYTES_PER_VISIBLE, ISECT_BYTES_PER_ENTRY))):
        ms = stage[name]
        gbs = (nbytes / 1e9) / (ms / 1e3) if ms > 0 else 0.0
        out[name] = {"kernel": kernel, "bytes": int(nbytes), "ms": ms, "achieved": round(gbs, 1),
                     "frac": round(gbs / pk["hbm_gbs"], 4), "units": units}
    return out


def pass_slots(p):
    """Speculated R_BID slots of a pass under a uniform rule: k_used per ray
    taken."""
    return p["n_processed"] * p["k_used"]


def measure_workload(wl, args, spr, _lib, torch, stream, rank, world, dist, local, comp,
                     headline=True):
    """Time `args.steps` renders of the workload (after warm-up) and the
    instrumented renders behind the stage breakdown; returns a dict."""
    import ctypes
    pk = peaks()
    vol = spr.spr_create_volume(wl["dims"], wl["rate"], comp, stream=stream)
    r = spr.spr_create_renderer(vol, wl["W"], wl["H"])
    spr.spr_set_cache_budget(r, wl["cache_bytes"])
    if wl["spec"] == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=wl["k"])
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=wl["k"])
    spr.spr_set_isovalue(r, wl["iso"])
    spr.spr_set_profiling(r, False)
    if args.warp_walk >= 0:
        spr.spr_set_warp_walk_threshold(r, args.warp_walk)
    if args.seg_lanes >= 0:
        spr.spr_set_segment_walk(r, args.seg_lanes)
    if args.isect_staged:
        spr.spr_set_intersect_staging(r, True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    L = _lib.load()
    f3 = ctypes.c_float * 3

    def cam_args(c):
        return tuple(f3(*[float(v) for v in c[k]]) for k in ("eye", "p00", "du", "dv"))

    def step(i):
        spr.spr_reset_cache(r)
        spr.spr_set_camera(r, pose(wl, replica_pose_index(rank, i)))
        return spr.spr_render_to_convergence(r, 100000, stream=stream)

    # The timed loop calls the C ABI directly with camera arrays prepared
    # beforehand; the per-pass records are converted after the end event.
    class Timed:
        def __init__(self, n, first):
            self.cams = [cam_args(pose(wl, replica_pose_index(rank, first + i))) for i in range(n)]
            self.rs = [_lib.RenderStats() for _ in range(n)]
            self.per = [(_lib.PassStats * 64)() for _ in range(n)]

        def run(self, i):
            _lib.check(L.spr_reset_cache(r.handle))
            _lib.check(L.spr_set_camera(r.handle, *self.cams[i]))
            _lib.check(L.spr_render_to_convergence(r.handle, ctypes.c_void_p(stream.cuda_stream), 64,
                                                   ctypes.byref(self.rs[i]), self.per[i]))

        def stats(self, i):
            rs = self.rs[i].as_dict()
            return rs, [self.per[i][k].as_dict() for k in range(rs["passes"])]

    res = {}
    with ClockSampler(local) as clk:
        # warm-up: at least `warmup` renders and at least `warm_s` seconds of
        # them, so that the clock record covers the load the timed renders run in
        t_end = time.perf_counter() + (args.warm_s if headline else 0.0)
        i = 0
        while i < args.warmup or time.perf_counter() < t_end:
            flush.fill_(i & 255)
            step(i)
            torch.cuda.synchronize()
            i += 1
        res["warmup_renders"] = i
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        timed = Timed(args.steps, args.warmup)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_((i + 7) & 255)          # L2 flush, outside the timed region
            ev0[i].record(stream)
            timed.run(i)
            ev1[i].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    res["clocks"] = clk.summary()
    stats = [timed.stats(i) for i in range(args.steps)]
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms_image = max_over_ranks(statistics.mean(step_ms), dist, device="cuda")
    res["ms_image"] = ms_image
    res["ms_image_median"] = statistics.median(step_ms)
    res["stats"] = stats

    # Per-stage device times: the same poses again, each pass attempt as a
    # captured graph with events between its stages.
    n_prof = min(args.steps, 16)
    prof_stats = []
    spr.spr_set_profiling(r, True)
    for i in range(n_prof):
        flush.fill_((i + 7) & 255)
        prof_stats.append(step(args.warmup + i))
    spr.spr_set_profiling(r, False)
    torch.cuda.synchronize()
    stage_names = ["traverse", "group", "cache", "decode", "intersect", "resolve"]
    stage = {n: 0.0 for n in stage_names}
    per_index = {}
    isect_entries, isect_ms = 0, 0.0
    for rs, passes in prof_stats:
        for p in passes:
            p["n_entries_cap"] = pass_slots(p)
            for k, n in enumerate(stage_names):
                stage[n] += p["ms_stage"][k]
            per_index.setdefault(p["pass"], []).append(p["ms"])
            isect_entries += p["n_entries"]
            isect_ms += p["ms_stage"][4]
    n_prof_r = max(1, len(prof_stats))
    rl = stage_rooflines(prof_stats, stage, wl["rate"], pk)
    dom = max(rl, key=lambda n: stage[n])
    total_stage = sum(stage.values()) or 1.0
    d = rl[dom]
    res["roofline"] = {
        "kernel": d["kernel"], "stage": dom, "bound": "hbm", "achieved": d["achieved"],
        "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": d["frac"],
        "traffic": None, "peak_source": pk["src"] + " HBM copy peak (MEASURED_PEAKS.json hbm_gbs)",
        "work": d["units"] + " (per-pass counters of the instrumented renders)",
        "share": round(stage[dom] / total_stage, 3),
        "timing": "CUDA-event time of the kernel's stage, %d instrumented renders of the same poses" % n_prof_r}
    tr = MEASURED_TRAFFIC.get((d["kernel"], tuple(wl["dims"]), wl["rate"]))
    if tr:
        res["roofline"]["traffic"] = tr[0]
        res["roofline"]["traffic_source"] = tr[1]
    res["stage_roofline"] = {k: {kk: v[kk] for kk in ("kernel", "achieved", "frac", "units")} | {
        "ms_per_image": round(v["ms"] / n_prof_r, 4)} for k, v in rl.items()}
    res["stage_ms_per_image"] = {k: round(v / n_prof_r, 4) for k, v in stage.items()}
    res["ms_per_pass_index"] = {str(k): round(statistics.mean(v), 4) for k, v in sorted(per_index.items())}
    res["isect"] = (isect_entries, isect_ms)
    dec_ms = stage["decode"]
    dec_bytes = rl["decode"]["bytes"]
    res["decoded_gbs"] = (dec_bytes / 1e9) / (dec_ms / 1e3) if dec_ms > 0 else 0.0
    res["prof_stats"] = prof_stats
    if not headline:
        r.close()
        vol.close()
        return res

    # end to end through the C ABI with host buffers: camera in, image out
    # (the RGBA image and its depth; the per-pixel block, cell, pass and
    # status diagnostics of the parity tests stay on the device)
    n = wl["W"] * wl["H"]
    host = {k: torch.empty(n * sz, dtype=torch.uint8, pin_memory=True)
            for k, sz in (("depth", 4), ("rgba", 4))}
    e2e, pass_reads = [], []
    h2d = 4 * 12 + 4
    d2h = sum(t.numel() for t in host.values())
    e2e_cams = [pose(wl, i) for i in range(args.e2e_steps)]
    for i in range(args.e2e_steps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        spr.spr_reset_cache(r)
        spr.spr_set_camera(r, e2e_cams[i])
        spr.spr_set_isovalue(r, wl["iso"])
        rs, _ = spr.spr_render_to_convergence(r, 100000, stream=stream)
        _lib.check(L.spr_read_framebuffer(r.handle, ctypes.c_void_p(stream.cuda_stream),
                                          *[ctypes.c_void_p(host[k].data_ptr() if k in host else None) for k in
                                            ("depth", "rgba", "block", "cell", "final", "status")]))
        e2e.append(1e3 * (time.perf_counter() - t0))
        pass_reads.append(rs["passes"] + 1)
    res["e2e"] = {"value": round(statistics.mean(e2e), 4), "unit": "ms", "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": int(d2h + 64 * statistics.mean(pass_reads)),
                  "read_back": "RGBA image and depth (8 B per pixel) through spr_read_framebuffer into "
                               "pinned host buffers, plus the per-pass records"}

    # Decode of a contiguous run of blocks (up to 16M blocks, 4 GB out)
    # through spr_decode_blocks: the decoder alone against the HBM copy
    # peak.  The library's 4-byte error flag comes from torch's caching
    # allocator, so no cudaMalloc sits between the events.
    import numpy as np
    nb_vol = int(np.prod([(x + 3) // 4 for x in wl["dims"]]))
    nb_all = min(nb_vol, 16 << 20)
    first = (nb_vol - nb_all) // 2      # centred on the middle z layer (the mixing layer)
    dec_ids = torch.arange(first, first + nb_all, dtype=torch.int64, device="cuda").to(torch.int32)
    dec_out = torch.empty((nb_all, 64), dtype=torch.float32, device="cuda")
    spr.use_torch_allocator()
    try:
        for _ in range(2):
            spr.spr_decode_blocks(comp, nb_vol, wl["rate"], ids=dec_ids, n=nb_all, out=dec_out, stream=stream)
        dec_times = []
        for i in range(5):
            flush.fill_(i & 255)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            spr.spr_decode_blocks(comp, nb_vol, wl["rate"], ids=dec_ids, n=nb_all, out=dec_out, stream=stream)
            b.record(stream)
            b.synchronize()
            dec_times.append(a.elapsed_time(b))
    finally:
        spr.spr_set_allocator()
    del dec_out, dec_ids
    ms_ = statistics.median(dec_times)
    gbs = nb_all * (decode_bytes_per_block(wl["rate"]) + 4) / 1e9 / (ms_ / 1e3)
    res["decode_all"] = {"kernel": "decode_list_kernel", "blocks": nb_all, "ms": round(ms_, 4),
                         "achieved": round(gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": round(gbs / pk["hbm_gbs"], 4), "first_block": first,
                         "bytes_per_block": decode_bytes_per_block(wl["rate"]) + 4,
                         "timing": "median of 5 CUDA-event timed calls, L2 flushed before each"}
    r.close()
    vol.close()
    return res


def summarise(wl, res, world):
    stats = res["stats"]
    n_pass = sum(rs["passes"] for rs, _ in stats)
    blocks = sum(rs["blocks_decoded"] for rs, _ in stats)
    entries = sum(rs["entries"] for rs, _ in stats) / max(1, len(stats))
    ie, ims = res["isect"]
    return {
        "ms_per_pass": round(res["ms_image"] * len(stats) / max(1, n_pass), 4),
        "passes_per_image": round(n_pass / len(stats), 2),
        "blocks_decoded_per_image": round(blocks / len(stats), 1),
        "decoded_gbs": round(res["decoded_gbs"], 1),
        "images_per_s": round(1e3 / res["ms_image"] * world, 2),
        "stage_ms_per_image": res["stage_ms_per_image"],
        "ms_per_pass_index": res["ms_per_pass_index"],
        "ray_block_tests_per_s": {
            "intersect_stage": round(ie / (ims / 1e3), 1) if ims > 0 else None,
            "whole_render": round(entries / (res["ms_image"] / 1e3), 1),
            "entries_per_image": round(entries, 1),
            "timing": "entries of the instrumented renders over their intersection stage time; "
                      "entries of the timed renders over their ms to the final image"},
        "gpu_launches": int(sum(rs["kernel_launches"] for rs, _ in stats)),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=128)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warm-s", type=float, default=2.0,
                    help="minimum seconds of warm-up renders (clock record under load)")
    ap.add_argument("--impl", default="spr", choices=["spr", "reference"])
    ap.add_argument("--workload", default="paper", choices=sorted(WORKLOADS))
    ap.add_argument("--dims", type=int, nargs=3, default=None,
                    help="override the workload's volume size (quick runs; the line names it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-medium", action="store_true",
                    help="skip the medium workload's sub-object in the paper-scale line")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--dump", default="", help="write per-pass details to this JSON file")
    ap.add_argument("--study", default="",
                    help="instead of the bench line: write the speculation sweep, resolution "
                         "scaling and decode-all-active comparison to this JSON file")
    ap.add_argument("--serve", default="",
                    help="instead of the bench line: run the render service on a Poisson request "
                         "trace and write latency percentiles to this JSON file")
    ap.add_argument("--learned", default="",
                    help="instead of the bench line: train the speculation policy on traces of the "
                         "workload and compare it with the plain rule on held-out poses")
    ap.add_argument("--learn-train", type=int, default=64)
    ap.add_argument("--learn-eval", type=int, default=32)
    ap.add_argument("--learn-mod", type=int, default=16)
    ap.add_argument("--learn-samples", type=int, default=24 << 20)
    ap.add_argument("--learn-epochs", type=int, default=8)
    ap.add_argument("--oracle-passes", action="store_true",
                    help="time the oracle's raycaster with visible lists and its pass simulator (host cores)")
    ap.add_argument("--decode-slab", action="store_true",
                    help="instead of the bench line: the decode rate of the paper-scale field's "
                         "interface blocks (one JSON line)")
    ap.add_argument("--batched", default="",
                    help="instead of the bench line: several volumes rendered by one graph launch against "
                         "the plain one-at-a-time loop on the serving mix (JSON to this file)")
    ap.add_argument("--batch-requests", type=int, default=96)
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--warp-walk", type=int, default=-1,
                    help="live-ray count below which a pass walks one ray per warp (-1: the library default)")
    ap.add_argument("--seg-lanes", type=int, default=-1,
                    help="lane budget of the segmented walk (-1: the library default, 0: off)")
    ap.add_argument("--isect-staged", action="store_true",
                    help="intersect from dual grids staged in shared memory (a variant; results unchanged)")
    ap.add_argument("--cache-mb", type=int, default=0,
                    help="override the workload's block-cache budget (MB; 0 keeps it)")
    ap.add_argument("--fixed-k", type=int, default=0,
                    help="fixed speculation count instead of the workload's rule (sweeps; 0 keeps it)")
    ap.add_argument("--k-max", type=int, default=0,
                    help="override the workload's speculation limit (k sweeps; 0 keeps it)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.dims:
        wl["dims"] = tuple(args.dims)
        wl["name"] = wl["name"].replace("2048x2048x1920", "x".join(map(str, args.dims))).replace(
            "512^3", "x".join(map(str, args.dims)))
    if args.cache_mb > 0:
        wl["cache_bytes"] = args.cache_mb << 20
        wl["name"] = re.sub(r"cache [^,]*", "cache %d MB" % args.cache_mb, wl["name"], count=1)
    if args.fixed_k > 0:
        wl["spec"], wl["k"] = "fixed", args.fixed_k
        wl["name"] = wl["name"].rsplit(", adaptive", 1)[0] + ", fixed k=%d" % args.fixed_k
    if args.k_max > 0:
        wl["k"] = args.k_max
        wl["name"] = wl["name"].rsplit("k<=", 1)[0] + f"k<={args.k_max}" if "k<=" in wl["name"] else wl["name"]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.oracle_passes:
        return run_oracle_passes(args, wl)
    if args.study:
        return run_study(args, wl)
    if args.serve:
        return run_serve(args)
    if args.learned:
        return run_learned(args, wl)
    if args.decode_slab:
        return run_decode_slab(args)
    if args.batched:
        return run_batched(args)
    if args.warmup < 3:
        args.warmup = 3

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2309_10212_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    import paper_2309_10212_gb300 as spr
    from paper_2309_10212_gb300 import _lib

    want_cpu = rank == 0 and not args.no_cpu_baseline
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # one generation of the raw volume feeds both encoders: the library's
        # (the GPU path's input) and, for the CPU baseline, the oracle's own
        comp, comp_host = compress_volume(wl, spr, torch, library=True, oracle_side=want_cpu)
        res = measure_workload(wl, args, spr, _lib, torch, stream, rank, world, dist, local, comp)
        del comp
        torch.cuda.empty_cache()
        med = None
        if wl["field"] == "mixing" and not args.no_medium and not args.dims:
            mwl = dict(WORKLOADS["medium"])
            mcomp = compress_volume(mwl, spr, torch)[0]
            margs = argparse.Namespace(**vars(args))
            margs.steps = max(16, min(args.steps, 64))
            med = measure_workload(mwl, margs, spr, _lib, torch, stream, rank, world, dist, local, mcomp,
                                   headline=False)
            del mcomp

    cpu = None
    if want_cpu:
        cb = cpu_baseline(wl, comp_host, pose(wl, 0))
        a, o = cb["all"], cb["one"]
        cpu = {"value": round(a["ms"], 1), "unit": "ms", "cores": a["threads"], "kind": "oracle",
               "sample": describe_sample(a, wl["W"], wl["H"]) + "; pose 0",
               "one_core": {"value": round(o["ms"], 1), "unit": "ms", "cores": 1,
                            "sample": describe_sample(o, wl["W"], wl["H"])},
               "input": "the oracle's own FRC4 encoding of the synth volume"}
        del comp_host
    elif rank == 0:
        cpu = {"value": None, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "not run (--no-cpu-baseline)"}

    if rank == 0:
        sm = summarise(wl, res, world)
        line = {
            "metric": METRIC,
            "value": round(res["ms_image"], 4),
            "unit": "ms",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(res["ms_image"], 4),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "dims": list(wl["dims"]), "rate": wl["rate"],
                       "image": [wl["W"], wl["H"]], "iso": wl["iso"],
                       "cache_bytes": wl["cache_bytes"],
                       "speculation": "%s k%s%d" % (wl["spec"], "<=" if wl["spec"] == "adaptive"
                                                    else "=", wl["k"]),
                       "cold_cache_per_step": True,
                       "l2": "256 MB buffer written between timed steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "ms_median": round(res["ms_image_median"], 4),
        }
        line.update({k: v for k, v in sm.items() if k != "gpu_launches"})
        line["roofline"] = res["roofline"]
        line["stage_roofline"] = res["stage_roofline"]
        line["decode_all"] = res["decode_all"]
        line["cpu_baseline"] = cpu
        line["e2e"] = res["e2e"]
        line["gpu_launches"] = sm["gpu_launches"]
        clocks = res["clocks"]
        if clocks:
            clocks["window"] = ("nvidia-smi every 50 ms from the first warm-up render (%d renders, "
                                ">= %.1f s) to the end of the timed renders" % (res["warmup_renders"], args.warm_s))
        line["clocks"] = clocks
        if med is not None:
            msm = summarise(WORKLOADS["medium"], med, world)
            line["medium"] = {"workload": WORKLOADS["medium"]["name"], "ms": round(med["ms_image"], 4),
                              "steps": len(med["stats"]),
                              "passes_per_image": msm["passes_per_image"], "ms_per_pass": msm["ms_per_pass"],
                              "blocks_decoded_per_image": msm["blocks_decoded_per_image"],
                              "decoded_gbs": msm["decoded_gbs"], "stage_ms_per_image": msm["stage_ms_per_image"],
                              "ms_per_pass_index": msm["ms_per_pass_index"],
                              "roofline": med["roofline"], "stage_roofline": med["stage_roofline"],
                              "gpu_launches": msm["gpu_launches"]}
        print(json.dumps(line))
        if args.dump:
            json.dump({"line": line, "steps": [{"render": rs, "passes": ps} for rs, ps in res["stats"]],
                       "profiled": [{"render": rs, "passes": ps} for rs, ps in res["prof_stats"]]},
                      open(args.dump, "w"), indent=1)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
