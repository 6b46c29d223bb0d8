#!/usr/bin/env python
"""Benchmark of the sort-last compositing hot path on GB300.

Default workload (one "step", the thesis's large-frame sort-last case, 5.2.1 and
5.3): 64 partial images of a 7680x4320 frame, RGBA8 + float32 depth, ~25%
coverage each, clustered and stored cropped to their ROI; every source's colour
(swizzled, mode 2) and depth (mode 1) is RLE-compressed (5.5.1), the 128
streams are decompressed, and the 64 decompressed sources are depth-composited
into the frame.  Inputs are resident in HBM when a step starts; L2 is flushed
between timed steps, outside the timed events: 2x its size is written, then
another 2x its size is read, so that the timed step neither finds its inputs in
L2 nor pays for writing back the flush's lines.  Step times are medians.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ec|reference]
                    [--workload cfg5d|cfg1|cfg2|cfg3|cfg3h|cfg3fused|cfg3hfused|cfg4|cfg5a|cfg5afused|cfg5afusedq|roi2|asm4k|sched2|rle0|rle0big|yuv2]
                    [--sources S]

The default line also carries, measured in the same run: the 16 x 1920x1080
pipeline (secondary), the 1000 uneven tiles batched against per-tile launches,
and the alpha forward / backward / fused forward+backward ratios at 32 x 2048^2
(FP32 and FP16) and 128 x 3840x2160 (FP16).  --sources S keeps only the first
S sources of a depth workload (small cases for profiling).

Prints ONE JSON line (rank 0).  Metric: composited Gpixel-layers/s (sum over
sources of |roi_i ∩ frame| per step, divided by the step time).  With N > 1
(launched by torch.distributed.run) each rank runs an independent replica of
the workload on its own GPU ("replicas only": nothing is exchanged), value is
all ranks' pixel-layers over the slowest rank's time.

--impl reference times the CPU oracle (test infrastructure, plain C) on the
same workload on the host cores, as the reference arm.
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
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "composited Gpixel-layers/s"
UNIT = "Gpixel-layers/s"
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ec", choices=["ec", "reference"])
    p.add_argument("--workload", default="cfg5d")
    p.add_argument("--sources", type=int, default=0,
                   help="depth workloads: keep only the first S sources (0 = all)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the secondary workloads measured beside the default one")
    p.add_argument("--oracle-single-core", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


# ----------------------------------------------------------------- plumbing


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local):
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, ms_slowest: float, world: int) -> float:
    """Throughput of the whole job in G units/s: every rank processes
    units_per_rank per step, and a step lasts as long as the slowest rank."""
    return world * units_per_rank / (ms_slowest * 1e-3) / 1e9


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
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
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# Source files each measured kernel is built from (its traffic record stays
# valid while they are unchanged); kernels not listed hash every source.
KERNEL_SOURCES = {
    "rle_compress": ["k_rle.cu", "rle_codec.cuh", "ec_internal.cuh"],
    "rle_decompress": ["k_rle.cu", "rle_codec.cuh", "ec_internal.cuh"],
    "composite_depth": ["k_composite.cu", "composite_body.cuh", "ec_internal.cuh"],
    "composite_alpha": ["k_composite.cu", "composite_body.cuh", "ec_internal.cuh"],
    "composite_alpha_fwd_bwd": ["k_backward.cu", "ec_internal.cuh"],
    "batch": ["k_batch.cu", "composite_body.cuh", "ec_internal.cuh"],
}


def kernel_hash(kernel: str = "") -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_08755_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(csrc))
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the kernel's current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload][kernel]
        if e.get("source_hash") == kernel_hash(kernel):
            return float(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


# ---------------------------------------------------------------- workloads


class DepthPipeline:
    """cfg1 / cfg2 / cfg5d: RLE compress -> decompress -> depth composite."""

    def __init__(self, cfg, n, W, H, coverage, clustered, cropped, device, keep=0):
        import paper_1902_08755_gb300 as ec
        import synthetic as S
        self.ec = ec
        self.W, self.H, self.cfg = W, H, cfg
        self.n = min(n, keep) if keep > 0 else n
        self.n_total = n
        who = f"{n} sources" if self.n == n else f"the first {self.n} of {n} sources"
        self.desc = (f"{who} {W}x{H} RGBA8+Z32, ~{int(coverage * 100)}% coverage, "
                     f"{'ROI-cropped' if cropped else 'uncropped'}; RLE compress (colour mode 2, "
                     f"depth mode 1) -> decompress -> depth composite")
        self.srcs = [S.depth_source(W, H, coverage, cfg, i, clustered=clustered, cropped=cropped, device=device)
                     for i in range(self.n)]
        self.planes = []
        for s in self.srcs:
            self.planes.append((s.color, 2))
            self.planes.append((s.depth.view(torch.uint32), 1))
        self.units = sum(max(0, min(s.roi[2], W)) * max(0, min(s.roi[3], H)) for s in self.srcs)
        self.stored_px = sum(s.pvp[2] * s.pvp[3] for s in self.srcs)
        self.kernels = ["rle_compress", "rle_decompress", "composite_depth"]
        if torch.device(device).type != "cuda":
            return
        self.ctx = ec.default_context(torch.device(device).index or 0)
        self.bufs = [torch.empty(ec.rle_max_size(t.shape[1], t.shape[0]), dtype=torch.uint8, device=device)
                     for t, _ in self.planes]
        self.sizes = [torch.zeros(1, dtype=torch.uint64, device=device) for _ in self.planes]
        self.dec = [torch.empty_like(t) for t, _ in self.planes]
        self.imgs = [ec.Image(color=self.dec[2 * i], depth=self.dec[2 * i + 1].view(torch.float32),
                              pvp=s.pvp, roi=s.roi) for i, s in enumerate(self.srcs)]
        self.out_c = torch.empty((H, W), dtype=torch.int32, device=device).view(torch.uint32)
        self.out_d = torch.empty((H, W), dtype=torch.float32, device=device)
        self.cjobs = [(t, m, None, b, sz) for (t, m), b, sz in zip(self.planes, self.bufs, self.sizes)]
        # the batched codec calls' argument arrays are built once
        self.comp, _ = ec.prepare_rle_compress_batch(self.cjobs, ctx=self.ctx)
        self.decomp, _ = ec.prepare_rle_decompress_batch([(b, t.shape[1], t.shape[0], d, None)
                                                          for b, (t, _), d in zip(self.bufs, self.planes, self.dec)],
                                                         ctx=self.ctx)

    def step(self, ev=None):
        ec = self.ec
        if ev:
            ev[0].record()
        self.comp.run()
        if ev:
            ev[1].record()
        self.decomp.run()
        if ev:
            ev[2].record()
        ec.composite_depth(self.imgs, self.out_c, self.out_d, ctx=self.ctx)
        if ev:
            ev[3].record()

    def launches_per_step(self):
        return 7                             # compress: five kernels; decompress; merge

    def compressed_bytes(self):
        return sum(int(s.item()) for s in self.sizes)

    def algorithmic_bytes(self):
        comp = self.compressed_bytes()
        raw = 8 * self.stored_px
        return {"rle_compress": raw + comp, "rle_decompress": comp + raw,
                "composite_depth": 8 * self.units + 8 * self.W * self.H}

    # end to end: sources from pinned host memory, frame back to pinned host
    # memory.  The sources are copied in four parts on a copy stream; each
    # part is compressed and decoded as soon as it has landed, so the codec
    # overlaps the copies of the later parts.
    E2E_PARTS = 4

    def setup_e2e(self):
        ec = self.ec
        self.h_planes = [t.view(torch.int32).cpu().pin_memory() for t, _ in self.planes]
        self.h_out = torch.empty((self.H, self.W), dtype=torch.int32).pin_memory()
        self.h_outd = torch.empty((self.H, self.W), dtype=torch.float32).pin_memory()
        self.h2d = sum(t.numel() * 4 for t in self.h_planes)
        self.d2h = self.H * self.W * 8
        self.copy_stream = torch.cuda.Stream()
        P = self.E2E_PARTS
        bounds = [2 * ((len(self.planes) // 2) * k // P) for k in range(P + 1)]   # whole sources per part
        self.parts = []
        for k in range(P):
            lo, hi = bounds[k], bounds[k + 1]
            if hi <= lo:
                continue
            comp, _ = ec.prepare_rle_compress_batch(self.cjobs[lo:hi], ctx=self.ctx)
            dec, _ = ec.prepare_rle_decompress_batch([(self.bufs[i], self.planes[i][0].shape[1],
                                                       self.planes[i][0].shape[0], self.dec[i], None)
                                                      for i in range(lo, hi)], ctx=self.ctx)
            self.parts.append((lo, hi, comp, dec, torch.cuda.Event()))
        self.ev_start = torch.cuda.Event()

    def e2e_step(self):
        cur = torch.cuda.current_stream()
        self.ev_start.record(cur)
        self.copy_stream.wait_event(self.ev_start)
        with torch.cuda.stream(self.copy_stream):
            for lo, hi, _, _, ev in self.parts:
                for i in range(lo, hi):
                    self.planes[i][0].view(torch.int32).copy_(self.h_planes[i], non_blocking=True)
                ev.record(self.copy_stream)
        for lo, hi, comp, dec, ev in self.parts:
            cur.wait_event(ev)
            comp.run()
            dec.run()
        self.ec.composite_depth(self.imgs, self.out_c, self.out_d, ctx=self.ctx)
        self.h_out.copy_(self.out_c.view(torch.int32), non_blocking=True)
        self.h_outd.copy_(self.out_d, non_blocking=True)

    # oracle (reference arm / cpu baseline): same pipeline on the host cores
    def oracle_step(self, pool, cores, k=0):
        """The same pipeline on the host cores, over the first k sources (all
        when k is 0): each plane's codec calls on a pool thread, then the
        composite of those sources in row bands.  Sets sample_units."""
        import oracle
        k = min(k, self.n) if k > 0 else self.n
        if getattr(self, "_host_k", None) != k:
            self._host = [(t.view(torch.int32).cpu().numpy().view(np.uint32), m) for t, m in self.planes[:2 * k]]
            self._host_k = k
        host = self._host
        self.sample_units = sum(max(0, min(s.roi[2], self.W)) * max(0, min(s.roi[3], self.H))
                                for s in self.srcs[:k])
        self.sample_desc = ("full steps" if k == self.n_total else
                            f"the first {k} of the {self.n_total} sources (codec of their planes, "
                            f"composite of those sources over the whole frame)")
        t0 = time.perf_counter()
        streams = list(pool.map(lambda a: oracle.rle_compress(a[0], a[1]), host))
        dec = list(pool.map(lambda a: oracle.rle_decompress(a[0], a[1][0].shape[1], a[1][0].shape[0]),
                            zip(streams, host)))
        imgs = [oracle.Image(s.pvp, s.roi, dec[2 * i], dec[2 * i + 1].view(np.float32))
                for i, s in enumerate(self.srcs[:k])]
        bands = np.linspace(0, self.H, cores + 1).astype(int)

        def part(b):
            y0, y1 = int(bands[b]), int(bands[b + 1])
            return oracle.composite_depth(imgs, (0, y0, self.W, y1 - y0))
        list(pool.map(part, range(cores)))
        return time.perf_counter() - t0


class CodecPipeline:
    """The cfg2 sources (16 x 1920x1080 RGBA8+Z32, cropped) through the other
    compressors of thesis 5.5, then decoded and depth-composited:
      rle0: basic 64-bit RLE (mode 0) for colour and depth;
      yuv2: colour through the lossy YUV compressor and RLE mode 1, depth mode 1;
      rle0big: mode 0 on the 64 x 7680x4320 sources of cfg5d (~25% coverage),
      a size at which every coding warp has many chunks."""

    def __init__(self, kind, device):
        import paper_1902_08755_gb300 as ec
        import synthetic as S
        self.ec, self.kind = ec, kind
        big = kind == "rle0big"
        cfg, cov = (5, 0.25) if big else (2, 0.3)
        self.W, self.H, self.n = (7680, 4320, 64) if big else (1920, 1080, 16)
        self.yuv = kind == "yuv2"
        self.desc = (f"{self.n} sources {self.W}x{self.H} RGBA8+Z32, ~{int(cov * 100)}% coverage, ROI-cropped; "
                     + ("colour YUV 4:2:0 (BT.601 fixed point) + RLE mode 1, depth RLE mode 1"
                        if self.yuv else "basic 64-bit RLE (mode 0) for colour and depth")
                     + " -> decode -> depth composite")
        self.srcs = S.depth_sources(cfg, self.n, self.W, self.H, cov, clustered=True, cropped=True, device=device)
        self.units = sum(max(0, min(s.roi[2], self.W)) * max(0, min(s.roi[3], self.H)) for s in self.srcs)
        self.stored_px = sum(s.pvp[2] * s.pvp[3] for s in self.srcs)
        self.kernels = (["yuv_encode", "rle_compress", "rle_decompress", "yuv_decode", "composite_depth"]
                        if self.yuv else ["rle_compress", "rle_decompress", "composite_depth"])
        if torch.device(device).type != "cuda":
            return
        self.ctx = ec.default_context(torch.device(device).index or 0)
        self.packed = [torch.empty(ec.yuv_packed_shape(s.pvp[2], s.pvp[3]), dtype=torch.int32,
                                   device=device).view(torch.uint32) for s in self.srcs] if self.yuv else []
        self.planes = []
        for i, s in enumerate(self.srcs):
            self.planes.append((self.packed[i], 1) if self.yuv else (s.color, 0))
            self.planes.append((s.depth.view(torch.uint32), 1 if self.yuv else 0))
        self.bufs = [torch.empty(ec.rle_max_size(t.shape[1], t.shape[0]), dtype=torch.uint8, device=device)
                     for t, _ in self.planes]
        self.sizes = [torch.zeros(1, dtype=torch.uint64, device=device) for _ in self.planes]
        self.dec = [torch.empty_like(t) for t, _ in self.planes]
        self.colour = [torch.empty_like(s.color) for s in self.srcs] if self.yuv else [self.dec[2 * i] for i in range(self.n)]
        self.imgs = [ec.Image(color=self.colour[i], depth=self.dec[2 * i + 1].view(torch.float32),
                              pvp=s.pvp, roi=s.roi) for i, s in enumerate(self.srcs)]
        self.out_c = torch.empty((self.H, self.W), dtype=torch.int32, device=device).view(torch.uint32)
        self.out_d = torch.empty((self.H, self.W), dtype=torch.float32, device=device)
        self.cjobs = [(t, m, None, b, sz) for (t, m), b, sz in zip(self.planes, self.bufs, self.sizes)]
        if self.yuv:
            self.enc = ec.prepare_yuv_batch([(s.color, p, s.pvp[2], s.pvp[3]) for s, p in zip(self.srcs, self.packed)],
                                            True, ctx=self.ctx)
            self.ydec = ec.prepare_yuv_batch([(self.dec[2 * i], self.colour[i], s.pvp[2], s.pvp[3])
                                              for i, s in enumerate(self.srcs)], False, ctx=self.ctx)
        self.comp, _ = ec.prepare_rle_compress_batch(self.cjobs, ctx=self.ctx)
        self.decomp, _ = ec.prepare_rle_decompress_batch([(b, t.shape[1], t.shape[0], d, None)
                                                          for b, (t, _), d in zip(self.bufs, self.planes, self.dec)],
                                                         ctx=self.ctx)

    def step(self, ev=None):
        ec = self.ec
        k = 0
        if ev:
            ev[0].record()
        if self.yuv:
            self.enc.run()
            k += 1
            if ev:
                ev[k].record()
        self.comp.run()
        k += 1
        if ev:
            ev[k].record()
        self.decomp.run()
        k += 1
        if ev:
            ev[k].record()
        if self.yuv:
            self.ydec.run()
            k += 1
            if ev:
                ev[k].record()
        ec.composite_depth(self.imgs, self.out_c, self.out_d, ctx=self.ctx)
        if ev:
            ev[k + 1].record()

    def launches_per_step(self):
        return 9 if self.yuv else 7          # compress: five kernels

    def compressed_bytes(self):
        return sum(int(s.item()) for s in self.sizes)

    def raw_bytes(self):
        return sum(4 * t.numel() for t, _ in self.planes)

    def algorithmic_bytes(self):
        comp = self.compressed_bytes()
        raw = self.raw_bytes()
        out = {"rle_compress": raw + comp, "rle_decompress": comp + raw,
               "composite_depth": 8 * self.units + 8 * self.W * self.H}
        if self.yuv:
            packed = sum(4 * p.numel() for p in self.packed)
            out["yuv_encode"] = 4 * self.stored_px + packed
            out["yuv_decode"] = packed + 4 * self.stored_px
        return out

    def setup_e2e(self):
        self.h_c = [s.color.view(torch.int32).cpu().pin_memory() for s in self.srcs]
        self.h_d = [s.depth.cpu().pin_memory() for s in self.srcs]
        self.h_out = torch.empty((self.H, self.W), dtype=torch.int32).pin_memory()
        self.h_outd = torch.empty((self.H, self.W), dtype=torch.float32).pin_memory()
        self.h2d = sum(t.numel() * 4 for t in self.h_c + self.h_d)
        self.d2h = self.H * self.W * 8

    def e2e_step(self):
        for s, hc, hd in zip(self.srcs, self.h_c, self.h_d):
            s.color.view(torch.int32).copy_(hc, non_blocking=True)
            s.depth.copy_(hd, non_blocking=True)
        self.step()
        self.h_out.copy_(self.out_c.view(torch.int32), non_blocking=True)
        self.h_outd.copy_(self.out_d, non_blocking=True)

    def oracle_step(self, pool, cores):
        import oracle
        if not hasattr(self, "_host"):
            self._host = [(s.color.view(torch.int32).cpu().numpy().view(np.uint32), s.depth.cpu().numpy())
                          for s in self.srcs]
        t0 = time.perf_counter()

        def codec(a):
            c, d = a
            w, h = c.shape[1], c.shape[0]
            if self.yuv:
                p = oracle.yuv_encode(c)
                p = oracle.rle_decompress(oracle.rle_compress(p, 1), p.shape[1], p.shape[0])
                c2 = oracle.yuv_decode(p, w, h)
                d2 = oracle.rle_decompress(oracle.rle_compress(d.view(np.uint32), 1), w, h)
            else:
                c2 = oracle.rle_decompress(oracle.rle_compress(c, 0), w, h)
                d2 = oracle.rle_decompress(oracle.rle_compress(d.view(np.uint32), 0), w, h)
            return c2, d2.view(np.float32)
        dec = list(pool.map(codec, self._host))
        imgs = [oracle.Image(s.pvp, s.roi, c, d) for s, (c, d) in zip(self.srcs, dec)]
        bands = np.linspace(0, self.H, cores + 1).astype(int)

        def part(k):
            y0, y1 = int(bands[k]), int(bands[k + 1])
            return oracle.composite_depth(imgs, (0, y0, self.W, y1 - y0))
        list(pool.map(part, range(cores)))
        return time.perf_counter() - t0


class AlphaForward:
    """cfg3 / cfg3h / cfg5a: ordered front-to-back 'over' of L layers."""

    def __init__(self, cfg, L, W, H, amax, dtype, device):
        import paper_1902_08755_gb300 as ec
        import synthetic as S
        self.ec = ec
        self.W, self.H, self.L = W, H, L
        self.desc = f"{L} layers {W}x{H} premultiplied RGBA {'FP16' if dtype == torch.float16 else 'FP32'} storage, alpha in [0,{amax}]; ordered 'over' forward"
        self.lay = S.alpha_layers(cfg, L, W, H, amax, dtype=dtype, device=device)
        self.units = L * W * H
        self.bpp = 16 if dtype == torch.float32 else 8
        self.kernels = ["composite_alpha"]
        if torch.device(device).type != "cuda":
            return
        self.imgs = [ec.Image(color=self.lay[k]) for k in range(L)]
        self.out = torch.empty((H, W, 4), dtype=dtype, device=device)
        self.ctx = ec.default_context(torch.device(device).index or 0)

    def step(self, ev=None):
        if ev:
            ev[0].record()
        self.ec.composite_alpha(self.imgs, self.out, ctx=self.ctx)
        if ev:
            ev[1].record()

    def launches_per_step(self):
        return 1

    def algorithmic_bytes(self):
        return {"composite_alpha": self.units * self.bpp + self.W * self.H * self.bpp}

    def setup_e2e(self):
        self.h_lay = self.lay.cpu().pin_memory()
        self.h_out = torch.empty_like(self.out, device="cpu").pin_memory()
        self.h2d = self.h_lay.numel() * self.h_lay.element_size()
        self.d2h = self.h_out.numel() * self.h_out.element_size()

    def e2e_step(self):
        self.lay.copy_(self.h_lay, non_blocking=True)
        self.step()
        self.h_out.copy_(self.out, non_blocking=True)

    def oracle_step(self, pool, cores):
        import oracle
        rows = max(1, min(self.H, 16))       # bounded sample: the first rows
        host = self.lay[:, :rows].cpu().numpy()
        t0 = time.perf_counter()
        bands = np.linspace(0, rows, min(cores, rows) + 1).astype(int)

        def part(k):
            y0, y1 = int(bands[k]), int(bands[k + 1])
            ims = [oracle.Image((0, y0, self.W, y1 - y0), (0, y0, self.W, y1 - y0),
                                np.ascontiguousarray(host[j, y0:y1])) for j in range(self.L)]
            return oracle.composite_alpha(ims, (0, y0, self.W, y1 - y0))
        list(pool.map(part, range(len(bands) - 1)))
        self.sample_fraction = rows / self.H
        return (time.perf_counter() - t0) / self.sample_fraction


class AlphaFused(AlphaForward):
    """cfg3fused / cfg3hfused / cfg5afused: forward and the gradient of
    L = sum(w * out) with respect to every layer, in one kernel pass."""

    def __init__(self, cfg, L, W, H, amax, dtype, device):
        super().__init__(cfg, L, W, H, amax, dtype, device)
        import synthetic as S
        self.desc = self.desc.replace("ordered 'over' forward", "fused forward + backward of sum(w * out)")
        self.w = S.grad_weights(cfg, W, H, device=device)
        self.kernels = ["composite_alpha_fwd_bwd"]
        if torch.device(device).type != "cuda":
            return
        self.grads = [torch.empty_like(self.lay[k]) for k in range(L)]

    def step(self, ev=None):
        if ev:
            ev[0].record()
        self.ec.composite_alpha_fwd_bwd(self.imgs, self.out, self.w, self.grads, ctx=self.ctx)
        if ev:
            ev[1].record()

    def algorithmic_bytes(self):
        px = self.W * self.H
        return {"composite_alpha_fwd_bwd": 2 * self.units * self.bpp + px * 16 + px * self.bpp}

    def setup_e2e(self):
        super().setup_e2e()
        self.h_w = self.w.cpu().pin_memory()
        self.h2d += self.h_w.numel() * 4

    def e2e_step(self):
        self.lay.copy_(self.h_lay, non_blocking=True)
        self.w.copy_(self.h_w, non_blocking=True)
        self.step()
        self.h_out.copy_(self.out, non_blocking=True)


class RoiDetect:
    """roi2: automatic ROI (thesis 5.3) of the 16 uncropped 1920x1080 sources of
    the depth pipeline: every depth buffer is scanned for pixels below the
    cleared depth, giving each source's bounding box and 64-px tile occupancy
    grid (holes), all in one launch."""

    def __init__(self, cfg, n, W, H, coverage, device, tile=64):
        import ctypes as C

        import paper_1902_08755_gb300 as ec
        from paper_1902_08755_gb300 import _abi as A
        import synthetic as S
        self.ec = ec
        self.W, self.H, self.n, self.tile = W, H, n, tile
        self.desc = (f"{n} uncropped sources {W}x{H} (~{int(coverage * 100)}% coverage, clustered): "
                     f"bounding box of depth < 1 and {tile}-px occupancy grids, one launch")
        self.srcs = S.depth_sources(cfg, n, W, H, coverage, clustered=True, device=device)
        self.units = n * W * H
        self.kernels = ["detect_roi"]
        self.gw, self.gh = -(-W // tile), -(-H // tile)
        if torch.device(device).type != "cuda":
            return
        self.ctx = ec.default_context(torch.device(device).index or 0)
        self.rois = torch.zeros((n, 4), dtype=torch.int32, device=device)
        self.grids = [torch.empty((self.gh, self.gw), dtype=torch.uint8, device=device) for _ in range(n)]
        # the C entry point with arguments marshalled once
        self._arr = (A.ec_image * n)(*[A.ec_image(A.ec_rect(0, 0, W, H), A.ec_rect(0, 0, W, H), W, A.EC_RGBA8,
                                                  s.color.data_ptr(), s.depth.data_ptr()) for s in self.srcs])
        self._occ = (C.c_void_p * n)(*[g.data_ptr() for g in self.grids])
        self._fn = A.load().ec_detect_roi

    def step(self, ev=None):
        if ev:
            ev[0].record()
        rc = self._fn(self.ctx.h, self._arr, self.n, self.tile, self._occ, self.rois.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
        if rc:
            raise SystemExit(f"ec_detect_roi failed: {rc}")
        if ev:
            ev[1].record()

    def launches_per_step(self):
        return 2                             # the depth kind's scan, then the finalize kernel

    def algorithmic_bytes(self):
        return {"detect_roi": 4 * self.units + self.n * (self.gw * self.gh + 16)}

    def setup_e2e(self):
        self.h_depth = [s.depth.cpu().pin_memory() for s in self.srcs]
        self.h_rois = torch.empty((self.n, 4), dtype=torch.int32).pin_memory()
        self.h2d = 4 * self.units
        self.d2h = self.n * 16

    def e2e_step(self):
        for s, h in zip(self.srcs, self.h_depth):
            s.depth.copy_(h, non_blocking=True)
        self.step()
        self.h_rois.copy_(self.rois, non_blocking=True)

    def oracle_step(self, pool, cores):
        import oracle
        host = [s.depth.cpu().numpy() for s in self.srcs[:min(self.n, cores)]]
        t0 = time.perf_counter()
        full = (0, 0, self.W, self.H)
        list(pool.map(lambda d: oracle.detect_roi(full, full, self.W, 0, depth=d, tile=self.tile), host))
        self.sample_fraction = len(host) / self.n
        self.sample_desc = f"{len(host)} of the {self.n} sources"
        return (time.perf_counter() - t0) / self.sample_fraction


class Assembly:
    """asm4k: the assembly steps of the other compound modes (thesis 4.2) on a
    3840x2160 RGBA8 frame: a sort-first frame from 8 x 8 tiles, a 2 x 2 pixel
    compound from 4 interleaved sources, and the average of 8 subpixel samples."""

    def __init__(self, W, H, device, nt=8, kern=(2, 2), ns=8):
        import ctypes as C

        import paper_1902_08755_gb300 as ec
        from paper_1902_08755_gb300 import _abi as A
        from paper_1902_08755_gb300 import api
        self.ec = ec
        self.W, self.H = W, H
        self.desc = (f"{W}x{H} RGBA8: sort-first frame from {nt}x{nt} tiles, {kern[0]}x{kern[1]} pixel "
                     f"compound, average of {ns} subpixel samples")
        self.kernels = ["assemble_tiles", "assemble_pixels", "average"]
        self.units = W * H * (2 + ns)                   # source pixels read per step
        self.bytes = {"assemble_tiles": 8 * W * H, "assemble_pixels": 8 * W * H, "average": 4 * W * H * (ns + 1)}
        if torch.device(device).type != "cuda":
            return
        g = torch.Generator(device=device)
        g.manual_seed(190208755)
        rnd = lambda h, w: torch.randint(-2 ** 31, 2 ** 31 - 1, (h, w), generator=g, dtype=torch.int32,
                                         device=device).view(torch.uint32)
        self.ctx = ec.default_context(torch.device(device).index or 0)
        dev = self.ctx.device
        self.out = [torch.empty((H, W), dtype=torch.int32, device=device).view(torch.uint32) for _ in range(3)]
        tw, th = -(-W // nt), -(-H // nt)
        tiles = []
        for j in range(nt):
            for i in range(nt):
                r = (i * tw, j * th, min(tw, W - i * tw), min(th, H - j * th))
                tiles.append(ec.Image(color=rnd(r[3], r[2]), pvp=r, roi=r))
        nx, ny = kern
        pix = [rnd(-(-(H - ky) // ny), -(-(W - kx) // nx)) for ky in range(ny) for kx in range(nx)]
        offs = [(kx, ky) for ky in range(ny) for kx in range(nx)]
        samples = [ec.Image(color=rnd(H, W)) for _ in range(ns)]
        self._keep = (tiles, pix, samples)
        lib = A.load()
        arr_t = (A.ec_image * len(tiles))(*[api._image_struct(im, dev, False) for im in tiles])
        arr_p = (A.ec_image * len(pix))(*[A.ec_image(A.ec_rect(0, 0, t.shape[1], t.shape[0]),
                                                     A.ec_rect(0, 0, t.shape[1], t.shape[0]), t.shape[1],
                                                     A.EC_RGBA8, t.data_ptr(), None) for t in pix])
        kx = (C.c_int32 * len(offs))(*[o[0] for o in offs])
        ky = (C.c_int32 * len(offs))(*[o[1] for o in offs])
        arr_s = (A.ec_image * ns)(*[api._image_struct(im, dev, False) for im in samples])
        tg = [api._target(o, None, None, dev) for o in self.out]
        self._calls = [(lib.ec_assemble_tiles, (self.ctx.h, arr_t, len(tiles), C.byref(tg[0]))),
                       (lib.ec_assemble_pixels, (self.ctx.h, arr_p, kx, ky, len(pix), nx, ny, C.byref(tg[1]))),
                       (lib.ec_average, (self.ctx.h, arr_s, ns, C.byref(tg[2])))]
        self._args = (arr_t, arr_p, arr_s, kx, ky, tg)

    def step(self, ev=None):
        st = torch.cuda.current_stream().cuda_stream
        for i, (fn, args) in enumerate(self._calls):
            if ev:
                ev[i].record()
            rc = fn(*args, st)
            if rc:
                raise SystemExit(f"assembly call {i} failed: {rc}")
        if ev:
            ev[len(self._calls)].record()

    def launches_per_step(self):
        return 3

    def algorithmic_bytes(self):
        return dict(self.bytes)

    def setup_e2e(self):
        tiles, pix, samples = self._keep
        self._dev_in = [im.color for im in tiles] + list(pix) + [im.color for im in samples]
        self._host_in = [t.cpu().pin_memory() for t in self._dev_in]
        self._host_out = [o.cpu().pin_memory() for o in self.out]
        self.h2d = sum(t.numel() * 4 for t in self._dev_in)
        self.d2h = sum(o.numel() * 4 for o in self.out)

    def e2e_step(self):
        for d, h in zip(self._dev_in, self._host_in):
            d.copy_(h, non_blocking=True)
        self.step()
        for h, o in zip(self._host_out, self.out):
            h.copy_(o, non_blocking=True)

    def oracle_step(self, pool, cores):
        import oracle
        rows, ns = 16, 8                                 # bounded sample: a 16-row band of the average
        r = np.random.default_rng(190208755)
        band = [oracle.Image((0, 0, self.W, rows), (0, 0, self.W, rows),
                             r.integers(0, 2 ** 32, (rows, self.W), dtype=np.uint64).astype(np.uint32))
                for _ in range(ns)]
        t0 = time.perf_counter()
        oracle.average(band, (0, 0, self.W, rows), 0)
        self.sample_fraction = rows / self.H * (ns / (ns + 2))
        self.sample_desc = f"a {rows}-row band of the average"
        return (time.perf_counter() - t0) / self.sample_fraction


class Schedules:
    """sched2: a multi-stage compositing schedule (thesis 5.2.2, 5.2.3) over the
    cfg2 sources (16 x 1920x1080 RGBA8+Z32, cropped): binary swap, transfers
    RLE-compressed, every stage a fused decode-and-merge; the whole schedule
    is one CUDA graph.  The other schedules and variants are timed beside it."""

    OTHERS = [("binary_swap", "rle"), ("binary_swap", "raw"), ("direct_send", "rle"),
              ("direct_send", "raw"), ("two_three_swap", "fused"), ("stream", "fused")]
    VARIANTS = {"fused": dict(rle=True, fused=True), "rle": dict(rle=True, fused=False),
                "raw": dict(rle=False, fused=False)}

    def __init__(self, device, algo="binary_swap", variant="fused"):
        import paper_1902_08755_gb300 as ec
        import synthetic as S
        self.ec = ec
        self.W, self.H, self.n = 1920, 1080, 16
        self.algo, self.variant = algo, variant
        self.desc = (f"{self.n} sources {self.W}x{self.H} RGBA8+Z32, ~30% coverage, ROI-cropped; {algo} "
                     f"schedule, {variant} transfers ({'RLE colour mode 2 / depth mode 1, decoded inside the merge' if variant == 'fused' else variant}); one CUDA graph per step")
        self.srcs = S.depth_sources(2, self.n, self.W, self.H, 0.3, clustered=True, cropped=True, device=device)
        self.units = sum(max(0, min(s.roi[2], self.W)) * max(0, min(s.roi[3], self.H)) for s in self.srcs)
        self.stored_px = sum(s.pvp[2] * s.pvp[3] for s in self.srcs)
        if torch.device(device).type != "cuda":
            self.kernels = []
            return
        self.ctx = ec.default_context(torch.device(device).index or 0)
        self.imgs = [ec.Image(color=s.color, depth=s.depth, pvp=s.pvp, roi=s.roi) for s in self.srcs]
        self.out_c = torch.empty((self.H, self.W), dtype=torch.int32, device=device).view(torch.uint32)
        self.out_d = torch.empty((self.H, self.W), dtype=torch.float32, device=device)
        self.sch = self._plan(algo, variant)
        self.launch_list = self.sch.launches()
        self.kernels = [f"L{lv}:{kind}" for lv, kind, _ in self.launch_list]
        self.kind_of = [kind for _, kind, _ in self.launch_list]

    def _plan(self, algo, variant):
        return self.ec.Schedule("depth", algo, self.imgs, self.out_c, self.out_d, ctx=self.ctx,
                                **self.VARIANTS[variant])

    def step(self, ev=None):
        """Launch by launch, an event after each (for the per-kernel times)."""
        if ev is None:
            self.sch.run()
            return
        ev[0].record()
        for i in range(len(self.launch_list)):
            self.sch.run_launch(i)
            ev[i + 1].record()

    def graph_step(self):
        self.sch.run()

    def launches_per_step(self):
        return len(self.launch_list)

    def compressed_bytes(self):
        if self.variant == "raw":
            return 0
        return sum(c + d for c, d in self.sch.stream_sizes())

    def algorithmic_bytes(self):
        out = {}
        for _, kind, b in self.launch_list:
            out[kind] = out.get(kind, 0) + b
        if self.variant != "raw":
            for m, (c, d) in zip(self.sch.messages(), self.sch.stream_sizes()):
                out["rle_compress"] = out.get("rle_compress", 0) + c + d          # streams written
                k = "fused_depth" if m[3] else "rle_decompress"                  # streams read
                out[k] = out.get(k, 0) + c + d
        return out

    def others(self, flush, reps=30):
        res = {}
        for algo, variant in [(self.algo, self.variant)] + self.OTHERS:
            sch = self._plan(algo, variant)
            ms = _timed(sch.run, flush, reps)
            info = sch.info()
            comp = 0 if variant == "raw" else sum(c + d for c, d in sch.stream_sizes())
            res[f"{algo}/{variant}"] = {"ms": ms, "gpixel_layers_s": self.units / (ms * 1e-3) / 1e9,
                                        "levels": info["levels"], "transfers": info["messages"],
                                        "launches": info["launches"], "compressed_bytes": comp}
            sch.close()
        return res

    def setup_e2e(self):
        self.h_c = [s.color.view(torch.int32).cpu().pin_memory() for s in self.srcs]
        self.h_d = [s.depth.cpu().pin_memory() for s in self.srcs]
        self.h_out = torch.empty((self.H, self.W), dtype=torch.int32).pin_memory()
        self.h_outd = torch.empty((self.H, self.W), dtype=torch.float32).pin_memory()
        self.h2d = sum(t.numel() * 4 for t in self.h_c + self.h_d)
        self.d2h = self.H * self.W * 8

    def e2e_step(self):
        for s, hc, hd in zip(self.srcs, self.h_c, self.h_d):
            s.color.view(torch.int32).copy_(hc, non_blocking=True)
            s.depth.copy_(hd, non_blocking=True)
        self.sch.run()
        self.h_out.copy_(self.out_c.view(torch.int32), non_blocking=True)
        self.h_outd.copy_(self.out_d, non_blocking=True)

    def oracle_step(self, pool, cores):
        """The oracle's schedule (plan, RLE transfers, merges), a level's stages
        spread over the host cores."""
        import oracle
        from oracle import schedules as OS
        if not hasattr(self, "_host"):
            self._host = [oracle.Image(s.pvp, s.roi, s.color.view(torch.int32).cpu().numpy().view(np.uint32),
                                       s.depth.cpu().numpy()) for s in self.srcs]
        algo = {"stream": OS.CHAIN, "direct_send": OS.DIRECT_SEND, "binary_swap": OS.BINARY_SWAP,
                "two_three_swap": OS.TWO_THREE_SWAP}[self.algo]
        t0 = time.perf_counter()
        pl = OS.plan(algo, (0, 0, self.W, self.H), [OS.intersect(tuple(i.roi), tuple(i.pvp)) for i in self._host])
        OS.run_depth(pl, self._host, compress=self.variant != "raw", map=pool.map)
        return time.perf_counter() - t0


class BatchedTiles:
    """cfg4: 1000 uneven tiles (w, h log-uniform in [16, 1024], 2..64 layers, half
    depth RGBA8+Z32 at 30% box coverage, half alpha FP32 with a <= 0.3), all in
    one persistent graph-captured launch (autotuned tile shapes)."""

    def __init__(self, device, n_tiles=1000):
        import ctypes as C

        import paper_1902_08755_gb300 as ec
        from paper_1902_08755_gb300 import _abi as A
        from paper_1902_08755_gb300 import api
        import synthetic as S
        self.ec = ec
        self.desc = (f"{n_tiles} tiles, w,h log-uniform [16,1024], layers U{{2..64}}, half depth "
                     f"RGBA8+Z32 (30% coverage), half alpha FP32 (a<=0.3); one persistent "
                     f"graph-captured launch vs one launch per tile")
        self.tiles = S.uneven_tiles(4, n_tiles, device=device)
        self.units = sum(t.w * t.h * t.L for t in self.tiles)
        self.bytes = sum(t.w * t.h * (t.L * (8 if t.mode == "depth" else 16) + (8 if t.mode == "depth" else 16))
                         for t in self.tiles)
        self.ctx = ec.default_context(torch.device(device).index or 0)
        self.jobs = []
        for t in self.tiles:
            if t.mode == "depth":
                imgs = [ec.Image(color=t.color[k], depth=t.depth[k]) for k in range(t.L)]
                out = torch.empty((t.h, t.w), dtype=torch.int32, device=device).view(torch.uint32)
                dep = torch.empty((t.h, t.w), dtype=torch.float32, device=device)
                self.jobs.append(ec.Job("depth", imgs, out, out_depth=dep))
            else:
                imgs = [ec.Image(color=t.color[k]) for k in range(t.L)]
                out = torch.empty((t.h, t.w, 4), dtype=torch.float32, device=device)
                self.jobs.append(ec.Job("alpha", imgs, out))
        t0 = time.perf_counter()
        self.batch = ec.Batch(self.jobs, ctx=self.ctx)
        self.plan_s = time.perf_counter() - t0
        # per-tile baseline: the plain entry points, arguments marshalled once
        lib = A.load()
        self._calls = []
        for jb in self.jobs:
            dev = self.ctx.device
            arr = (A.ec_image * len(jb.images))(*[api._image_struct(im, dev, jb.mode == "depth") for im in jb.images])
            tgt = api._target(jb.out_color, jb.out_depth, None, dev)
            if jb.mode == "depth":
                self._calls.append((lib.ec_composite_depth, (self.ctx.h, arr, len(jb.images), C.byref(tgt), None, None)))
            else:
                self._calls.append((lib.ec_composite_alpha, (self.ctx.h, arr, None, len(jb.images), C.byref(tgt), None, None)))
            self._calls[-1] += (arr, tgt)
        self.kernels = ["batch"]

    def step(self, ev=None):
        if ev:
            ev[0].record()
        self.batch.run()
        if ev:
            ev[1].record()

    def per_tile(self):
        s = torch.cuda.current_stream().cuda_stream
        for fn, args, *_ in self._calls:
            fn(*args, s)

    def launches_per_step(self):
        return 1

    def algorithmic_bytes(self):
        return {"batch": self.bytes}

    def setup_e2e(self):
        self.h2d = 0
        self.d2h = 0

    def e2e_step(self):
        self.step()


class L2Flush:
    """Evicts L2 between timed steps: writes 2x L2, then reads another 2x L2
    (clean lines), so no dirty flush lines are written back inside a step."""

    def __init__(self, device, l2_bytes):
        n = max(2 * l2_bytes, 256 << 20)
        self.dirty = torch.empty(n, dtype=torch.uint8, device=device)
        self.clean = torch.zeros(n // 4, dtype=torch.int32, device=device)

    def __call__(self, k):
        self.dirty.fill_(k & 0xFF)
        self.sink = self.clean.sum()


def _timed(fn, flush, reps):
    """Median CUDA-event time (ms) of fn over reps calls, L2 flushed before each."""
    ts = []
    for k in range(reps):
        flush(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        ts.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ts)


ALPHA_RATIO_CASES = [
    # key, cfg, layers, W, H, alpha max, storage
    ("fp32", 3, 32, 2048, 2048, 0.3, torch.float32),
    ("fp16", 3, 32, 2048, 2048, 0.3, torch.float16),
    ("cfg5a_fp16", 5, 128, 3840, 2160, 0.1, torch.float16),
]


def alpha_fwd_bwd_ratio(device, flush, peak, reps=20):
    """Ordered compositing, plain forward, separate backward (the autograd
    path: forward, then backward) and the fused forward+backward, with the
    ratios to the plain forward: 32 layers at 2048^2 (FP32 and FP16 storage)
    and 128 FP16 layers at 3840x2160."""
    import paper_1902_08755_gb300 as ec
    import synthetic as S
    res = {}
    for tag, cfg, L, W, H, amax, dtype in ALPHA_RATIO_CASES:
        w = S.grad_weights(cfg, W, H, device=device)
        lay = S.alpha_layers(cfg, L, W, H, amax, dtype=dtype, device=device)
        imgs = [ec.Image(color=lay[k]) for k in range(L)]
        out = torch.empty((H, W, 4), dtype=dtype, device=device)
        grads = [torch.empty_like(lay[k]) for k in range(L)]
        s = 16 if dtype == torch.float32 else 8
        px = W * H
        fwd = lambda: ec.composite_alpha(imgs, out)
        bwd = lambda: ec.composite_alpha_backward(imgs, (0, 0, W, H), w, grads)
        fused = lambda: ec.composite_alpha_fwd_bwd(imgs, out, w, grads)
        for f in (fwd, bwd, fused):
            f()
        torch.cuda.synchronize()
        t_f, t_b, t_x = _timed(fwd, flush, reps), _timed(bwd, flush, reps), _timed(fused, flush, reps)
        b_f = L * px * s + px * s
        b_b = L * px * s + px * 16 + L * px * s
        b_x = L * px * s + px * 16 + px * s + L * px * s
        gb = lambda b, t: b / (t * 1e-3) / 1e9
        res[tag] = {"layers": L, "size": f"{W}x{H}", "storage": "FP32" if dtype == torch.float32 else "FP16",
                    "fwd_ms": t_f, "bwd_ms": t_b, "fused_fwd_bwd_ms": t_x,
                    "fwd_plus_bwd_over_fwd": (t_f + t_b) / t_f, "fused_over_fwd": t_x / t_f,
                    "fwd_frac_of_peak": gb(b_f, t_f) / peak, "bwd_frac_of_peak": gb(b_b, t_b) / peak,
                    "fused_frac_of_peak": gb(b_x, t_x) / peak,
                    "fwd_gpixel_layers_s": L * px / (t_f * 1e-3) / 1e9}
        del lay, imgs, out, grads, w
        torch.cuda.empty_cache()
    return res


def make_workload(name, device, sources=0):
    if name == "cfg1":
        return DepthPipeline(1, 4, 640, 480, 0.4, False, False, device, keep=sources)
    if name == "cfg2":
        return DepthPipeline(2, 16, 1920, 1080, 0.3, True, True, device, keep=sources)
    if name == "cfg5d":
        return DepthPipeline(5, 64, 7680, 4320, 0.25, True, True, device, keep=sources)
    if name == "cfg4":
        return BatchedTiles(device)
    if name == "roi2":
        return RoiDetect(2, 16, 1920, 1080, 0.3, device)
    if name == "asm4k":
        return Assembly(3840, 2160, device)
    if name == "sched2":
        return Schedules(device)
    if name in ("rle0", "yuv2", "rle0big"):
        return CodecPipeline(name, device)
    if name == "cfg3":
        return AlphaForward(3, 32, 2048, 2048, 0.3, torch.float32, device)
    if name == "cfg3h":
        return AlphaForward(3, 32, 2048, 2048, 0.3, torch.float16, device)
    if name == "cfg3fused":
        return AlphaFused(3, 32, 2048, 2048, 0.3, torch.float32, device)
    if name == "cfg3hfused":
        return AlphaFused(3, 32, 2048, 2048, 0.3, torch.float16, device)
    if name == "cfg5afused":
        return AlphaFused(5, 128, 3840, 2160, 0.1, torch.float16, device)
    if name == "cfg5a":
        return AlphaForward(5, 128, 3840, 2160, 0.1, torch.float16, device)
    if name == "cfg5afusedq":               # a quarter of the frame's rows: sized for ncu captures
        return AlphaFused(5, 128, 3840, 540, 0.1, torch.float16, device)
    raise SystemExit(f"unknown workload {name}")


# -------------------------------------------------------------------- arms

# Sources per oracle step of the depth workloads' CPU legs: (all cores, one core).
CPU_SAMPLE = {"cfg1": (4, 4), "cfg2": (16, 2), "cfg5d": (8, 1)}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                return v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip().lower() == "model name":
                    return v.strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_reps(wl, pool, cores, k, budget_s, max_reps):
    times = []
    t_start = time.perf_counter()
    while len(times) < max_reps and (not times or (time.perf_counter() - t_start) < budget_s):
        times.append(wl.oracle_step(pool, cores, k) if k else wl.oracle_step(pool, cores))
    return times


def _sample_value(wl, t):
    units = getattr(wl, "sample_units", None)
    if units is None:                      # row-band samples are scaled inside oracle_step
        units = wl.units
    return units / t / 1e9


def oracle_single_core(args):
    """Child process of cpu_baseline: the oracle pinned to one core, on the
    first sources of the workload, generated here on the host."""
    cpus = sorted(os.sched_getaffinity(0))
    os.sched_setaffinity(0, {cpus[-1]})
    torch.set_num_threads(1)
    wl = make_workload(args.workload, "cpu", sources=args.sources)
    with ThreadPoolExecutor(max_workers=1) as pool:
        times = _oracle_reps(wl, pool, 1, 0, 15.0, 10)
    t = statistics.median(times)
    print(json.dumps({"value": _sample_value(wl, t), "ms_per_step": t * 1e3, "reps": len(times),
                      "cpu": cpus[-1], "sample": getattr(wl, "sample_desc", "full steps")}), flush=True)


def cpu_baseline(args, wl, budget_s=12.0, max_reps=20):
    """The oracle as it stands on the host cores: all cores over a bounded
    sample of the workload, and (depth workloads) one pinned core."""
    cores = os.cpu_count() or 1
    many, one = CPU_SAMPLE.get(args.workload, (0, 0))
    with ThreadPoolExecutor(max_workers=cores) as pool:
        times = _oracle_reps(wl, pool, cores, many, budget_s, max_reps)
    t = statistics.median(times)
    frac = getattr(wl, "sample_fraction", 1.0)
    desc = getattr(wl, "sample_desc", "full steps")
    sample = (f"{len(times)} steps, each {desc}" if frac == 1.0 else
              f"{len(times)} x {desc}, scaled to a full step")
    res = {"value": _sample_value(wl, t), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
           "ms_per_step": t * 1e3, "cpu_model": cpu_model()}
    if one:
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-single-core", "--workload", args.workload,
               "--sources", str(one)]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
            d = json.loads(r.stdout.strip().splitlines()[-1])
            res["single_core"] = {"value": d["value"], "unit": UNIT, "cores": 1, "pinned_cpu": d["cpu"],
                                  "ms_per_step": d["ms_per_step"],
                                  "sample": f"{d['reps']} steps, each {d['sample']}, one thread pinned to one core"}
        except (OSError, subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
            res["single_core"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return res


REF_BUDGET_S = 100.0     # wall-clock cap of the reference arm's warm-up and timed steps


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    many = CPU_SAMPLE.get(args.workload, (0, 0))[0]
    wl = make_workload(args.workload, "cpu", sources=args.sources or many)
    cores = os.cpu_count() or 1
    # W warm-up and K timed steps, each a bounded sample of the workload; the run
    # stops early (and reports the steps it ran) once it has used REF_BUDGET_S
    t_start = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as pool:
        warm = 0
        while warm < args.warmup and (warm == 0 or time.perf_counter() - t_start < REF_BUDGET_S / 4):
            wl.oracle_step(pool, cores)
            warm += 1
        times = []
        while len(times) < max(1, args.steps) and (not times or time.perf_counter() - t_start < REF_BUDGET_S):
            times.append(wl.oracle_step(pool, cores))
    t = statistics.median(times)
    val = _sample_value(wl, t)
    frac = getattr(wl, "sample_fraction", 1.0)
    desc = getattr(wl, "sample_desc", "full steps")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": warm, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "rgba8+f32",
            "data": "synthetic", "config": {"workload": f"{args.workload}: {wl.desc}"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc if frac == 1.0 else f"{desc}, scaled", "cpu_model": cpu_model()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def step_events(wl, steps):
    nk = len(wl.kernels)
    return [[torch.cuda.Event(enable_timing=True) for _ in range(nk + 1)] for _ in range(steps)]


def kernel_times(wl, evs):
    """Per-kernel event times [kernel][step] (launches of one kernel kind in a
    step summed), the kernel names and launches of each per step."""
    nk, steps = len(wl.kernels), len(evs)
    per_kernel = [[evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(steps)] for i in range(nk)]
    names = list(wl.kernels)
    launches_of = {n: 1 for n in names}
    if hasattr(wl, "kind_of"):              # several launches of one kernel per step: sum them
        agg, cnt = {}, {}
        for i, kd in enumerate(wl.kind_of):
            a = agg.setdefault(kd, [0.0] * steps)
            cnt[kd] = cnt.get(kd, 0) + 1
            for k in range(steps):
                a[k] += per_kernel[i][k]
        names = list(agg)
        per_kernel = [agg[n] for n in names]
        launches_of = cnt
    return per_kernel, names, launches_of


def kernel_table(wl, per_kernel, names, launches_of, peak):
    algo = wl.algorithmic_bytes()
    steps = len(per_kernel[0])
    step_ms = statistics.median(sum(per_kernel[i][k] for i in range(len(names))) for k in range(steps))
    kern = {}
    for i, name in enumerate(names):
        kms = statistics.median(per_kernel[i])
        gbs = algo[name] / (kms * 1e-3) / 1e9
        kern[name] = {"ms": kms, "share": kms / step_ms, "algorithmic_bytes": algo[name],
                      "achieved_gbs": gbs, "frac_of_peak": gbs / peak, "launches_per_step": launches_of[name]}
    return kern


def depth_secondary(name, device, flush, peak, steps=50, warmup=5):
    """A depth pipeline other than the headline one, timed the same way."""
    wl = make_workload(name, device)
    for _ in range(warmup):
        wl.step()
    torch.cuda.synchronize()
    evs = step_events(wl, steps)
    for k in range(steps):
        flush(k)
        wl.step(evs[k])
    torch.cuda.synchronize()
    wl.ctx.check_status(what=name)
    per_kernel, names, launches_of = kernel_times(wl, evs)
    step_ms = statistics.median(sum(per_kernel[i][k] for i in range(len(names))) for k in range(steps))
    res = {"workload": f"{name}: {wl.desc}", "value": wl.units / (step_ms * 1e-3) / 1e9, "unit": UNIT,
           "ms_per_step": step_ms, "steps": steps, "pixel_layers_per_step": wl.units,
           "rle_compressed_bytes_per_step": wl.compressed_bytes(),
           "kernels": kernel_table(wl, per_kernel, names, launches_of, peak)}
    del wl
    torch.cuda.empty_cache()
    return res


def batched_extra(device, flush, peak, reps=20):
    """The 1000 uneven tiles: one persistent graph-captured launch against one
    plain launch per tile (median times)."""
    wl = BatchedTiles(device)
    wl.step()
    wl.per_tile()
    torch.cuda.synchronize()
    b = _timed(wl.step, flush, reps)
    pt = _timed(wl.per_tile, flush, max(5, reps // 2))
    wl.ctx.check_status(what="batched tiles")
    res = {"workload": f"cfg4: {wl.desc}", "batched_ms": b, "per_tile_ms": pt, "speedup": pt / b,
           "algorithmic_bytes": wl.bytes, "batched_frac_of_peak": wl.bytes / (b * 1e-3) / 1e9 / peak,
           "gpixel_layers_s": wl.units / (b * 1e-3) / 1e9, "plan_s": wl.plan_s, "config": wl.batch.config}
    wl.batch.close()
    del wl
    torch.cuda.empty_cache()
    return res


def run_ec(args):
    rank, world, local = dist_env()
    dist_init(world, local)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    import paper_1902_08755_gb300 as ec
    ec.load()
    wl = make_workload(args.workload, device, sources=args.sources)
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = L2Flush(device, l2)
    peak, peak_src = hbm_peak()

    for _ in range(max(3, args.warmup)):
        wl.step()
    wl.ctx.check_status(what="warm-up")
    torch.cuda.synchronize()

    evs = step_events(wl, args.steps)
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush(k)                               # evict the previous step's data from L2
        wl.step(evs[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    barrier(world)
    st = wl.ctx.status_sync()
    if st != 0:
        raise SystemExit(f"device status {st} after the timed region")
    per_kernel, names, launches_of = kernel_times(wl, evs)
    step_ms = [sum(per_kernel[i][k] for i in range(len(names))) for k in range(args.steps)]
    ms = statistics.median(step_ms)
    per_launch_sum_ms = ms
    if hasattr(wl, "graph_step"):            # the step as users run it: one graph launch
        g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush(k)
            g_ev[k][0].record()
            wl.graph_step()
            g_ev[k][1].record()
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in g_ev)
    ms = max_over_ranks(ms, world)
    value = whole_job_value(wl.units, ms, world)

    # end to end through the public API, host buffers in pinned memory
    wl.setup_e2e()
    for _ in range(3):
        wl.e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(50, min(args.steps, 200))
    barrier(world)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(e2e_steps):
        wl.e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world)
    wl.ctx.check_status(what="end to end")

    if rank != 0:
        return
    kern = kernel_table(wl, per_kernel, names, launches_of, peak)
    dom = max(kern, key=lambda k: kern[k]["ms"])
    traffic = measured_traffic(dom, args.workload if not args.sources else f"{args.workload}_s{args.sources}")
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_gbs"], "peak": peak,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
            "unit": "GB/s", "frac": kern[dom]["achieved_gbs"] / peak, "traffic": traffic}
    cfg = {"workload": f"{args.workload}: {wl.desc}",
           "l2": "flushed between timed steps (2x L2 written, then 2x L2 read; outside the events)",
           "timing": f"median over {args.steps} steps of the per-kernel CUDA events",
           "pixel_layers_per_step": wl.units, "parallelism": f"replicas x{world}"}
    if hasattr(wl, "compressed_bytes"):
        cfg["rle_compressed_bytes_per_step"] = wl.compressed_bytes()
        cfg["rle_raw_bytes_per_step"] = wl.raw_bytes() if hasattr(wl, "raw_bytes") else 8 * wl.stored_px
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "rgba8+f32" if isinstance(wl, (DepthPipeline, BatchedTiles, RoiDetect, Schedules, CodecPipeline)) else "u8" if isinstance(wl, Assembly) else "f32",
            "data": "synthetic (seeded boxes / layers shaped like the thesis's workloads)",
            "config": cfg, "roofline": roof, "kernels": kern,
            "e2e": {"value": whole_job_value(wl.units, e2e_ms, world), "unit": UNIT,
                    "ms_per_step": e2e_ms, "steps": e2e_steps, "h2d_bytes_per_step": wl.h2d,
                    "d2h_bytes_per_step": wl.d2h},
            "gpu_launches": wl.launches_per_step() * args.steps,
            "clocks": clk, "wall_s_timed_loop": t_wall}
    if hasattr(wl, "graph_step"):
        cfg["per_launch_sum_ms"] = per_launch_sum_ms
        if not args.no_extras:
            line["schedules"] = wl.others(flush)
    if isinstance(wl, BatchedTiles):
        pt = _timed(wl.per_tile, flush, 10)
        line["batched_vs_per_tile"] = {"batched_ms": ms, "per_tile_ms": pt, "speedup": pt / ms,
                                       "plan_s": wl.plan_s, "config": wl.batch.config}
    if world == 1 and not args.no_cpu_baseline and hasattr(wl, "oracle_step"):
        line["cpu_baseline"] = cpu_baseline(args, wl)
    if args.workload == "cfg5d" and not args.sources and not args.no_extras:
        # free the headline's buffers, then the other targets beside it
        del wl
        torch.cuda.empty_cache()
        line["secondary"] = {"cfg2": depth_secondary("cfg2", device, flush, peak)}
        line["batched_vs_per_tile"] = batched_extra(device, flush, peak)
        line["alpha_fwd_bwd"] = alpha_fwd_bwd_ratio(device, flush, peak)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_single_core:
        oracle_single_core(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ec(args)


if __name__ == "__main__":
    main()
