"""Benchmark of the tensorial template matching hot path on GB300.

One step = the whole per-tomogram path on one tomogram: tensorial
correlation with local normalisation (ttm_correlate: prefilter, image
spectrum, FP64 local sums, fused z pass, y pass, x pass with the w
epilogue) and the score + orientation maps (ttm_peak_map). The tensor field
(built once per template) is outside the timed region, as in the paper.

Workload: 512 x 512 x 200 float32 tomogram of Gaussian-low-passed noise
(sigma = 1) with 300 copies of a 40^3 six-Gaussian template planted at
uniform random rotations (SNR 0.1), tensor order 4 (15 components), mask
radius 16. Inputs (210 MB tomogram, 3.1 GB C maps) are larger than L2, so no
explicit flush between steps.

Prints one JSON line. `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2408_02398_gb300 import synth  # noqa: E402  (seeded input generators only)

WORKLOAD = "ttm_n4_512x512x200_t40_r16_300copies_snr0.1"
METRIC = "TTM voxels/s (score+orientation map)"
UNIT = "voxels/s"


def kernel_sources_digest(entry: str = "") -> str:
    """SHA-256 over CUDA sources of the library (file names and bytes,
    sorted), to tell whether a recorded ncu figure still describes them: all
    of csrc/, or with `entry` (a csrc/ file name) that file and the headers
    it includes, directly or not."""
    import glob
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2408_02398_gb300", "csrc")
    if entry:
        files, todo = set(), [os.path.join(csrc, entry)]
        while todo:
            f = os.path.normpath(todo.pop())
            if f in files or not os.path.exists(f):
                continue
            files.add(f)
            for inc in re.findall(r'^\s*#include\s+"([^"]+)"', open(f).read(), re.M):
                todo.append(os.path.join(os.path.dirname(f), inc))
        files = sorted(files)
    else:
        files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                       glob.glob(os.path.join(csrc, "*.h")))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def recorded_value(name: str, key: str):
    """A figure `key:` recorded in an ncu summary under profiles/, with the
    same source-digest check as recorded_traffic; None when absent or stale."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        line = line.strip().strip("`")
        for k in (key + ":", "sources_sha256:", "sources:"):
            if line.startswith(k):
                vals[k] = line[len(k):].strip()
    if vals.get("sources_sha256:") != kernel_sources_digest(vals.get("sources:", "")) or key + ":" not in vals:
        return None
    return float(vals[key + ":"])


def recorded_traffic(name: str):
    """DRAM bytes per voxel recorded in an ncu summary under profiles/ that
    states `dram_bytes_per_voxel:`, the `sources_sha256:` of the kernels it
    measured and, optionally, `sources:` (the csrc/ file those kernels come
    from, for a digest of that file and its headers only); None when the
    sources have changed since."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        line = line.strip().strip("`")
        for key in ("dram_bytes_per_voxel:", "sources_sha256:", "sources:"):
            if line.startswith(key):
                vals[key] = line[len(key):].strip()
    if vals.get("sources_sha256:") != kernel_sources_digest(vals.get("sources:", "")) or \
            "dram_bytes_per_voxel:" not in vals:
        return None
    return float(vals["dram_bytes_per_voxel:"])


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region.

    start() returns once the sampler has written its first line, so that the
    samples counted (those written between start() and stop()) fall inside
    the region that the caller times between the two calls. A region shorter
    than the interval may see none; then the last sample written before
    stop() stands in, and "in_region" says so."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.skip = 0

    def _rows(self):
        rows = []
        with open(self.path) as f:
            for line in f:
                if not line.endswith("\n"):
                    break
                r = [x.strip() for x in line.split(",")]
                if len(r) >= 9:
                    rows.append(r)
        return rows

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.perf_counter()
            while not self._rows() and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = len(self._rows())
        except Exception:
            self.proc = None
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        all_rows = self._rows()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        os.unlink(self.path)
        rows = all_rows[self.skip:]
        in_region = bool(rows)
        if not rows:
            rows = all_rows[-1:]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "in_region": in_region}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("TTM_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- CPU oracle --

def oracle_sample_rate(wl, n_voxels: int, seed: int = 1):
    """Time the FP64 oracle on n_voxels of the valid interior: local
    normaliser, direct-sum tensorial correlation and dense-sampling +
    Newton maximiser. Setup (filter of the volume, template normalisation
    and a field built with 192 rotations -- the per-voxel cost of the timed
    steps does not depend on the quadrature size) is excluded."""
    import oracle as O
    n = wl.order_n
    pr = O.Prepared(wl.tomo, wl.template, wl.mask_radius)
    T = O.tensor_field(pr.tp, O.rotation_set(8), n, 3)
    vox = O.valid_voxels(pr.g.shape, pr.tshape)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(vox.size, size=min(n_voxels, vox.size), replace=False))
    v = vox[sel]
    t0 = time.perf_counter()
    w, _, _ = O.local_w(pr.g, pr.m, v, False, pr.floor)
    C = O.correlate(pr.g, T, v, False, w)
    O.maximise(C, n, 3, 20000)
    dt = time.perf_counter() - t0
    return v.size / dt, v.size, dt, O.num_threads()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2408_02398_gb300 import synth
    wl = synth.workload_order4()
    # calibrate the sample so the whole run stays within a few minutes
    rate0, _, _, cores = oracle_sample_rate(wl, 200)
    per_step = max(200, int(rate0 * 8.0))
    times = []
    nv = 0
    for i in range(args.warmup + args.steps):
        r, nv, dt, cores = oracle_sample_rate(wl, per_step, seed=i + 2)
        if i >= args.warmup:
            times.append(dt)
    value = nv * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_voxels_per_step": nv},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d random valid-interior voxels per step: local normaliser, direct-sum "
                                       "correlation (15 components), 20000-sample + Newton maximiser" % nv},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU path --

def _events(stream):
    import torch
    e = torch.cuda.Event(enable_timing=True)
    e.record(stream)
    return e


def _step_ms(fn, steps, warmup, stream):
    """Milliseconds per call of fn: CUDA events on `stream`, after warm-up."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = _events(stream)
    for _ in range(steps):
        fn()
    e1 = _events(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def e2e_pipelined(ttm, m, h_tomo, steps, warmup, dev):
    """End to end through the public calls with host buffers, copies inside
    the timed region: per step the pinned tomogram goes to the device
    (copy stream), ttm_correlate + ttm_peak_map run (compute stream) and the
    score and orientation maps come back to pinned host memory (copy-out
    stream). Two buffer sets let step i+1's upload and step i-1's download
    overlap step i's kernels; events order every reuse of a buffer."""
    import torch
    Z, Y, X = h_tomo.shape
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    d_in = [torch.empty((Z, Y, X), device=dev) for _ in range(2)]
    d_s = [torch.empty((Z, Y, X), device=dev) for _ in range(2)]
    d_o = [torch.empty((3, Z, Y, X), device=dev) for _ in range(2)]
    h_s = [torch.empty((Z, Y, X)).pin_memory() for _ in range(2)]
    h_o = [torch.empty((3, Z, Y, X)).pin_memory() for _ in range(2)]
    ev = lambda: torch.cuda.Event()  # noqa: E731
    in_ready, in_free, maps_ready, maps_free = ([ev(), ev()] for _ in range(4))
    for e in in_free + maps_free:
        e.record(s_cmp)

    def step(i):
        b = i % 2
        s_in.wait_event(in_free[b])
        with torch.cuda.stream(s_in):
            d_in[b].copy_(h_tomo, non_blocking=True)
        in_ready[b].record(s_in)
        s_cmp.wait_event(in_ready[b])
        s_cmp.wait_event(maps_free[b])
        ttm.ttm_correlate(m.plan, d_in[b], m.C, stream=s_cmp)
        in_free[b].record(s_cmp)
        ttm.ttm_peak_map(m.plan, m.C, d_s[b], d_o[b], stream=s_cmp)
        maps_ready[b].record(s_cmp)
        s_out.wait_event(maps_ready[b])
        with torch.cuda.stream(s_out):
            h_s[b].copy_(d_s[b], non_blocking=True)
            h_o[b].copy_(d_o[b], non_blocking=True)
        maps_free[b].record(s_out)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    for i in range(steps):
        step(i)
    s_in.wait_stream(s_out)
    t1.record(s_in)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def tm_comparator(ttm, ctx, wl, p, dev, n_rot):
    """Classical per-rotation TM (tm_correlate) on the same volume over
    n_rot rotations taken evenly from the 45 123-rotation super-Fibonacci
    list (the count the paper cites for a 7-degree step, Sec. 1). One call
    is timed on the host around its synchronising return; the library's
    per-call set-up (workspace, image preparation) is amortised over the
    rotations."""
    import torch
    full = ttm.ttm_rotation_set(45123, cube=False)
    sel = full[np.linspace(0, full.shape[0] - 1, n_rot).astype(np.int64)]
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    t = torch.as_tensor(wl.template, device=dev)
    best = torch.empty(wl.tomo.shape, device=dev)
    idx = torch.empty(wl.tomo.shape, dtype=torch.int32, device=dev)
    ttm.tm_correlate(ctx, d_tomo, t, p, sel[:4], best, idx)     # warm-up (kernels, allocator)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ttm.tm_correlate(ctx, d_tomo, t, p, sel, best, idx)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    return {"rotations_timed": int(n_rot), "ms_per_rotation": 1e3 * s / n_rot,
            "implied_45123_rotations_s": s / n_rot * 45123.0}


def cufft_comparator(ttm, m, wl, dev, steps):
    """The same correlation through cuFFT (torch.fft), timed only:
    G = rfftn(g), then for each of the K components irfftn(G conj(T_hat))
    times w, written into a K x V map; and the local sums of Eq. 2 as FP64
    cuFFT transforms of g and g^2 against the mask spectrum. g (the 3-tap
    filter), w and the template spectra are prepared outside the timed
    region, as the library's plan holds its spectra."""
    import torch
    Z, Y, X = wl.tomo.shape
    K = m.C.shape[0]
    f = torch.as_tensor(wl.tomo, device=dev)[None, None]
    a = 0.2
    taps = torch.tensor([a, 1 - 2 * a, a], device=dev)
    g = f
    for ax in range(3):
        shape = [1, 1, 1, 1, 1]
        shape[2 + ax] = 3
        pad = [0, 0, 0]
        pad[ax] = 1
        g = torch.nn.functional.conv3d(g, taps.reshape(shape), padding=tuple(pad))
    g = g[0, 0].contiguous()
    w = torch.empty((Z, Y, X), device=dev)
    ttm.ttm_plan_copy_w(m.plan, w)
    tz, ty, tx = m.field.shape[1:]
    Tg = torch.zeros((K, Z, Y, X), dtype=torch.float32, device=dev)
    cz, cy, cx = tz // 2, ty // 2, tx // 2
    # place each component at the origin of the working grid (wrapped)
    zi = torch.tensor([(d - cz) % Z for d in range(tz)], device=dev)
    yi = torch.tensor([(d - cy) % Y for d in range(ty)], device=dev)
    xi = torch.tensor([(d - cx) % X for d in range(tx)], device=dev)
    Tg[:, zi[:, None, None], yi[None, :, None], xi[None, None, :]] = m.field.float()
    That = torch.fft.rfftn(Tg, dim=(1, 2, 3))
    del Tg
    out = torch.empty((K, Z, Y, X), device=dev)
    mk = torch.zeros((Z, Y, X), dtype=torch.float64, device=dev)
    msk = torch.as_tensor(synth.sphere_mask_values(tz, wl.mask_radius), dtype=torch.float64, device=dev)
    mk[zi[:, None, None], yi[None, :, None], xi[None, None, :]] = msk
    Mhat = torch.fft.rfftn(mk)
    M = float(msk.sum())
    stream = torch.cuda.current_stream()

    def corr():
        G = torch.fft.rfftn(g)
        for k in range(K):
            torch.mul(torch.fft.irfftn(G * That[k].conj(), s=(Z, Y, X)), w, out=out[k])

    def lsum():
        gd = g.double()
        S1 = torch.fft.irfftn(torch.fft.rfftn(gd) * Mhat.conj(), s=(Z, Y, X))
        S2 = torch.fft.irfftn(torch.fft.rfftn(gd * gd) * Mhat.conj(), s=(Z, Y, X))
        var = S2 - S1 * S1 / M
        return var

    ms_corr = _step_ms(corr, steps, 1, stream)
    ms_ls = _step_ms(lsum, steps, 1, stream)
    torch.cuda.synchronize()
    err = float((out - m.C).abs().max().item())
    del That, out, Mhat, mk
    torch.cuda.empty_cache()
    return {"correlate_K_components_ms": ms_corr, "localsums_fp64_ms": ms_ls,
            "what": "torch.fft (cuFFT): rfftn(g), K x (product, irfftn, times w); local sums FP64 rfftn/irfftn",
            "max_abs_diff_vs_ttm_correlate": err}


def forms_order4(ttm, ctx, wl, dev, steps, warmup, crop_voxels):
    """FP32, FP16 and BF16 template spectra on the benchmark volume, each
    timed (correlate + maximiser, double-float local sums) and checked
    against the FP64 oracle at sampled valid voxels of the centred 128^3
    crop. Both sides use a 24 x 64-rotation field (the per-tomogram kernels
    do not depend on the quadrature)."""
    import torch
    import oracle as O
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=64)
    t = torch.as_tensor(wl.template, device=dev)
    field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device=dev)
    ttm.ttm_build_tensor_field(ctx, t, p, field)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    C = torch.empty((K, Z, Y, X), device=dev)
    score = torch.empty((Z, Y, X), device=dev)
    orient = torch.empty((3, Z, Y, X), device=dev)
    vox = _crop_voxels((Z, Y, X), wl.template.shape, 128, crop_voxels, 11)
    tv = torch.as_tensor(vox, device=dev)
    pr = O.Prepared(wl.tomo, wl.template, r)
    ofield = O.tensor_field(pr.tp, O.rotation_set(64), n, 3)
    wref, _, _ = O.local_w(pr.g, pr.m, vox, False, pr.floor)
    Cref = O.correlate(pr.g, ofield, vox, False, wref)
    sref, _, _ = O.maximise(Cref, n, 3, 20000)
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp32", ttm.TTM_PREC_FP32), ("fp16", ttm.TTM_PREC_FP16_SPECTRA),
                       ("bf16", ttm.TTM_PREC_BF16_SPECTRA)):
        plan = ttm.Plan(ctx, field, p, (Z, Y, X), precision=prec)
        ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
        mc = _step_ms(lambda: ttm.ttm_correlate(plan, d_tomo, C), steps, warmup, stream)
        mp = _step_ms(lambda: ttm.ttm_peak_map(plan, C, score, orient), steps, warmup, stream)
        # per-stage times of separate, instrumented calls (not the timed ones)
        ttm.ttm_plan_stage_times(plan)
        ttm.ttm_plan_enable_timing(plan, True)
        for _ in range(steps):
            ttm.ttm_correlate(plan, d_tomo, C)
            ttm.ttm_peak_map(plan, C, score, orient)
        st = {k: v / steps for k, v in ttm.ttm_plan_stage_times(plan).items()}
        ttm.ttm_plan_enable_timing(plan, False)
        got = C.reshape(K, -1)[:, tv].cpu().numpy().astype(np.float64)
        sg = score.flatten()[tv].cpu().numpy().astype(np.float64)
        out[name] = {"correlate_ms": mc, "peak_map_ms": mp, "voxels_per_s": V / ((mc + mp) / 1e3),
                     "stages_ms": st,
                     "C_max_abs_err": float(np.abs(got - Cref).max()),
                     "C_rel_l2_err": float(np.linalg.norm(got - Cref) / np.linalg.norm(Cref)),
                     "score_max_abs_err": float(np.abs(sg - sref).max())}
        del plan
    for name in ("fp16", "bf16"):
        out[name]["vs_fp32_whole_step"] = out[name]["voxels_per_s"] / out["fp32"]["voxels_per_s"]
        out[name]["vs_fp32_correlate"] = out["fp32"]["correlate_ms"] / out[name]["correlate_ms"]
    out["error_sample"] = "%d valid voxels of the centred 128^3 crop vs the FP64 oracle" % vox.size
    del C, score, orient, field
    torch.cuda.empty_cache()
    return out


def plain_order6(ttm, ctx, dev, steps, warmup, crop_voxels):
    """The plain FP32 form on the largest configuration: 1024 x 1024 x 256,
    48^3 template, r = 19, n = 6 (28 components), 2000 copies at SNR 0.05;
    timed per call, and checked against the FP64 oracle at sampled voxels of
    the centred 128^3 crop (24 x 64-rotation field on both sides)."""
    import torch
    import oracle as O
    t0 = time.perf_counter()
    wl = synth.workload_order6()
    gen_s = time.perf_counter() - t0
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=64)
    t = torch.as_tensor(wl.template, device=dev)
    field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device=dev)
    ttm.ttm_build_tensor_field(ctx, t, p, field)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    C = torch.empty((K, Z, Y, X), device=dev)
    score = torch.empty((Z, Y, X), device=dev)
    orient = torch.empty((3, Z, Y, X), device=dev)
    plan = ttm.Plan(ctx, field, p, (Z, Y, X))
    ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
    stream = torch.cuda.current_stream()
    mc = _step_ms(lambda: ttm.ttm_correlate(plan, d_tomo, C), steps, warmup, stream)
    mp = _step_ms(lambda: ttm.ttm_peak_map(plan, C, score, orient), steps, warmup, stream)
    vox = _crop_voxels((Z, Y, X), wl.template.shape, 128, crop_voxels, 13)
    tv = torch.as_tensor(vox, device=dev)
    got = C.reshape(K, -1)[:, tv].cpu().numpy().astype(np.float64)
    sg = score.flatten()[tv].cpu().numpy().astype(np.float64)
    pr = O.Prepared(wl.tomo, wl.template, r)
    ofield = O.tensor_field(pr.tp, O.rotation_set(64), n, 3)
    wref, _, _ = O.local_w(pr.g, pr.m, vox, False, pr.floor)
    Cref = O.correlate(pr.g, ofield, vox, False, wref)
    sref, _, _ = O.maximise(Cref, n, 3, 20000)
    del plan, C, score, orient, field, d_tomo
    torch.cuda.empty_cache()
    return {"workload": wl.name, "shape_zyx": [Z, Y, X], "order_n": n, "components": K,
            "correlate_ms": mc, "peak_map_ms": mp, "voxels_per_s": V / ((mc + mp) / 1e3),
            "local_sums": "double-float", "spectra": "fp32",
            "C_max_abs_err": float(np.abs(got - Cref).max()), "score_max_abs_err": float(np.abs(sg - sref).max()),
            "error_sample": "%d valid voxels of the centred 128^3 crop" % vox.size, "generation_s": gen_s}


def run_ours(args, ws, rank, local):
    import torch
    from paper_2408_02398_gb300 import build
    build.build()
    from paper_2408_02398_gb300 import ttm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    if args.zyx:
        # a smaller volume of the same workload (profiling captures): copies
        # scale with the volume
        shp = tuple(int(v) for v in args.zyx.split(","))
        wl = synth.workload_order4(shape=shp, copies=max(1, int(300 * np.prod(shp) / (200 * 512 * 512))))
    else:
        wl = synth.workload_order4()
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n = wl.order_n
    K = ttm.ttm_num_components(n)
    ctx = ttm.Context(local)
    p = ttm.params(order_n=n, mask_radius=wl.mask_radius, n_rot_base=2048)
    t0 = time.perf_counter()
    m = ttm.Matcher(ctx, wl.template, p, (Z, Y, X), device=dev)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    ls_main = ttm.TTM_LOCALSUM_DF64 if args.localsum == "df64" else ttm.TTM_LOCALSUM_FP64
    ttm.ttm_plan_set_localsum(m.plan, ls_main)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ttm.ttm_correlate(m.plan, d_tomo, m.C)
        ttm.ttm_peak_map(m.plan, m.C, m.score, m.orient, m.frob)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ttm.ttm_plan_stage_times(m.plan)  # discard
    ttm.ttm_plan_enable_timing(m.plan, True)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ttm.ttm_kernel_launches()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = _events(stream)
    for _ in range(args.steps):
        step()
    e1 = _events(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = ttm.ttm_kernel_launches() - launches0
    ms_total = e0.elapsed_time(e1)
    stages = ttm.ttm_plan_stage_times(m.plan)
    ttm.ttm_plan_enable_timing(m.plan, False)
    ck = clocks.stop()
    ms_total = max_over_ranks(ms_total, ws, dev)
    ms_step = ms_total / args.steps
    value = V * args.steps * ws / (ms_total / 1e3)

    # the other local-sum arithmetic, same plan, same steps
    other = ttm.TTM_LOCALSUM_FP64 if ls_main == ttm.TTM_LOCALSUM_DF64 else ttm.TTM_LOCALSUM_DF64
    ttm.ttm_plan_set_localsum(m.plan, other)
    ms_other = max_over_ranks(_step_ms(step, args.steps, 2, stream), ws, dev)
    ttm.ttm_plan_set_localsum(m.plan, ls_main)

    # end to end through the public calls with pinned host buffers
    h_tomo = torch.from_numpy(wl.tomo).pin_memory()
    ms_e2e = max_over_ranks(e2e_pipelined(ttm, m, h_tomo, args.steps, max(2, args.warmup // 2), dev), ws, dev)
    e2e_value = V * ws / (ms_e2e / 1e3)

    # Rooflines (stages: per-step milliseconds of CUDA events on the
    # launching stream). The maximiser's dense work is the probe product on
    # the tensor cores (FP16 mma.sync, same rate as BF16): 2 K P flops per
    # voxel (P = 128 probes; the kernel pads K to 16, which is not counted), against the
    # measured dense 16-bit peak; its time goes to the scalar Newton and
    # start-selection work around that product (instruction issue), so the
    # fraction is small by construction. The correlate path is HBM-bound:
    # 4 + 4K algorithmic bytes per voxel (read f, write K maps).
    st_ms = {k: v / args.steps for k, v in stages.items()}
    corr_ms = sum(v for k, v in st_ms.items() if k != "peak_map")   # ttm_correlate
    pk, how = peaks_file()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    tc_peak = float(pk.get("bf16_tflops", 1900.0))
    pm_flops = 2.0 * K * 128 * V
    tpm = recorded_traffic("traffic_peakmap_n4.md") if n == 4 else None
    roof_pm = {"bound": "tensor", "kernel": "k_peakmap<%d> (ttm_peak_map)" % n,
               "achieved": pm_flops / (st_ms["peak_map"] / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
               "peak_source": how + " dense BF16 (burst); FP16 mma has the same rate",
               "traffic": None if tpm is None else tpm * V,
               "traffic_source": "profiles/traffic_peakmap_n4.md (ncu dram bytes of one k_peakmap<4> launch on "
                                 "200x256x256, per voxel, scaled to this launch; null once its sources changed)",
               "flops_per_voxel": 2 * K * 128,
               "note": "issue-bound on the scalar Newton / start work around the probe product",
               "warp_inst_per_voxel": recorded_value("k_peakmap_n4_64x512x512.md", "warp_inst_per_voxel") if n == 4
               else None}
    roof_pm["frac"] = roof_pm["achieved"] / roof_pm["peak"]
    if roof_pm["warp_inst_per_voxel"] is not None:
        # what bounds it: warp instructions issued per second against the
        # SMs' issue peak (4 schedulers per SM, one warp instruction each per
        # cycle, at the SM clock sampled during the run, else the maximum)
        sm_mhz = (ck or {}).get("sm_mhz") or 2070.0
        issue_peak = 4.0 * props.multi_processor_count * sm_mhz * 1e6
        issued = roof_pm["warp_inst_per_voxel"] * V / (st_ms["peak_map"] / 1e3)
        roof_pm["issue"] = {"achieved": issued, "peak": issue_peak, "unit": "warp instructions/s",
                            "frac": issued / issue_peak}
    alg_bytes_corr = (4 + 4 * K) * V
    tpv = recorded_traffic("traffic_correlate_n4.md")
    roof_corr = {"bound": "hbm", "kernel": "ttm_correlate (stages prefilter..xpass)",
                 "achieved": alg_bytes_corr / (corr_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                 "peak_source": how, "traffic": None if tpv is None else tpv * V, "bytes_per_voxel": 4 + 4 * K,
                 "traffic_source": "profiles/traffic_correlate_n4.md (ncu dram bytes of every ttm_correlate kernel "
                                   "on 200x256x256, per voxel, scaled to this call; null once the kernels "
                                   "changed)"}
    roof_corr["frac"] = roof_corr["achieved"] / roof_corr["peak"]
    dominant = roof_pm if st_ms["peak_map"] >= corr_ms else roof_corr
    other_roof = roof_corr if dominant is roof_pm else roof_pm

    cpu = None
    extras = {}
    if rank == 0 and ws == 1 and not args.zyx:
        if not args.no_comparators:
            extras["comparators"] = {
                "tm_per_rotation": tm_comparator(ttm, ctx, wl, p, dev, args.tm_rotations),
                "cufft": cufft_comparator(ttm, m, wl, dev, max(2, args.steps // 2))}
            tm = extras["comparators"]["tm_per_rotation"]
            tm["ttm_speedup_vs_45123_rotations"] = tm["implied_45123_rotations_s"] * 1e3 / ms_step
        if not args.no_forms:
            del m
            torch.cuda.empty_cache()
            extras["forms"] = {"spectra_precision_order4": forms_order4(ttm, ctx, wl, dev, max(3, args.steps // 2),
                                                                         2, args.crop_voxels),
                               "plain_fp32_order6_1024x1024x256": plain_order6(ttm, ctx, dev, max(3, args.steps // 2),
                                                                               2, args.crop_voxels)}
        if not args.no_cpu:
            rate, nv, dt, cores = oracle_sample_rate(wl, args.cpu_voxels)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d random valid-interior voxels (%.1f s): local normaliser, direct-sum correlation "
                             "(15 components), 20000-sample + Newton maximiser; setup excluded" % (nv, dt)}

    if rank == 0:
        names = {ttm.TTM_LOCALSUM_DF64: "double-float (FP32 pairs, ~48-bit significand)",
                 ttm.TTM_LOCALSUM_FP64: "fp64"}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if not args.zyx else "ttm_n4_%dx%dx%d_t40" % (X, Y, Z),
                           "shape_zyx": [Z, Y, X], "template": 40, "order_n": n,
                           "components": K, "mask_radius": wl.mask_radius, "rotations_field": 24 * 2048,
                           "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "1gpu",
                           "local_sums": names[ls_main], "spectra": "fp32", "sms": props.multi_processor_count},
                "local_sums_other": {"local_sums": names[other], "value": V * ws / (ms_other / 1e3),
                                     "ms_per_step": ms_other},
                "roofline": dominant, "roofline_other": other_roof, "stages_ms": st_ms, "setup_s": setup_s,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": V * 4,
                        "d2h_bytes_per_step": V * 4 * 4, "ms_per_step": ms_e2e,
                        "how": "pinned host buffers, copy-in / compute / copy-out streams, two buffer sets"},
                "gpu_launches": int(launches), "clocks": ck}
        line.update(extras)
        print(json.dumps(line), flush=True)


# ------------------------------------------------- the three other forms --
#
# Each prints one JSON line with the form's throughput as `value` and the
# plain FP32 form measured in the same run beside it (`plain`), plus the
# stated error. They are not the default workload.

def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _crop_voxels(shape, tshape, edge, count, seed):
    """Random valid-interior voxels of the centred edge^3 crop."""
    import oracle as O
    vox = O.valid_voxels(shape, tshape)
    z, y, x = np.unravel_index(vox, shape)
    c = [d // 2 for d in shape]
    sel = (np.abs(z - c[0]) < edge // 2) & (np.abs(y - c[1]) < edge // 2) & (np.abs(x - c[2]) < edge // 2)
    v = vox[sel]
    return np.sort(np.random.default_rng(seed).choice(v, min(count, v.size), replace=False))


def run_mixed(args):
    """Order 6 on 1024 x 1024 x 256 (48^3 template, r = 19, 2000 copies at
    SNR 0.05): FP32, FP16 and BF16 spectra; error against the FP64 oracle at
    sampled valid voxels of the centred 128^3 crop (the oracle uses its own
    field; both sides use 24 x 64 rotations, which the per-tomogram kernels
    do not depend on)."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    import oracle as O
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    wl = synth.workload_order6()
    gen_s = time.perf_counter() - t0
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    ctx = ttm.Context(0)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=64)
    t = torch.as_tensor(wl.template, device=dev)
    field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device=dev)
    ttm.ttm_build_tensor_field(ctx, t, p, field)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    C = torch.empty((K, Z, Y, X), device=dev)
    score = torch.empty((Z, Y, X), device=dev)
    orient = torch.empty((3, Z, Y, X), device=dev)
    vox = _crop_voxels((Z, Y, X), wl.template.shape, 128, args.crop_voxels, 7)
    tv = torch.as_tensor(vox, device=dev)
    pr = O.Prepared(wl.tomo, wl.template, r)
    ofield = O.tensor_field(pr.tp, O.rotation_set(64), n, 3)
    w, _, _ = O.local_w(pr.g, pr.m, vox, False, pr.floor)
    Cref = O.correlate(pr.g, ofield, vox, False, w)
    sref, _, _ = O.maximise(Cref, n, 3, 20000)
    stream = torch.cuda.current_stream()
    forms = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, prec in (("fp32", ttm.TTM_PREC_FP32), ("fp16", ttm.TTM_PREC_FP16_SPECTRA),
                       ("bf16", ttm.TTM_PREC_BF16_SPECTRA)):
        plan = ttm.Plan(ctx, field, p, (Z, Y, X), precision=prec)
        ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
        ms_corr = _timed(lambda: ttm.ttm_correlate(plan, d_tomo, C), args.steps, args.warmup, stream)
        ms_pm = _timed(lambda: ttm.ttm_peak_map(plan, C, score, orient), args.steps, args.warmup, stream)
        got = C.reshape(K, -1)[:, tv].cpu().numpy().astype(np.float64)
        sg = score.flatten()[tv].cpu().numpy()
        forms[name] = {"correlate_ms": ms_corr, "peak_map_ms": ms_pm, "voxels_per_s": V / ((ms_corr + ms_pm) / 1e3),
                       "correlate_voxels_per_s": V / (ms_corr / 1e3),
                       "C_max_abs_err": float(np.abs(got - Cref).max()),
                       "C_rel_l2_err": float(np.linalg.norm(got - Cref) / np.linalg.norm(Cref)),
                       "C_max_abs": float(np.abs(Cref).max()),
                       "score_max_abs_err": float(np.abs(sg - sref).max())}
        del plan
    ck = clocks.stop()
    pk, how = peaks_file()
    f16 = forms["fp16"]
    alg = (4 + 4 * K) * V
    line = {"metric": METRIC + ", FP16 spectra form", "value": f16["voxels_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f16["correlate_ms"] + f16["peak_map_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 storage / f32 math",
            "data": "synthetic",
            "config": {"workload": wl.name, "shape_zyx": [Z, Y, X], "template": 48, "order_n": n, "components": K,
                       "mask_radius": r, "copies_planted": int(len(wl.planted.centres)), "snr": 0.05,
                       "rotations_field": 24 * 64, "local_sums": "double-float",
                       "error_sample": "%d valid voxels of the centred 128^3 crop" % vox.size,
                       "generation_s": gen_s},
            "forms": forms,
            "vs_plain_fp32": {"whole_step": f16["voxels_per_s"] / forms["fp32"]["voxels_per_s"],
                              "correlate": forms["fp32"]["correlate_ms"] / f16["correlate_ms"],
                              "bf16_correlate": forms["fp32"]["correlate_ms"] / forms["bf16"]["correlate_ms"]},
            "roofline_correlate": {"bound": "hbm", "achieved": alg / (f16["correlate_ms"] / 1e3) / 1e9,
                                   "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s", "peak_source": how,
                                   "traffic": None, "bytes_per_voxel": 4 + 4 * K},
            "clocks": ck}
    line["roofline_correlate"]["frac"] = line["roofline_correlate"]["achieved"] / line["roofline_correlate"]["peak"]
    print(json.dumps(line), flush=True)


def run_quaternion(args):
    """The quaternion form (d' = 4, n = 4, K = 35) on the order-4 volume
    (512 x 512 x 200, 40^3 template, r = 16, 300 copies at SNR 0.1): FP32
    correlation of the 35 components and the maximiser over unit
    quaternions, timed per stage against the d' = 3 plain form on the same
    volume; error against the FP64 oracle (its own d' = 4 field, 24 x 64
    rotations on both sides) at sampled valid voxels of the centred 128^3
    crop, and the rotation error at the planted centres."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    import oracle as O
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    wl = synth.workload_order4()
    gen_s = time.perf_counter() - t0
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = 4, wl.mask_radius
    ctx = ttm.Context(0)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    t = torch.as_tensor(wl.template, device=dev)
    stream = torch.cuda.current_stream()
    vox = _crop_voxels((Z, Y, X), wl.template.shape, 128, args.crop_voxels, 9)
    tv = torch.as_tensor(vox, device=dev)
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for dp in (3, 4):
        K = ttm.ttm_num_components(n, dp)
        p = ttm.params(order_n=n, mask_radius=r, n_rot_base=64, dprime=dp)
        field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device=dev)
        ttm.ttm_build_tensor_field(ctx, t, p, field)
        plan = ttm.Plan(ctx, field, p, (Z, Y, X))
        ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
        C = torch.empty((K, Z, Y, X), device=dev)
        score = torch.empty((Z, Y, X), device=dev)
        orient = torch.empty((dp, Z, Y, X), device=dev)
        frob = torch.empty((Z, Y, X), device=dev)
        ms_corr = _timed(lambda: ttm.ttm_correlate(plan, d_tomo, C), args.steps, args.warmup, stream)
        ms_pm = _timed(lambda: ttm.ttm_peak_map(plan, C, score, orient, frob), args.steps, args.warmup, stream)
        res[dp] = {"components": K, "correlate_ms": ms_corr, "peak_map_ms": ms_pm,
                   "voxels_per_s": V / ((ms_corr + ms_pm) / 1e3)}
        if dp == 4:
            # TTM-ref (Alg. 3) on the P = 300 highest peaks of the Frobenius map (Sec. 3.2)
            pk, _ = ttm.ttm_find_peaks(plan, frob, 300, 2.0 * r)
            ttm.ttm_refine_peaks(plan, t, orient, pk, 3.0)
            t_ref = time.perf_counter()
            ridx, _, _ = ttm.ttm_refine_peaks(plan, t, orient, pk, 3.0)
            res[dp]["refine"] = {"peaks": int(pk.size), "r_s": 3.0, "candidates_per_peak": 123,
                                 "ms": (time.perf_counter() - t_ref) * 1e3,
                                 "moved_frac": float(np.mean(ridx != pk)),
                                 "note": "host-timed call (H2D of the list, kernel, D2H, host selection)"}
        cen = np.array([(int(c[0]) * Y + int(c[1])) * X + int(c[2]) for c in wl.planted.centres])
        oc = orient.reshape(dp, -1)[:, torch.as_tensor(cen, device=dev)].cpu().numpy().T
        if dp == 3:
            ez = np.array([synth.quat_matrix(q)[:, 2] for q in wl.planted.quats])
            ang3 = np.degrees(np.arccos(np.clip(np.abs(np.sum(oc * ez, axis=1)), 0, 1)))
        else:
            got = C.reshape(K, -1)[:, tv].cpu().numpy().astype(np.float64)
            sg = score.flatten()[tv].cpu().numpy()
            qc = oc
        del plan, C, score, orient, field, frob
    ck = clocks.stop()
    pr = O.Prepared(wl.tomo, wl.template, r)
    ofield = O.tensor_field(pr.tp, O.rotation_set(64), n, 4)
    w, _, _ = O.local_w(pr.g, pr.m, vox, False, pr.floor)
    Cref = O.correlate(pr.g, ofield, vox, False, w)
    sref, _, _ = O.maximise(Cref, n, 4, 20000)
    q0 = np.asarray(wl.planted.quats)
    ang = np.degrees(2 * np.arccos(np.clip(np.abs(np.sum(qc * q0, axis=1)), 0, 1)))
    q4 = res[4]
    pk, how = peaks_file()
    K = q4["components"]
    kx = (K + 15) // 16 * 16
    probe_flops = 2.0 * kx * 512 * V
    alg = (4 + 4 * K) * V
    line = {"metric": METRIC + ", quaternion form (d'=4)", "value": q4["voxels_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": q4["correlate_ms"] + q4["peak_map_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ttm_n4_dprime4_512x512x200_t40", "shape_zyx": [Z, Y, X], "template": 40,
                       "order_n": n, "dprime": 4, "components": K, "mask_radius": r,
                       "copies_planted": int(len(cen)), "rotations_field": 24 * 64, "local_sums": "double-float",
                       "error_sample": "%d valid voxels of the centred 128^3 crop" % vox.size,
                       "generation_s": gen_s},
            "forms": {"dprime4": q4, "dprime3": res[3]},
            "accuracy": {"C_max_abs_err": float(np.abs(got - Cref).max()), "C_max_abs": float(np.abs(Cref).max()),
                         "score_max_abs_err": float(np.abs(sg - sref).max()),
                         "planted_rotation_err_deg_median": float(np.median(ang)),
                         "planted_rotation_err_deg_p90": float(np.percentile(ang, 90)),
                         "dprime3_planted_axis_err_deg_median": float(np.median(ang3)),
                         "note": "planted-copy errors at SNR 0.1 in low-passed noise: the d'=3 axis R e_z "
                                 "is no better resolved there, so these are the workload's, not the kernels'"},
            "roofline_correlate": {"bound": "hbm", "achieved": alg / (q4["correlate_ms"] / 1e3) / 1e9,
                                   "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s", "peak_source": how,
                                   "traffic": None, "bytes_per_voxel": 4 + 4 * K},
            "roofline_peak_map": {"bound": "tensor", "achieved": probe_flops / (q4["peak_map_ms"] / 1e3) / 1e12,
                                  "peak": float(pk.get("bf16_tflops", 1900.0)), "unit": "TFLOP/s",
                                  "peak_source": how + " (bf16 dense; the probe product is FP16 mma.sync)",
                                  "note": "probe-product flops only (2 x %d x 512 per voxel) over the whole maximiser"
                                          % kx},
            "clocks": ck}
    for k in ("roofline_correlate", "roofline_peak_map"):
        line[k]["frac"] = line[k]["achieved"] / line[k]["peak"]
    print(json.dumps(line), flush=True)


def run_blocked(args):
    """Block processing (Sec. 3.4) of the order-4 volume (512 x 512 x 200,
    40^3 template, r = 16, n = 4) held in host memory: the 300 highest score
    peaks at exclusion 2r, by z-slabs of 40 and 80 output planes, against the
    whole-volume path (tomogram copied to the device, correlation, maximiser,
    Find Peaks). Each run is timed end to end on the host, per call; the
    blocked calls include their per-slab plan set-up (template spectra on
    each slab grid)."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    dev = torch.device("cuda", 0)
    wl = synth.workload_order4()
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    ctx = ttm.Context(0)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=64)
    t = torch.as_tensor(wl.template, device=dev)
    field = torch.empty((K,) + wl.template.shape, dtype=torch.float64, device=dev)
    ttm.ttm_build_tensor_field(ctx, t, p, field)
    host = torch.as_tensor(wl.tomo).pin_memory()
    plan = ttm.Plan(ctx, field, p, (Z, Y, X))
    d_tomo = torch.empty((Z, Y, X), device=dev)
    C = torch.empty((K, Z, Y, X), device=dev)
    score = torch.empty((Z, Y, X), device=dev)
    orient = torch.empty((3, Z, Y, X), device=dev)

    def whole():
        d_tomo.copy_(host, non_blocking=True)
        ttm.ttm_correlate(plan, d_tomo, C)
        ttm.ttm_peak_map(plan, C, score, orient)
        return ttm.ttm_find_peaks(plan, score, 300, 2 * r)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3, out

    clocks = ClockSampler(0)
    clocks.start()
    ms_whole, (wi, wv) = timed(whole, args.steps)
    res = {}
    for sz in (40, 80):
        # one-shot call (plans built per call) and a session kept across
        # calls (plans and buffers once; pinned tomogram, uploads overlapping
        # the slab kernels)
        ms1, (bi, bv) = timed(lambda: ttm.ttm_blocked_peaks(ctx, field, p, wl.tomo, sz, 300, 2 * r), 1)
        sess = ttm.Blocked(ctx, field, p, (Z, Y, X), sz)
        ms, (si, sv) = timed(lambda: sess.run(host, 300, 2 * r), max(1, args.steps // 2))
        del sess
        res[str(sz)] = {"ms": ms, "voxels_per_s": V / (ms / 1e3), "one_shot_ms": ms1,
                        "slabs": int(len(ttm.ttm_slab_ranges(Z, 40, sz))),
                        "same_list_as_whole": bool(list(bi) == list(wi) and list(si) == list(wi)),
                        "max_value_diff": float(np.abs(sv - wv).max()) if len(sv) == len(wv) else None}
    ck = clocks.stop()
    best = min(res.values(), key=lambda d: d["ms"])
    line = {"metric": METRIC + ", block processing (peaks)", "value": best["voxels_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": best["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ttm_n4_512x512x200_t40_blocked", "shape_zyx": [Z, Y, X], "order_n": n,
                       "components": K, "P": 300, "min_dist": 2 * r,
                       "timing": "host clock per call, end to end; value: a session kept across calls"},
            "slabs": res, "whole_volume": {"ms": ms_whole, "voxels_per_s": V / (ms_whole / 1e3)},
            "clocks": ck}
    print(json.dumps(line), flush=True)


def run_study(args):
    """Synthetic accuracy study (the analogue of Sec. 5.1, Tabs. 1-2 and the
    SNR sweep): for each template (six-Gaussian blob, cylinder, L-shape;
    21^3, r = 9), a tomogram with a 5 x 5 x 5 grid of 125 copies at uniform
    random rotations, noise-free or with white noise at SNR 1 and 0.1; the
    quaternion form (d' = 4) at n = 2 and 4; the 125 highest peaks of the
    Frobenius map at exclusion 2r (TTM), then TTM-ref (r_s = 3). Each planted
    copy is matched to the nearest peak within 6 voxels. Position error is
    the Euclidean distance in voxels; rotation error 2 acos |q . q0| in
    degrees, except for the cylinder, whose roll is undefined: the angle
    between the axes R e_z."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    dev = torch.device("cuda", 0)
    ctx = ttm.Context(0)
    N, r = 21, 9.0
    templates = {"blob6": synth.gaussian_blob_template(N, seed=11), "cylinder": synth.cylinder_template(N),
                 "l_shape": synth.l_shape_template(N)}
    rows = []
    t_start = time.perf_counter()
    for name, tmpl in templates.items():
        tmpl = tmpl.astype(np.float32)
        t = torch.as_tensor(tmpl, device=dev)
        for n in (2, 4):
            p = ttm.params(order_n=n, mask_radius=r, n_rot_base=2048, dprime=4)
            K = ttm.ttm_num_components(n, 4)
            field = torch.empty((K, N, N, N), dtype=torch.float64, device=dev)
            ttm.ttm_build_tensor_field(ctx, t, p, field)
            for snr in (None, 1.0, 0.1):
                vol, pl = synth.grid_tomogram(tmpl, 5, 26, 6, 31, snr, r)
                shape = vol.shape
                plan = ttm.Plan(ctx, field, p, shape, work_shape=ttm.ttm_autotune_shape(ctx, shape))
                Zw, Yw, Xw = plan.shape
                C = torch.empty((K, Zw, Yw, Xw), device=dev)
                score = torch.empty((Zw, Yw, Xw), device=dev)
                q = torch.empty((4, Zw, Yw, Xw), device=dev)
                F = torch.empty((Zw, Yw, Xw), device=dev)
                ttm.ttm_correlate(plan, torch.as_tensor(vol, device=dev), C)
                ttm.ttm_peak_map(plan, C, score, q, F)
                pk, _ = ttm.ttm_find_peaks(plan, F, 125, 2 * r)
                ridx, rq, _ = ttm.ttm_refine_peaks(plan, t, q, pk, 3.0)
                qmap = q.reshape(4, -1)[:, torch.as_tensor(pk, device=dev)].cpu().numpy().T

                def zyx(i):
                    return np.stack([i // (Yw * Xw), (i // Xw) % Yw, i % Xw], axis=1).astype(float)

                def rot_err(qa, q0):
                    if len(qa) == 0:
                        return np.zeros(0)
                    if name == "cylinder":
                        a = np.array([synth.quat_matrix(v)[:, 2] for v in qa])
                        b = np.array([synth.quat_matrix(v)[:, 2] for v in q0])
                        return np.degrees(np.arccos(np.clip(np.abs(np.sum(a * b, 1)), 0, 1)))
                    return np.degrees(2 * np.arccos(np.clip(np.abs(np.sum(qa * q0, 1)), 0, 1)))

                row = {"template": name, "n": n, "snr": snr if snr is not None else "inf"}
                for tag, pos, qq in (("ttm", zyx(pk), qmap), ("ttm_ref", zyx(ridx), rq)):
                    d = np.linalg.norm(pos[None, :, :] - np.asarray(pl.centres, float)[:, None, :], axis=2)
                    j = np.argmin(d, axis=1)
                    ok = d[np.arange(len(j)), j] <= 6.0
                    pe = d[np.arange(len(j)), j][ok]
                    re = rot_err(qq[j[ok]], np.asarray(pl.quats)[ok])
                    row[tag] = {"found": int(ok.sum()), "pos_mean": float(pe.mean()) if ok.any() else None,
                                "pos_max": float(pe.max()) if ok.any() else None,
                                "rot_mean_deg": float(re.mean()) if ok.any() else None,
                                "rot_max_deg": float(re.max()) if ok.any() else None}
                rows.append(row)
                del plan, C, score, q, F
    key = next(rw for rw in rows if rw["template"] == "blob6" and rw["n"] == 4 and rw["snr"] == "inf")
    line = {"metric": "TTM-ref mean rotation error, noise-free, n = 4 (synthetic study)",
            "value": key["ttm_ref"]["rot_mean_deg"], "unit": "deg", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "ttm_study_grid125_t21", "tomogram": "137^3, 5x5x5 copies",
                                            "templates": list(templates), "dprime": 4, "orders": [2, 4],
                                            "snr": ["inf", 1.0, 0.1], "rotations_field": 24 * 2048,
                                            "r_s": 3.0},
            "rows": rows, "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Order 6 on the same 1024 x 1024 x 256 volume: the network is trained
    on 10^6 (C / ||C||_F, plain maximiser direction) pairs from a separate
    seeded 160^3 tomogram with the same template, then the learned
    maximiser is timed against the plain one on the big volume and checked
    by it over every valid voxel."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    wl = synth.workload_order6()
    gen_s = time.perf_counter() - t0
    Z, Y, X = wl.tomo.shape
    V = Z * Y * X
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    ctx = ttm.Context(0)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=2048)
    stream = torch.cuda.current_stream()
    # training pairs
    tshape = (160, 160, 160)
    tvol, _ = synth.make_tomogram(tshape, wl.template, r, 60, 20240905, snr=0.05)
    Mt = ttm.Matcher(ctx, wl.template, p, tshape, device=dev)
    Mt.run(torch.as_tensor(tvol, device=dev))
    b = Mt.plan.valid_box()
    zz, yy, xx = np.meshgrid(np.arange(b[0], b[1]), np.arange(b[2], b[3]), np.arange(b[4], b[5]), indexing="ij")
    idx = ((zz * tshape[1] + yy) * tshape[2] + xx).ravel()
    idx = np.random.default_rng(1).choice(idx, min(10 ** 6, idx.size), replace=False)
    dX = torch.empty((idx.size, K), device=dev)
    dU = torch.empty((idx.size, 3), device=dev)
    ttm.ttm_mlp_make_pairs(ctx, Mt.C, n, Mt.orient, torch.as_tensor(idx, device=dev), dX, dU)
    net = ttm.Mlp(ctx, K, seed=5)
    net.set_precision(ttm.TTM_MLP_BF16)   # BF16 tensor-core products, FP32 master weights
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(20):
        loss = net.train(dX, dU, epochs=1, batch=4096, lr=1e-3, seed=100 + ep)
    for ep in range(10):
        loss = net.train(dX, dU, epochs=1, batch=4096, lr=3e-4, seed=200 + ep)
    train_s = time.perf_counter() - t0
    # the network's inference alone (BF16 tensor cores) on the training rows,
    # for the time breakdown
    dUi = torch.empty_like(dU)
    ms_infer = _timed(lambda: net.infer(dX, dUi), 3, 1, stream)
    infer_ns_per_voxel = ms_infer * 1e6 / dX.shape[0]
    field = Mt.field
    del Mt, dX, dU
    torch.cuda.empty_cache()
    # the big volume
    plan = ttm.Plan(ctx, field, p, (Z, Y, X))
    ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
    d_tomo = torch.as_tensor(wl.tomo, device=dev)
    C = torch.empty((K, Z, Y, X), device=dev)
    sp = torch.empty((Z, Y, X), device=dev)
    op = torch.empty((3, Z, Y, X), device=dev)
    sl = torch.empty((Z, Y, X), device=dev)
    ol = torch.empty((3, Z, Y, X), device=dev)
    clocks = ClockSampler(0)
    clocks.start()
    ms_corr = _timed(lambda: ttm.ttm_correlate(plan, d_tomo, C), args.steps, args.warmup, stream)
    ms_plain = _timed(lambda: ttm.ttm_peak_map(plan, C, sp, op), args.steps, args.warmup, stream)
    launches0 = ttm.ttm_kernel_launches()
    ms_learn = _timed(lambda: ttm.ttm_peak_map(plan, C, sl, ol, mlp=net), args.steps, args.warmup, stream)
    launches = (ttm.ttm_kernel_launches() - launches0) / (args.steps + args.warmup)
    ck = clocks.stop()
    fb = ttm.ttm_plan_fallback_count(plan)
    bb = plan.valid_box()
    d = (sl - sp)[bb[0]:bb[1], bb[2]:bb[3], bb[4]:bb[5]]
    viol = int((d < -1e-4).sum())
    nvalid = d.numel()
    # orientation agreement where the scores agree
    ang = torch.rad2deg(torch.acos(torch.clamp((ol * op).sum(0).abs(), 0, 1)))[bb[0]:bb[1], bb[2]:bb[3], bb[4]:bb[5]]
    vl = V / ((ms_corr + ms_learn) / 1e3)
    vp = V / ((ms_corr + ms_plain) / 1e3)
    mlp_flops = 2.0 * (K * 128 + 128 * 128 + 128 * 3) * V
    line = {"metric": METRIC + ", learned warm-start form", "value": vl, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_corr + ms_learn,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (MLP bf16)",
            "data": "synthetic",
            "config": {"workload": wl.name, "shape_zyx": [Z, Y, X], "order_n": n, "components": K,
                       "mlp": "%d-128-128-3 GELU(tanh), unit output" % K, "train_pairs": int(idx.size),
                       "training": "bf16 operands on the tensor cores, fp32 accumulation and master weights",
                       "train_volume": "160^3, same template, seed 20240905", "epochs": 30,
                       "generation_s": gen_s},
            "plain": {"value": vp, "peak_map_ms": ms_plain},
            "learned": {"peak_map_ms": ms_learn, "correlate_ms": ms_corr, "train_s": train_s,
                        "final_batch_loss": loss, "fallback_voxels": fb, "fallback_frac": fb / V,
                        "kernel_launches_per_call": launches},
            "check_vs_plain": {"valid_voxels": nvalid, "violations_below_plain_1e-4": viol,
                      "min_score_diff": float(d.min().item()), "max_score_diff": float(d.max().item()),
                      "orientation_deg_p99": float(torch.quantile(ang.flatten()[::97].float(), 0.99).item())},
            "vs_plain": {"whole_step": vl / vp, "peak_map": ms_plain / ms_learn},
            "breakdown": {"plain_maximiser_ns_per_voxel": ms_plain * 1e6 / V,
                          "network_inference_alone_ns_per_voxel": infer_ns_per_voxel,
                          "learned_maximiser_ns_per_voxel": ms_learn * 1e6 / V,
                          "note": "the learned form runs the network, the probe product and check, and the plain "
                                  "maximiser on every rejected voxel; it cannot be faster than plain when the "
                                  "network alone costs more than the plain maximiser's whole start search"},
            "roofline_mlp": {"bound": "tensor", "achieved": mlp_flops / (ms_learn / 1e3) / 1e12,
                             "peak": float(peaks_file()[0].get("bf16_tflops", 1900.0)), "unit": "TFLOP/s",
                             "note": "network flops only over the whole learned maximiser time (mma.sync BF16)"},
            "clocks": ck}
    line["roofline_mlp"]["frac"] = line["roofline_mlp"]["achieved"] / line["roofline_mlp"]["peak"]
    print(json.dumps(line), flush=True)


def run_batched(args):
    """64 sub-tomograms of uneven sizes (each axis uniform in 96..256) x 8
    templates (32^3, r = 12, order 4): the batched form (autotuned working
    grids, one preparation per sub-tomogram, valid-box maximiser, concurrent
    branches, one graph launch) against the plain form (one padded plan per
    pair, correlate + whole-grid maximiser in sequence) on the first
    `--plain-tomos` sub-tomograms."""
    import torch
    from paper_2408_02398_gb300 import build, synth
    build.build()
    from paper_2408_02398_gb300 import ttm
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    wl = synth.workload_batched()
    gen_s = time.perf_counter() - t0
    n, r = wl.order_n, wl.mask_radius
    K = ttm.ttm_num_components(n)
    ctx = ttm.Context(0)
    p = ttm.params(order_n=n, mask_radius=r, n_rot_base=2048)
    fields = []
    for tm in wl.templates:
        f = torch.empty((K,) + tm.shape, dtype=torch.float64, device=dev)
        ttm.ttm_build_tensor_field(ctx, torch.as_tensor(tm, device=dev), p, f)
        fields.append(f)
    tomos = [torch.as_tensor(t, device=dev) for t in wl.tomos]
    items = []
    for i, t in enumerate(wl.tomos):
        for j in range(len(fields)):
            items.append((i, j, torch.empty(t.shape, device=dev), torch.empty((3,) + t.shape, device=dev), None))
    vox_total = sum(int(np.prod(t.shape)) for t in wl.tomos) * len(fields)
    t0 = time.perf_counter()
    B = ttm.Batch(ctx, p, fields, tomos, items, n_branches=args.branches,
                  flags=ttm.TTM_BATCH_AUTOTUNE | ttm.TTM_BATCH_LOCALSUM_DF64)
    create_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = ttm.ttm_kernel_launches()
    ms_b = _timed(lambda: B.run(), args.steps, args.warmup, stream)
    ck = clocks.stop()
    vb = vox_total / (ms_b / 1e3)
    # the plain form on the same pairs (all of them unless --plain-tomos
    # limits the tomograms): one padded plan per pair, correlate + maximiser
    # over the whole working grid, timed per pair after one warm-up call
    sub = list(range(len(wl.tomos) if args.plain_tomos <= 0 else min(args.plain_tomos, len(wl.tomos))))
    ms_p = 0.0
    vox_p = 0
    for i in sub:
        shape = wl.tomos[i].shape
        work = tuple(next_smooth7(d) for d in shape)
        for j in range(len(fields)):
            plan = ttm.Plan(ctx, fields[j], p, shape, work_shape=work)
            ttm.ttm_plan_set_localsum(plan, ttm.TTM_LOCALSUM_DF64)
            Cw = torch.empty((K,) + work, device=dev)
            sw = torch.empty(work, device=dev)
            ow = torch.empty((3,) + work, device=dev)

            def step():
                ttm.ttm_correlate(plan, tomos[i], Cw)
                ttm.ttm_peak_map(plan, Cw, sw, ow)
            ms_p += _timed(step, 1, 1, stream)
            vox_p += int(np.prod(shape))
            del plan, Cw, sw, ow
    vp = vox_p / (ms_p / 1e3)
    sizes = [t.shape for t in wl.tomos]
    works = [B.work_shape(i) for i in range(len(wl.tomos))]
    line = {"metric": METRIC + ", batched form", "value": vb, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "pairs": len(items), "voxels_per_step": vox_total,
                       "order_n": n, "components": K, "template": 32, "mask_radius": r,
                       "branches": args.branches, "copies_planted": int(sum(wl.copies)),
                       "mean_padding": float(np.mean([np.prod(w) / np.prod(s) for w, s in zip(works, sizes)])),
                       "create_s": create_s, "generation_s": gen_s, "autotuned_lengths": ttm.ttm_autotune_entries(ctx)},
            "plain": {"value": vp, "pairs": len(sub) * len(fields), "same_pairs": len(sub) == len(wl.tomos),
                      "note": "one plan per pair on the next 7-smooth grid, correlate + whole-grid maximiser"},
            "vs_plain": vb / vp, "graph_launches_per_step": 1, "clocks": ck}
    print(json.dumps(line), flush=True)


def run_qmap(args):
    """A small case for kernel captures of the quaternion maximiser: a d' = 4
    plan (n = 4, 16^3 template, r = 7, 24 x 64 field rotations) on a
    --zyx white-noise tomogram (default 64 x 256 x 256); one correlation,
    then --steps timed calls of the maximiser (CUDA events)."""
    import torch
    from paper_2408_02398_gb300 import build
    build.build()
    from paper_2408_02398_gb300 import ttm
    shape = tuple(int(v) for v in (args.zyx or "64,256,256").split(","))
    ctx = ttm.Context(0)
    tmpl = synth.gaussian_blob_template(16, seed=5)
    p = ttm.params(order_n=4, mask_radius=7.0, n_rot_base=64, dprime=4)
    m = ttm.Matcher(ctx, tmpl, p, shape)
    tomo = torch.as_tensor(synth.normals(3, 1, int(np.prod(shape))).reshape(shape).astype(np.float32), device="cuda")
    m.run(tomo)
    torch.cuda.synchronize()
    ms = _step_ms(lambda: ttm.ttm_peak_map(m.plan, m.C, m.score, m.orient, m.frob), args.steps, 0,
                  torch.cuda.current_stream())
    print(json.dumps({"workload": "qmap", "shape_zyx": list(shape), "peak_map_ms": ms,
                      "voxels_per_s": float(np.prod(shape)) / (ms / 1e3)}), flush=True)


def next_smooth7(n):
    L = max(n, 2)
    while True:
        m = L
        for q in (2, 3, 5, 7):
            while m % q == 0:
                m //= q
        if m == 1:
            return L
        L += 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-voxels", type=int, default=250000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the forms block of the default line")
    ap.add_argument("--no-comparators", action="store_true", help="skip the TM and cuFFT comparators")
    ap.add_argument("--tm-rotations", type=int, default=256)
    ap.add_argument("--localsum", default="df64", choices=["df64", "fp64"],
                    help="arithmetic of the local sums of Eq. 2")
    ap.add_argument("--workload", default="order4", choices=["order4", "mixed", "learned", "batched", "quaternion", "blocked", "study", "qmap"],
                    help="order4: the default plain FP32 workload; the others time one form against it")
    ap.add_argument("--zyx", default="", help="Z,Y,X of a smaller order-4 volume (profiling captures)")
    ap.add_argument("--crop-voxels", type=int, default=200)
    ap.add_argument("--branches", type=int, default=4)
    ap.add_argument("--plain-tomos", type=int, default=0, help="batched workload: time the plain form on the "
                    "first N tomograms only (0: all, the same pairs as the batch)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "quaternion":
        run_quaternion(args)
    elif args.workload == "blocked":
        run_blocked(args)
    elif args.workload == "study":
        run_study(args)
    elif args.workload == "qmap":
        run_qmap(args)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
