"""Throughput of the PRENOM object-NeRF training step (fwd + bwd + Adam) on GB300.

Headline workload: 32 heterogeneous objects trained in ONE batched step -- the
category table's architectures (hash grid L=16, F=2, T = 2^14..2^19, res
16..2048; MLP width 16/32/64, 1-3 hidden layers), 256..8192 rays per object
(a projected-area share) x 48 samples drawn by the prior sampler (N_c = 48)
over each object's 64^3 prior grid of a random CSG shape, FP16 tensor-core MLP
with FP32 accumulation and master weights.  One step = sampling, encoding,
MLP, compositing, loss, backward and Adam for every parameter of every object.
Beside it: the same 32 objects trained one plain FP32 step at a time (the
metric's "plain FP32" side), and the equal-error check of the pair: both
trained for a fixed step budget over 3 seeds, held-out colour MSE and depth L1.
Under torchrun each rank trains its own copy of the workload (weak scaling, no
collective: objects are independent).

Timing: after the set-up (autotuner, graph capture) W warm-up steps, K timed
steps from initialisation (`from_init`), untimed training until every object has
taken TRAIN_AGE steps, the autotuner once more on the trained objects
(PRENOM_FLAG_RETUNE; set-up, it changes no state), 3 warm-up steps, then the K
headline steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead (bounded ray sample per step, extrapolated).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NeRF training samples/s (fwd+bwd+Adam), batched FP16 vs plain FP32, at equal error"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock
PRECISION = {"fp32": 0, "fp16": 1, "bf16": 2}
DTYPE = {"fp32": "f32", "fp16": "f16 MLP / f32 accumulate", "bf16": "bf16 MLP / f32 accumulate"}
FORM = {"fp32": "fp32", "fp16": "mixed precision (FP16 tensor-core MLP, FP32 master weights)",
        "bf16": "mixed precision (BF16 tensor-core MLP, FP32 master weights)"}

# ---- the 32-object batched workload (the headline)
# (log2 T, width, hidden layers) per object category, a stand-in for the
# architecture table the paper's genetic search produces (its values are not
# printed): display, laptop, chair, mug, ball, keyboard, mouse, book, plant.
CATEGORY_ARCHS = [(17, 32, 1), (16, 32, 2), (19, 64, 3), (18, 64, 2), (14, 16, 1), (17, 32, 2), (14, 16, 1),
                  (15, 16, 2), (19, 64, 3)]
BATCHED_OBJECTS, BATCHED_NR, BATCHED_SEED, GRID_RES = 32, 48, 7, 64
# The headline steps are timed once every object has taken at least this many
# training steps.  From initialisation every sample carries gradient; within the
# first 50-100 steps the surfaces turn opaque, the transmittance of the samples
# behind them underflows to zero, their gradients are exactly zero and the
# scatter skips their addends (measured: the 32-object step takes 3.67 ms over
# the objects' steps 5-24 and 3.28 ms after their 100th).  The rate from
# initialisation is reported beside it.
TRAIN_AGE = 100
WORKLOAD = ("32 heterogeneous objects in one batched step: category-table architectures (L=16 F=2, T 2^14..2^19, "
            "res 16..2048, MLP width 16/32/64 with 1-3 hidden layers), 256..8192 rays per object x 48 samples "
            "from the prior sampler (Nc=48) over 64^3 prior grids of random CSG shapes, 480x640 views, "
            "depth noise 2 mm, lambda_d 0.1, lambda_sigma 1e-3")

# ---- the single full-size object (reported under compare)
ARCH = dict(L=16, F=2, log2T=19, n_min=16, n_max=2048, width=64, hidden=2, lambda_d=0.1, lambda_sigma=0.0)
N_RAYS, NR, NC = 4096, 64, 64
SINGLE_WORKLOAD = ("single object at full size: hash grid L=16 F=2 T=2^19 res 16..2048, MLP 32-64-64-4, 4096 rays "
                   "x 64 samples/step from the prior sampler (Nc=64) over a 64^3 prior grid, random CSG scene")


def mlp_macs(W, H, IN=32):
    return W * IN + (H - 1) * W * W + 4 * W


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]), src="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, bf16=1900.0, src="fallback")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def batched_specs(seed: int = BATCHED_SEED):
    """(log2 T, W, H, rays) of the 32 objects: the category table's architectures,
    rays per object 32 * round(8 * 2^(5 a)), a ~ U[0,1) (256..8192, a projected-area share)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(BATCHED_OBJECTS):
        log2T, W, H = CATEGORY_ARCHS[i % len(CATEGORY_ARCHS)]
        out.append(dict(log2T=log2T, W=W, H=H, rays=int(32 * round(8 * 2 ** (5 * rng.random())))))
    return out


def batched_arch_dict(sp):
    return dict(L=16, F=2, log2T=sp["log2T"], n_min=16, n_max=2048, width=sp["W"], hidden=sp["H"], lambda_d=0.1,
                lambda_sigma=1e-3)


def batched_host(seed: int = BATCHED_SEED, only=None, pool_factor: int = 4):
    """Host data of the 32 objects: a random CSG scene and 64^3 prior grid each,
    a ray pool from 8 views of 480x640 (pool_factor x its rays, at least 4096),
    and four ray sets (rays, stratified uniforms, background colours)."""
    from synth import (cameras_on_sphere, make_ray_pool, prior_grid, random_colours, sample_batch,
                       scene_random_csg, stratified_uniforms)

    out = []
    for i, sp in enumerate(batched_specs(seed)):
        if only is not None and i not in only:
            continue
        rays = sp["rays"]
        sc = scene_random_csg(1000 * seed + i)
        pool = make_ray_pool(sc, cameras_on_sphere(8, 2.0, 50, 480, 640, i), max(pool_factor * rays, 4096), i,
                             depth_noise=0.004)
        sets = []
        for j in range(4):
            b = sample_batch(pool, rays, 10 * i + j)
            b["uniforms"] = stratified_uniforms(rays, BATCHED_NR, 20 * i + j)
            b["c_rand"] = random_colours(rays, 30 * i + j)
            sets.append(b)
        out.append(dict(index=i, spec=sp, scene=sc, grid=prior_grid(sc, GRID_RES, i), pool=pool, sets=sets))
    return out


def batched_totals(specs):
    samples = sum(sp["rays"] * BATCHED_NR for sp in specs)
    return samples, sum(sp["rays"] for sp in specs)


# NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*) that the record names
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}


class ClockSampler:
    """SM clock and clock-event (throttle) reasons during the timed region.

    Read through NVML (the driver's libnvidia-ml, queried every 5 ms from a
    thread) where it loads, so that a timed region of a few tens of ms still
    holds several samples; else nvidia-smi every 100 ms.  Only reads: no
    setting of the GPU is changed."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.005

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.rows = []  # (wall time, sm MHz, max sm MHz, [reason names])
        self.source = None

    def _nvml_start(self) -> bool:
        import ctypes
        import threading

        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            get_sm, get_max = lib.nvmlDeviceGetClockInfo, lib.nvmlDeviceGetMaxClockInfo
            try:
                get_reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:  # the older name of the same query
                get_reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
            handle = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByUUID(self.gpu_id.encode(), ctypes.byref(handle)) != 0:
                lib.nvmlShutdown()
                return False
        except Exception:
            return False
        self._lib, self._handle = lib, handle
        self._stop = threading.Event()

        def loop():
            sm, mx, reasons = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            while not self._stop.is_set():
                ok = (get_sm(handle, 1, ctypes.byref(sm)) == 0 and  # 1: NVML_CLOCK_SM
                      get_max(handle, 1, ctypes.byref(mx)) == 0 and get_reasons(handle, ctypes.byref(reasons)) == 0)
                if ok:
                    names = [nm for bit, nm in NVML_REASONS.items() if reasons.value & bit]
                    self.rows.append((time.time(), float(sm.value), float(mx.value), names))
                time.sleep(self.PERIOD_S)

        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        self.source = "nvml, every 5 ms"
        return True

    def __enter__(self):
        if not self._nvml_start():
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                     "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi, every 100 ms"
            except Exception:
                self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.25)
        if self.source and self.source.startswith("nvml"):
            self._stop.set()
            self._thread.join(timeout=5)
            self._lib.nvmlShutdown()
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.rows = self.parse_smi(out.splitlines())
        return False

    @staticmethod
    def parse_smi(lines):
        import datetime

        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             [nm for nm, v in zip(names, parts[5:9]) if v.lower() == "active"]))
            except ValueError:
                continue
        return rows

    def mark(self, t0: float, t1: float):
        """Wall-clock bounds of the timed region (samples outside it are dropped)."""
        self.window = (t0, t1)

    def summary(self):
        rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        t0, t1 = getattr(self, "window", (rows[0][0], rows[-1][0]))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        note = "inside the timed region"
        if not inside:  # region shorter than the sampling period: nearest sample
            mid = 0.5 * (t0 + t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            note = "nearest sample (timed region shorter than the sampling period)"
        reasons = sorted({nm for r in inside for nm in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "note": note, "source": self.source}


def gpu_identifier(dev: int) -> str:
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


def profiled(kernel: str):
    """A kernel's record in the committed ncu summary (DRAM bytes per launch and,
    where captured, L2 throughput and L2 reduction requests), if it was taken
    on the current kernel sources (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except Exception:
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for fn in rec.get("sources", []):
        with open(os.path.join(ROOT, fn), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec


def profiled_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary (None if it was
    taken on other kernel sources)."""
    rec = profiled(kernel)
    return float(rec["dram_bytes_per_launch"]) if rec else None


def profiled_l2(kernel: str, samples: int):
    """The launch's L2 figures from the committed ncu summary: lts__throughput
    (% of peak) and, for the scatter, L2 reduction requests per sample."""
    rec = profiled(kernel)
    if not rec or "lts_pct" not in rec:
        return None
    out = {"lts_pct_of_peak": rec["lts_pct"]}
    if rec.get("l2_red_requests"):
        out["l2_red_requests"] = rec["l2_red_requests"]
        out["red_per_sample"] = round(rec["l2_red_requests"] / max(samples, 1), 3)
    return out




# ------------------------------------------------------------------- oracle arm
def _oracle_objects(only=None):
    """The batched workload for the oracle: per object (index, Arch, grid, theta
    in FP64, ray set 0 with its uniforms and colours)."""
    import oracle as orc
    from synth import init_params

    objs = []
    for h in batched_host(only=only):
        a = orc.Arch(**batched_arch_dict(h["spec"]))
        theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 5 + h["index"]).astype(np.float64)
        objs.append((h["index"], a, h["grid"], theta, h["sets"][0]))
    return objs


def _oracle_rays(obj, budget_s: float):
    """Forward + backward of the oracle on 16-ray chunks of one object's batch
    until budget_s (at least one chunk): (rays done, seconds)."""
    import oracle as orc

    _, a, grid, theta, b = obj
    n = b["o"].shape[0]
    done, spent, chunk = 0, 0.0, 16
    while (spent < budget_s or done == 0) and done < n:
        sl = slice(done, done + chunk)
        sub = {k: b[k][sl] for k in ("o", "d", "rgb", "depth", "is_obj")}
        t0 = time.perf_counter()
        orc.batch(a, theta, grid, sub, BATCHED_NR, BATCHED_NR, u=b["uniforms"][sl], c_rand=b["c_rand"][sl],
                  want_grad=True, want_samples=False)
        spent += time.perf_counter() - t0
        done += min(chunk, n - done)
    return done, spent


def oracle_adam_seconds_per_param():
    """Seconds per parameter of the oracle's dense Adam pass (timed on 12.2 M parameters)."""
    import oracle as orc

    n = 12_204_288
    theta, m, v, g = (np.full(n, 1e-3) for _ in range(4))  # written once, so no first-touch page faults are timed
    t0 = time.perf_counter()
    orc.adam(theta, m, v, g, 1, 1e-2)
    return (time.perf_counter() - t0) / n


def oracle_param_total():
    import oracle as orc

    return sum(orc.param_count(orc.Arch(**batched_arch_dict(sp))) for sp in batched_specs())


def oracle_step_seconds(per_obj, cores: int, adam_s: float):
    """Step time extrapolated from per-object (rays done, seconds): every object's
    rays at its measured rate, the objects spread evenly over `cores` (they are
    independent), plus one single-thread Adam pass over every parameter."""
    specs = batched_specs()
    rays_s = sum(specs[i]["rays"] * t / max(d, 1) for i, (d, t) in per_obj.items())
    return rays_s / cores + adam_s


_BARRIER = None


def _oracle_pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    """One host process of the oracle timing: its objects' workloads are built,
    then (after a barrier shared with the other processes) each object's rays
    run for budget_s: {index: (rays, seconds)}."""
    only, budget_s = job
    objs = _oracle_objects(only=set(only))
    if _BARRIER is not None:
        _BARRIER.wait()
    return {o[0]: _oracle_rays(o, budget_s) for o in objs}


def oracle_timing(budget_s: float, cores: int):
    """The oracle, as it stands, in `cores` spawned host processes (none inherits
    a CUDA context), the 32 objects dealt round-robin, each object run for
    budget_s * cores / 32 seconds: {index: (rays, seconds)}."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores, timeout=300)
    per = budget_s * cores / BATCHED_OBJECTS
    jobs = [(list(range(k, BATCHED_OBJECTS, cores)), per) for k in range(cores)]
    with ctx.Pool(cores, initializer=_oracle_pool_init, initargs=(barrier,)) as pool:
        res = pool.map_async(_oracle_worker, jobs, chunksize=1).get(timeout=budget_s + 600)
    out = {}
    for r in res:
        out.update(r)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # per step a ray sample of at most 4 s over the 32 objects, shrunk so that
    # all K steps take about 150 s at most (every object runs at least one chunk)
    budget = min(float(os.environ.get("PRENOM_ORACLE_BUDGET_S", "4")), 150.0 / max(args.steps, 1))
    objs = _oracle_objects()  # built once
    adam_s = oracle_adam_seconds_per_param() * oracle_param_total()
    samples, _ = batched_totals(batched_specs())
    for _ in range(min(args.warmup, 1)):
        for o in objs:
            _oracle_rays(o, 0.0)
    vals, times = [], []
    for _ in range(args.steps):
        per_obj = {o[0]: _oracle_rays(o, budget / len(objs)) for o in objs}
        step_s = oracle_step_seconds(per_obj, 1, adam_s)
        vals.append(samples / step_s)
        times.append(step_s)
    value = statistics.median(vals)
    rays = sum(d for d, _ in per_obj.values())
    sample = (f"per step: {rays} of the step's rays fwd+bwd (each of the 32 objects for {budget / len(objs):.2f} s, "
              f"at least 16 rays) + one full Adam pass over every parameter ({adam_s:.2f} s, timed once on 12.2 M "
              f"parameters and scaled), extrapolated to the whole step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "form": "FP64 CPU oracle, 1 thread"},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- GPU arm
def _device_batches(batches_np, obj, stream):
    import torch

    out = []
    with torch.cuda.stream(stream):
        for b in batches_np:
            d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in b.items()}
            d["obj"] = obj
            out.append(d)
    return out


def _pack(batches_np):
    """All arrays of a list of host batches as one pinned byte block at 256-byte
    aligned offsets; returns (block, layout), layout[j] = [(key, offset, shape,
    dtype)] of batch j.  Blocks packed from lists of the same shapes share a layout."""
    import torch

    layout, off = [], 0
    for b in batches_np:
        ent = []
        for k, v in b.items():
            a = np.ascontiguousarray(v)
            ent.append((k, off, a.shape, a.dtype))
            off += -(-a.nbytes // 256) * 256
        layout.append(ent)
    buf = np.zeros(off, np.uint8)
    for b, ent in zip(batches_np, layout):
        for k, o, shape, dtype in ent:
            a = np.ascontiguousarray(b[k], dtype=dtype)
            assert a.shape == shape
            buf[o:o + a.nbytes] = a.reshape(-1).view(np.uint8)
    return torch.from_numpy(buf).pin_memory(), layout


def _unpack(buf, ent):
    """Typed views of one batch of a packed block (host or device) by its layout entry."""
    import torch

    tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.uint8): torch.uint8, np.dtype(np.int32): torch.int32}
    out = {}
    for k, o, shape, dtype in ent:
        n = int(np.prod(shape)) * np.dtype(dtype).itemsize
        out[k] = buf[o:o + n].view(tdt[np.dtype(dtype)]).view(shape)
    return out


def _time(stream, fn, steps, warmup, barrier=lambda: None, clocks=None):
    """Device time (ms) of `steps` calls of fn(i) on `stream`, after `warmup` calls."""
    import torch

    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    ev0.record(stream)
    for i in range(steps):
        fn(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.mark(w0, time.time())
    barrier()
    return ev0.elapsed_time(ev1)


def _batched_objects(pkg, ctx, stream, precision, host, thetas=None, features=0):
    """Objects of the batched workload on the device: ids and the four ray sets
    as lists of device batches (one per object)."""
    objs = []
    for k, h in enumerate(host):
        arch = pkg.make_arch(**batched_arch_dict(h["spec"]), precision=PRECISION[precision], features=features)
        obj = ctx.create_object(arch, None if thetas is None else thetas[k])
        ctx.set_prior_grid(obj, h["grid"])
        objs.append(obj)
    sets = [[_device_batches([h["sets"][j]], o, stream)[0] for h, o in zip(host, objs)] for j in range(4)]
    return objs, sets


def _e2e(ctx, stream, objs, host, opts, steps, barrier):
    """The batched step through the public API with host buffers: every step
    copies all 32 objects' rays, targets, uniforms and colours from pinned host
    memory (one block, one copy; on a copy stream, double-buffered, so the copy
    of step i+1 overlaps step i) and reads the 32 losses back into pinned memory
    (double-buffered on the device, on a stream of its own)."""
    import torch

    packed = [_pack([h["sets"][j] for h in host]) for j in range(4)]
    layout = packed[0][1]
    blocks = [p[0] for p in packed]
    h2d = blocks[0].numel()
    n = len(objs)
    staging = [torch.empty_like(blocks[0], device="cuda") for _ in range(2)]
    views = [[dict(_unpack(buf, ent), obj=o) for ent, o in zip(layout, objs)] for buf in staging]
    losses = [torch.zeros(n, device="cuda") for _ in range(2)]
    loss_host = torch.zeros((steps, n)).pin_memory()
    copy_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    stepped = [torch.cuda.Event() for _ in range(2)]
    read = [torch.cuda.Event() for _ in range(2)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        slot = i % 2
        if i >= 2:
            copy_stream.wait_event(stepped[slot])  # the step that read this input buffer is done
        with torch.cuda.stream(copy_stream):
            staging[slot].copy_(blocks[i % len(blocks)], non_blocking=True)
            copied[slot].record(copy_stream)
        stream.wait_event(copied[slot])
        if i >= 2:
            stream.wait_event(read[slot])  # this loss buffer's previous values have been read back
        ctx.train_step(views[slot], opts, losses[slot])
        stepped[slot].record(stream)
        d2h_stream.wait_event(stepped[slot])
        with torch.cuda.stream(d2h_stream):
            loss_host[i].copy_(losses[slot], non_blocking=True)
            read[slot].record(d2h_stream)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    assert np.all(np.isfinite(loss_host.numpy()))
    return secs, int(h2d), 4 * n


def _held_out(host, seed=99):
    """4 held-out 480x640 views per object, 4096 rays each object (o, d; targets)."""
    from synth import cameras_on_sphere, make_ray_pool

    out = []
    for h in host:
        p = make_ray_pool(h["scene"], cameras_on_sphere(4, 2.0, 50, 480, 640, seed + h["index"]), 4096,
                          seed + h["index"])
        out.append(p)
    return out


def _errors(ctx, objs, held, opts):
    """Mean over the objects of the held-out colour MSE (all rays, black behind
    the object) and depth L1 (object rays)."""
    import torch

    mse, l1 = [], []
    for o, p in zip(objs, held):
        r = ctx.render({"o": torch.from_numpy(p.o).cuda(), "d": torch.from_numpy(p.d).cuda(), "obj": o}, opts)
        rgb, depth = r["rgb"].cpu().numpy(), r["depth"].cpu().numpy()
        tgt = np.where(p.is_obj[:, None] == 1, p.rgb, 0.0)
        m = p.is_obj == 1
        mse.append(float(np.mean((rgb - tgt) ** 2)))
        l1.append(float(np.mean(np.abs(depth - p.depth)[m])) if m.any() else 0.0)
    return float(np.mean(mse)), float(np.mean(l1))


def _equal_error(pkg, ctx, stream, prec, steps=300, seeds=(0, 1, 2)):
    """The metric's condition on the headline workload: the 32 objects trained
    for `steps` Adam steps in the batched mixed-precision form and, from the same
    initial parameters and on the same rays, one plain FP32 step at a time; then
    held-out colour MSE and depth L1 (mean over the objects) for each seed.  Each
    step draws every object's rays from a pool of 16x its ray count (on the
    device, seeded) with the library's own Philox uniforms and background
    colours.  The mixed-precision form passes when its seed mean is within
    max(5 %, 2 x the FP32 seed-to-seed std) of the FP32 mean on both errors."""
    import torch
    from synth import init_params

    host = batched_host(pool_factor=16)
    held = _held_out(host)
    pools = [{k: torch.from_numpy(np.ascontiguousarray(getattr(h["pool"], k))).cuda()
              for k in ("o", "d", "rgb", "depth", "is_obj")} for h in host]
    opts = pkg.make_opts(nc=BATCHED_NR, nr=BATCHED_NR, lr=1e-2)
    runs = {prec: [], "fp32": []}
    for seed in seeds:
        thetas = []
        for h in host:
            a = batched_arch_dict(h["spec"])
            n = pkg.arch_param_count(pkg.make_arch(**a))
            nmlp = mlp_macs(a["width"], a["hidden"])
            shapes = [(a["width"], 32)] + [(a["width"], a["width"])] * (a["hidden"] - 1) + [(4, a["width"])]
            thetas.append(init_params(n - nmlp, shapes, 100 * seed + h["index"]))
        for form in (prec, "fp32"):
            objs, _ = _batched_objects(pkg, ctx, stream, form, host, thetas)
            g = torch.Generator(device="cuda")
            g.manual_seed(1000 + seed)
            loss = torch.zeros(len(objs), device="cuda")
            for i in range(steps):
                bs = []
                for h, o, pl in zip(host, objs, pools):
                    idx = torch.randint(0, pl["o"].shape[0], (h["spec"]["rays"],), device="cuda", generator=g)
                    bs.append({k: v[idx] for k, v in pl.items()} | {"obj": o})
                if form == "fp32":  # plain FP32, one object at a time
                    for j, b in enumerate(bs):
                        ctx.train_step([b], opts, loss[j:j + 1])
                else:
                    ctx.train_step(bs, opts, loss)
            runs[form].append(_errors(ctx, objs, held, opts) + (float(loss.mean().item()),))
            for o in objs:
                ctx.destroy_object(o)
    out = {}
    for form, rs in runs.items():
        a = np.array(rs)
        out[form] = {"colour_mse": float(a[:, 0].mean()), "colour_mse_std": float(a[:, 0].std(ddof=1)),
                     "depth_l1": float(a[:, 1].mean()), "depth_l1_std": float(a[:, 1].std(ddof=1)),
                     "final_loss": float(a[:, 2].mean()), "per_seed": [[round(x, 6) for x in r] for r in rs]}
    ok = True
    tol = {}
    for key in ("colour_mse", "depth_l1"):
        t = max(0.05 * out["fp32"][key], 2.0 * out["fp32"][key + "_std"])
        d = out[prec][key] - out["fp32"][key]
        tol[key] = {"tolerance": t, "difference": d, "within": abs(d) <= t}
        ok = ok and abs(d) <= t
    out["tolerance"] = tol
    out["pass"] = bool(ok)
    out["workload"] = (f"the headline's 32 objects, {steps} Adam steps each, batched {prec} vs one FP32 step per "
                       f"object at a time, same initial parameters; held-out: 4 views of 480x640 per object, 4096 "
                       f"rays; {len(seeds)} seeds")
    return out


def _single_compare(pkg, ctx, stream, prec, rank, steps, warmup):
    """The single full-size object (4096 rays x 64 samples) in the mixed-precision
    form and in plain FP32, one object per step."""
    import torch
    from synth import (cameras_on_sphere, init_params, make_ray_pool, prior_grid, random_colours, sample_batch,
                       scene_random_csg, stratified_uniforms)

    sc = scene_random_csg(rank)
    pool = make_ray_pool(sc, cameras_on_sphere(24, 2.0, 50, 480, 640, rank), 65536, rank, depth_noise=0.004)
    grid = prior_grid(sc, GRID_RES, rank)
    batches_np = []
    for i in range(8):
        b = sample_batch(pool, N_RAYS, 1000 * rank + i)
        b["uniforms"] = stratified_uniforms(N_RAYS, NR, 2000 * rank + i)
        b["c_rand"] = random_colours(N_RAYS, 3000 * rank + i)
        batches_np.append(b)
    opts = pkg.make_opts(nc=NC, nr=NR, lr=1e-2)
    loss = torch.zeros(1, device="cuda")
    out = {"workload": SINGLE_WORKLOAD}
    theta = None
    for form in (prec, "fp32"):
        arch = pkg.make_arch(**ARCH, precision=PRECISION[form])
        if theta is None:
            n = pkg.arch_param_count(arch)
            theta = init_params(n - mlp_macs(64, 2), [(64, 32), (64, 64), (4, 64)], rank + 1)
        obj = ctx.create_object(arch, theta)
        ctx.set_prior_grid(obj, grid)
        dev = _device_batches(batches_np, obj, stream)
        ctx.autotune([dev[0]], opts)
        f = lambda i: ctx.train_step([dev[i % len(dev)]], opts, loss)  # noqa: E731
        ms0 = _time(stream, f, steps, warmup)  # from initialisation
        _time(stream, f, 0, max(3, TRAIN_AGE - warmup - steps))
        ctx.autotune([dev[0]], pkg.make_opts(nc=NC, nr=NR, lr=1e-2, flags=pkg.PRENOM_FLAG_RETUNE))
        ms = _time(stream, f, steps, 3)
        out[form] = {"value": N_RAYS * NR * steps / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms / steps,
                     "from_init": {"value": N_RAYS * NR * steps / (ms0 / 1e3), "ms_per_step": ms0 / steps}}
        ctx.enable_timing(True)  # per-kernel device times of the same steps, launched directly
        _time(stream, f, max(steps // 4, 5), 0)
        out[form]["kernels_us"] = {lab.split()[6] + " " + pkg.KERNEL_NAMES[k]: round(1e3 * t_ms / n, 2)
                                   for lab, k, t_ms, n in ctx.timing_report()}
        ad = ctx.kernel_time(pkg.PRENOM_KERNEL_ADAM)
        out[form]["kernels_us"]["adam"] = round(1e3 * ad[0] / max(ad[1], 1), 2)
        ctx.enable_timing(False)
        ctx.destroy_object(obj)
    out["speedup"] = out[prec]["value"] / out["fp32"]["value"]
    return out


STRESS_OBJECTS, STRESS_RAYS, STRESS_NR = 64, 1 << 20, 64


def _stress_compare(pkg, ctx, stream, steps=200, warmup=20):
    """Real-time mapping stress: 64 objects of the category table in BF16 (MLP
    on the tensor cores; BF16 hash features, i.e. the gathers read a BF16 copy
    of the FP32 master tables), 2^20 rays per step in total split by a
    projected-area share 2^(5a), a ~ U[0,1), 64 samples per ray from each
    object's 64^3 prior, rays from 480x640 views, the internal Philox uniforms
    and background colours; the whole step (all objects, backward, Adam) is one
    batched call, autotuned and graph-captured before the warm-up, and each
    step's latency is timed with its own CUDA events.  The same workload with
    the gathers on the FP32 tables is reported beside it."""
    import torch
    from synth import cameras_on_sphere, make_ray_pool, prior_grid, sample_batch, scene_random_csg

    rng = np.random.default_rng(17)
    w = 2.0 ** (5 * rng.random(STRESS_OBJECTS))
    rays = [max(32, 32 * int(round(STRESS_RAYS * x / w.sum() / 32))) for x in w]
    n_smp = sum(rays) * STRESS_NR
    opts = pkg.make_opts(nc=STRESS_NR, nr=STRESS_NR, lr=1e-2)
    loss = torch.zeros(STRESS_OBJECTS, device="cuda")
    out = {}
    for features in (pkg.PRENOM_FEATURES_BF16, pkg.PRENOM_FEATURES_FP32):
        objs, sets = [], [[], []]
        for i in range(STRESS_OBJECTS):
            log2T, W, H = CATEGORY_ARCHS[i % len(CATEGORY_ARCHS)]
            arch = pkg.make_arch(L=16, log2T=log2T, n_min=16, n_max=2048, width=W, hidden=H, lambda_d=0.1,
                                 lambda_sigma=1e-3, precision=PRECISION["bf16"], features=features)
            sc = scene_random_csg(5000 + i)
            obj = ctx.create_object(arch)
            ctx.set_prior_grid(obj, prior_grid(sc, GRID_RES, i))
            pool = make_ray_pool(sc, cameras_on_sphere(8, 2.0, 50, 480, 640, 100 + i), 2 * rays[i], 100 + i,
                                 depth_noise=0.004)
            for j in range(2):
                sets[j].append(_device_batches([sample_batch(pool, rays[i], 50 * i + j)], obj, stream)[0])
            objs.append(obj)
        ctx.autotune(sets[0], opts)
        for i in range(warmup):
            ctx.train_step(sets[i % 2], opts, loss)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            ev[i][0].record(stream)
            ctx.train_step(sets[i % 2], opts, loss)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        for o in objs:
            ctx.destroy_object(o)
        out[features] = {"value": n_smp / (float(np.mean(ms)) / 1e3), "unit": "samples/s",
                         "latency_ms_p50": float(np.percentile(ms, 50)),
                         "latency_ms_p99": float(np.percentile(ms, 99))}
    res = {"workload": "64 objects of the category table, BF16 MLP and BF16 hash features (FP32 master tables), "
                       "%d rays x 64 samples per step (%d samples), 64^3 priors, one batched step" % (sum(rays), n_smp)}
    res.update(out[pkg.PRENOM_FEATURES_BF16])
    res.update(steps=steps, warmup=warmup, fp32_features=out[pkg.PRENOM_FEATURES_FP32])
    return res


META_TASKS, META_INNER, META_RAYS, META_NR = 16, 16, 2048, 48


def _meta_compare(pkg, ctx, stream, prec):
    """One Reptile meta step (§III-A): 16 tasks of one CSG topology with per-task
    scale jitter U[0.8, 1.2], each adapted by 16 inner Adam steps of 2048 rays x 48
    samples (all tasks of an inner step in one batched call), then the outer update
    of Eq. 2 (beta = 0.1); architecture L=8, F=2, T=2^14, res 16..256, MLP 16-32-32-4."""
    import torch
    from paper_2503_01582_gb300.meta import meta_step
    from synth import (cameras_on_sphere, make_ray_pool, prior_grid, random_colours, sample_batch,
                       scene_random_csg, stratified_uniforms)

    arch = pkg.make_arch(L=8, log2T=14, n_min=16, n_max=256, width=32, hidden=2, lambda_d=0.1, lambda_sigma=1e-3,
                         precision=PRECISION[prec])
    rng = np.random.default_rng(11)
    meta = ctx.create_object(arch)
    tasks, batches = [], []
    for t in range(META_TASKS):
        sc = scene_random_csg(21, scale=float(rng.uniform(0.8, 1.2)))
        obj = ctx.create_object(arch)
        ctx.set_prior_grid(obj, prior_grid(sc, 32, t))
        pool = make_ray_pool(sc, cameras_on_sphere(8, 2.0, 40, 128, 128, t), 4 * META_RAYS, t)
        bs = []
        for j in range(4):  # four rotating ray sets per task
            b = sample_batch(pool, META_RAYS, 1000 * t + j)
            b["uniforms"] = stratified_uniforms(META_RAYS, META_NR, 2000 * t + j)
            b["c_rand"] = random_colours(META_RAYS, 3000 * t + j)
            bs.append(_device_batches([b], obj, stream)[0])
        tasks.append(obj)
        batches.append(bs)
    inner = [[batches[t][j % 4] for t in range(META_TASKS)] for j in range(META_INNER)]
    opts = pkg.make_opts(nc=META_NR, nr=META_NR, lr=1e-2)
    loss = torch.zeros(META_TASKS, device="cuda")
    f = lambda i: meta_step(ctx, meta, tasks, inner, opts, 0.1, loss)  # noqa: E731
    steps = 3
    ms = _time(stream, f, steps, 2)
    for o in [meta] + tasks:
        ctx.destroy_object(o)
    n_smp = META_TASKS * META_INNER * META_RAYS * META_NR
    return {"workload": "Reptile meta step: 16 tasks x 16 inner Adam steps x 2048 rays x 48 samples, outer update "
                        "(Eq. 2, beta 0.1); L=8 T=2^14 res 16..256, MLP 16-32-32-4; %d samples per meta step" % n_smp,
            "value": n_smp * steps / (ms / 1e3), "unit": "samples/s", "ms_per_meta_step": ms / steps}


def _ablation_compare(pkg, ctx, stream, prec, steps=300, seeds=(0, 1, 2)):
    """Sampling ablation (the analogue of the paper's Table IV row on
    probabilistic sampling): the small scene (sphere + box, 8 views of 64x64)
    trained for `steps` Adam steps of 256 rays x 32 samples with prior sampling
    over the 32^3 prior grid (as given, refreshed from the field every 50
    steps as §III-B does, and a softer prior of peak density 8 whose dilated
    shell is not opaque) and with uniform sampling (a zero grid: every ray
    escapes, so the flat CDF of the escape rule applies), on the same rays; then
    colour MSE (all pixels, black background) and depth L1 (object pixels) on 4
    held-out 64x64 views, sampled the way each was trained.  Each seed draws its
    own initial parameters and ray batches; mean and standard deviation over the
    seeds are reported (a single run moves by tens of percent with the rounding
    of a kernel change)."""
    import torch
    from synth import (cameras_on_sphere, init_params, make_ray_pool, prior_grid, sample_batch, scene_sphere_box)

    sc = scene_sphere_box()
    pool = make_ray_pool(sc, cameras_on_sphere(8, 2.0, 40, 64, 64, 0), 65536, 0)
    held = make_ray_pool(sc, cameras_on_sphere(4, 2.0, 40, 64, 64, 99), 4096, 99)
    hb = {k: torch.from_numpy(np.ascontiguousarray(getattr(held, k))).cuda() for k in ("o", "d")}
    tgt = np.where(held.is_obj[:, None] == 1, held.rgb, 0.0)
    objm = held.is_obj == 1
    arch = pkg.make_arch(L=8, log2T=14, n_min=16, n_max=256, width=32, hidden=2, lambda_d=0.1, lambda_sigma=0.0,
                         precision=PRECISION[prec])
    probe = ctx.create_object(arch)
    n = ctx.param_count(probe)
    ctx.destroy_object(probe)
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2)
    loss = torch.zeros(1, device="cuda")
    prior = prior_grid(sc, 32, 0)
    # a second synthetic prior whose dilated shell is not opaque: peak density 8, so a
    # ray crossing the 2-voxel shell (2/32 of the cube) sees an optical depth of 0.5
    soft = prior_grid(sc, 32, 0, peak=8.0)
    variants = (("prior_sampling", prior, 0), ("prior_sampling_refresh_every_50", prior, 50),
                ("prior_sampling_soft_prior", soft, 0), ("uniform_sampling", np.zeros((32, 32, 32), np.float32), 0))
    runs = {name: [] for name, _, _ in variants}
    for seed in seeds:
        theta = init_params(n - (32 * 16 + 32 * 32 + 4 * 32), [(32, 16), (32, 32), (4, 32)], 5 + seed)
        theta = theta.astype(np.float32)
        batches = [_device_batches([sample_batch(pool, 256, 7000 + 1000 * seed + i)], 0, stream)[0]
                   for i in range(steps)]
        for name, grid, refresh in variants:
            obj = ctx.create_object(arch, theta)
            ctx.set_prior_grid(obj, grid)
            for b in batches:
                b["obj"] = obj

            def step(i, obj=obj, refresh=refresh):
                if refresh and i > 0 and i % refresh == 0:  # §III-B: the prior follows the field every m iterations
                    ctx.refresh_prior(obj, 32)
                ctx.train_step([batches[i]], opts, loss)

            ms = _time(stream, step, steps, 0)
            r = ctx.render(dict(hb, obj=obj), opts)
            rgb, depth = r["rgb"].cpu().numpy(), r["depth"].cpu().numpy()
            runs[name].append((float(np.mean((rgb - tgt) ** 2)), float(np.mean(np.abs(depth - held.depth)[objm])),
                               float(loss.item()), ms / steps))
            ctx.destroy_object(obj)
    out = {}
    for name, rs in runs.items():
        a = np.array(rs)
        out[name] = {"colour_mse": float(a[:, 0].mean()), "colour_mse_std": float(a[:, 0].std(ddof=1)),
                     "depth_l1": float(a[:, 1].mean()), "depth_l1_std": float(a[:, 1].std(ddof=1)),
                     "final_loss": float(a[:, 2].mean()), "ms_per_step": float(a[:, 3].mean())}
    out["workload"] = ("sphere+box scene, %d Adam steps x 256 rays x 32 samples (Nc 32), L=8 T=2^14 res 16..256, "
                       "MLP 16-32-32-4, same rays for every variant; 4 held-out 64x64 views; mean and std over "
                       "%d seeds" % (steps, len(seeds)))
    return out


def _roofline(pkg, report, specs, prec, adam_ms, n_params, peaks):
    """Each kernel of one batched step against its own bound, from the per-group
    timing report.  A group is every object of one MLP width; all objects have
    L=16, F=2, so a sample moves 8 L F x 4 B = 1024 B of table gathers (the
    encoder) or of FP32 reductions (the scatter), and its MLP work is 6 MAC FLOP
    (2 forward, 4 backward).  Records are per kernel: its launches over the
    groups (one per group per step) summed, achieved = the summed algorithmic
    work / the summed device time, with the per-group figures beside it.  The
    kernel with the largest device time per step is the dominant one."""
    names = {pkg.PRENOM_KERNEL_SAMPLE_ENCODE: "sample_encode_kernel", pkg.PRENOM_KERNEL_SCATTER: "hash_scatter_kernel"}
    kernels = {}
    for label, k, ms, n in report:
        tok = label.split()
        W, form = int(tok[1][1:]), tok[6]
        members = [sp for sp in specs if sp["W"] == W]
        samples = sum(sp["rays"] * BATCHED_NR for sp in members)
        flops = sum(sp["rays"] * BATCHED_NR * 6 * mlp_macs(sp["W"], sp["H"]) for sp in members)
        t = (ms / n) / 1e3
        if k == pkg.PRENOM_KERNEL_TRAIN and form.startswith("split"):
            tc = prec != "fp32"
            name = "fused_tc_kernel_split" if tc else "fused_fp32_kernel_split"
            unit, work, what = "TFLOP/s", flops, "6 x MAC FLOP/sample"
            base = {"bound": "tensor" if tc else "alu", "peak": round(peaks["bf16"] if tc else FP32_PEAK_TFLOPS, 1),
                    "peak_src": (peaks["src"] + " bf16 (fp16 same rate)") if tc else "FP32 FFMA 152x128x2x2070 MHz"}
        else:
            per = 2048 if k == pkg.PRENOM_KERNEL_TRAIN else 1024
            name = names.get(k, "fused_tc_kernel" if prec != "fp32" else "fused_fp32_kernel")
            unit, work, what = "GB/s", samples * per, f"{per} B/sample"
            base = {"bound": "hbm", "peak": peaks["hbm_gbs"], "peak_src": peaks["src"] + " copy bandwidth"}
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        rec = kernels.setdefault(name, dict(kernel=name, unit=unit, work=0.0, t=0.0, groups=[], what=what, **base))
        rec["work"] += work
        rec["t"] += t
        grp = {"group": label, "avg_us": round(t * 1e6, 2), "achieved": round(work / t / scale, 2),
               "frac": round(work / t / scale / rec["peak"], 4), "traffic": profiled_traffic(f"{name}/{prec}/W{W}")}
        if name in ("sample_encode_kernel", "hash_scatter_kernel"):  # bound by L1/L2 requests, not DRAM bytes
            grp["l2"] = profiled_l2(f"{name}/{prec}/W{W}", samples)
        rec["groups"].append(grp)
    kernels["adam_kernel"] = dict(kernel="adam_kernel", unit="GB/s", work=n_params * 28.0, t=adam_ms / 1e3, groups=[],
                                  what="28 B/parameter (read g, m, v, theta; write m, v, theta)", bound="hbm",
                                  peak=peaks["hbm_gbs"], peak_src=peaks["src"] + " copy bandwidth")
    recs = []
    for rec in kernels.values():
        scale = 1e12 if rec["unit"] == "TFLOP/s" else 1e9
        ach = rec["work"] / rec["t"] / scale
        out = {"kernel": rec["kernel"], "bound": rec["bound"], "achieved": round(ach, 2), "peak": rec["peak"],
               "unit": rec["unit"], "frac": round(ach / rec["peak"], 4),
               "algorithmic": f"{rec['what']}: {rec['work'] / (1e9 if rec['unit'] == 'TFLOP/s' else 1e6):.1f} "
                              f"{'GFLOP' if rec['unit'] == 'TFLOP/s' else 'MB'} per step over "
                              f"{max(len(rec['groups']), 1)} launch(es)",
               "avg_us_per_step": round(rec["t"] * 1e6, 2), "launches_per_step": max(len(rec["groups"]), 1),
               "peak_src": rec["peak_src"],
               "traffic": (profiled_traffic(f"adam_kernel/{prec}/batched") if rec["kernel"] == "adam_kernel"
                           else (sum(g["traffic"] for g in rec["groups"])
                                 if all(g["traffic"] is not None for g in rec["groups"]) else None))}
        if rec["groups"]:
            out["groups"] = rec["groups"]
        recs.append(out)
    dom = max(recs, key=lambda r: r["avg_us_per_step"])
    roof = dict(dom)
    roof["other_kernels"] = [r for r in recs if r is not dom]
    roof["step_kernels_us"] = round(sum(r["avg_us_per_step"] for r in recs), 2)
    return roof


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2503_01582_gb300 as pkg
    from paper_2503_01582_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    pkg._abi.lib()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stream = torch.cuda.Stream()
    # every torch op of the bench runs on the library's stream: inputs made here
    # are ordered before the steps that read them, and freed only after them
    torch.cuda.set_stream(stream)
    ctx = pkg.Context(seed=rank, stream=stream)
    prec = args.precision
    if args.workload == "single":  # the single full-size object alone (for profiling it), one JSON line
        if world == 1:
            out = _single_compare(pkg, ctx, stream, prec, rank, args.steps, args.warmup)
            print(json.dumps({"impl": "ours", "workload": "single", **out}), flush=True)
        ctx.close()
        return
    form_flags = {"auto": 0, "fused": pkg.PRENOM_FLAG_FUSED, "split": pkg.PRENOM_FLAG_SPLIT}[args.form]
    bopts = pkg.make_opts(nc=BATCHED_NR, nr=BATCHED_NR, lr=1e-2, flags=form_flags)
    specs = batched_specs()
    n_smp, n_rays = batched_totals(specs)

    # ---- headline: the 32 objects in one batched step, inputs resident in HBM.
    # The autotuner's calls and the graph captures run here, in set-up.
    host = batched_host()
    objs, sets = _batched_objects(pkg, ctx, stream, prec, host)
    n_params = sum(ctx.param_count(o) for o in objs)
    lossb = torch.zeros(len(objs), device="cuda")
    ctx.autotune(sets[0], bopts)
    step = lambda i: ctx.train_step(sets[i % 4], bopts, lossb)  # noqa: E731
    # the objects' first steps: W warm-up steps, then K timed
    ms_init = _time(stream, step, args.steps, args.warmup, barrier)
    if world > 1:
        t = torch.tensor([ms_init], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_init = t.item()
    # untimed training up to TRAIN_AGE steps per object (at least 3 more warm-up steps),
    # then the autotuner again on the trained objects (set-up: its calls leave them as
    # they were) and 3 warm-up steps on the graphs it captured
    age = args.warmup + args.steps + max(3, TRAIN_AGE - args.warmup - args.steps)
    _time(stream, step, 0, age - args.warmup - args.steps)
    ctx.autotune(sets[0], pkg.make_opts(nc=BATCHED_NR, nr=BATCHED_NR, lr=1e-2,
                                        flags=form_flags | pkg.PRENOM_FLAG_RETUNE))
    _time(stream, step, 0, 3)
    age += 3
    tuning = ctx.tuning_report().strip()
    cap0 = ctx.capture_count()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(gpu_identifier(local))
    with clocks:  # the step as a user runs it: CUDA-graph replay, no per-kernel events
        ms = _time(stream, step, args.steps, 0, barrier, clocks)
    launches = ctx.launch_count() - launches0
    assert ctx.capture_count() == cap0, "the timed region ran autotuner calls or graph captures"
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = t.item()
    value = n_smp * args.steps * world / (ms / 1e3)

    # per-kernel device times: the same steps launched directly, each kernel between CUDA events
    ctx.enable_timing(True)
    nk = max(args.steps // 4, 5)
    _time(stream, step, nk, 0)
    report = ctx.timing_report()
    adam_ms = ctx.kernel_time(pkg.PRENOM_KERNEL_ADAM)
    ctx.enable_timing(False)
    groups = [{"group": lab, "kernel": pkg.KERNEL_NAMES[k], "avg_us": round(1e3 * t_ms / n, 2)}
              for lab, k, t_ms, n in report]
    roofline = _roofline(pkg, report, specs, prec, adam_ms[0] / max(adam_ms[1], 1), n_params, load_peaks())

    # ---- end to end through the public API with host buffers
    e2e_s, h2d, d2h = _e2e(ctx, stream, objs, host, bopts, args.steps, barrier)
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = t.item()
    e2e_value = n_smp * args.steps * world / e2e_s

    # ---- the plain FP32 side of the pair: the same 32 objects from the same
    # parameters, one FP32 step per object at a time (each object autotuned first)
    thetas = [ctx.get_state(o).cpu().numpy() for o in objs]
    for o in objs:
        ctx.destroy_object(o)
    objs32, sets32 = _batched_objects(pkg, ctx, stream, "fp32", host, thetas)
    opts32 = pkg.make_opts(nc=BATCHED_NR, nr=BATCHED_NR, lr=1e-2)
    for b in sets32[0]:
        ctx.autotune([b], opts32)
    fl = lambda i: [ctx.train_step([b], opts32, lossb[j:j + 1]) for j, b in enumerate(sets32[i % 4])]  # noqa
    ms32 = _time(stream, fl, args.steps, args.warmup, barrier)
    if world > 1:
        t = torch.tensor([ms32], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms32 = t.item()
    fp32_loop = {"value": n_smp * args.steps * world / (ms32 / 1e3), "unit": "samples/s",
                 "ms_per_step": ms32 / args.steps,
                 "form": "32 single-object plain FP32 steps (each its own launch set, CUDA-graph replay), from the "
                         "headline objects' parameters after its timed steps"}
    for o in objs32:
        ctx.destroy_object(o)

    equal = None
    if world == 1 and not args.no_equal_error and prec != "fp32":
        equal = _equal_error(pkg, ctx, stream, prec, steps=args.equal_error_steps)

    compare = {}
    if world == 1 and not args.no_compare and prec != "fp32":
        # the same batched step with the gathers on BF16 copies of the tables
        objs_b, sets_b = _batched_objects(pkg, ctx, stream, prec, host, thetas, features=pkg.PRENOM_FEATURES_BF16)
        ctx.autotune(sets_b[0], bopts)
        fb = lambda i: ctx.train_step(sets_b[i % 4], bopts, lossb)  # noqa: E731
        msb = _time(stream, fb, args.steps, args.warmup)
        compare["batched_bf16_features"] = {"value": n_smp * args.steps / (msb / 1e3), "unit": "samples/s",
                                            "ms_per_step": msb / args.steps,
                                            "form": "the headline step with BF16 copies of the hash tables "
                                                    "serving the gathers (FP32 master tables)"}
        for o in objs_b:
            ctx.destroy_object(o)
    if world == 1 and not args.no_compare:
        compare["single_object_full_size"] = _single_compare(pkg, ctx, stream, prec, rank, max(args.steps, 20),
                                                             args.warmup)
        compare["reptile_meta_step"] = _meta_compare(pkg, ctx, stream, prec)
        compare["sampling_ablation"] = _ablation_compare(pkg, ctx, stream, prec)
        compare["mapping_stress_64_objects"] = _stress_compare(pkg, ctx, stream)

    if world > 1 and not args.no_compare:
        # the 32-object workload split over the ranks (longest processing time
        # first on the per-object cost), one batched step per rank, no exchange
        from paper_2503_01582_gb300.shard import object_cost, rank_objects

        costs = [object_cost(16, 2, sp["W"], sp["H"], pkg.arch_param_count(pkg.make_arch(**batched_arch_dict(sp))),
                             sp["rays"] * BATCHED_NR, 4 if prec == "fp32" else 2) for sp in specs]
        mine = rank_objects(costs, world, rank)
        hs = [h for h in host if h["index"] in set(mine)]
        objs_r, sets_r = _batched_objects(pkg, ctx, stream, prec, hs)
        lossr = torch.zeros(max(len(objs_r), 1), device="cuda")
        if objs_r:
            ctx.autotune(sets_r[0], bopts)
        fb = lambda i: ctx.train_step(sets_r[i % 4], bopts, lossr) if objs_r else None  # noqa: E731
        msb = _time(stream, fb, args.steps, args.warmup, barrier)
        t = torch.tensor([msb], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        compare["batched_32_objects_sharded"] = {
            "workload": "the 32-object batched workload split over %d GPUs by longest-processing-time "
                        "first; %d samples per step in total" % (world, n_smp),
            "value": n_smp * args.steps / (t.item() / 1e3), "unit": "samples/s",
            "ms_per_step": t.item() / args.steps, "scaling": "strong"}
        for o in objs_r:
            ctx.destroy_object(o)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            budget = float(os.environ.get("PRENOM_ORACLE_BUDGET_S", "12"))
            adam_s = oracle_adam_seconds_per_param() * oracle_param_total()
            try:  # in a spawned process of its own: no CUDA context or bench threads beside it
                r1 = oracle_timing(budget, 1)
                where = "one spawned host process"
            except Exception:
                r1 = {o[0]: _oracle_rays(o, budget / BATCHED_OBJECTS) for o in _oracle_objects()}
                where = "the bench process (the spawned process failed)"
            s1 = oracle_step_seconds(r1, 1, adam_s)
            cpu = {"value": n_smp / s1, "unit": "samples/s", "cores": 1, "kind": "oracle",
                   "sample": (f"{sum(d for d, _ in r1.values())} of the step's {n_rays} rays fwd+bwd (each of the "
                              f"32 objects for {budget / BATCHED_OBJECTS:.2f} s) in {where} + one full Adam pass "
                              f"over {oracle_param_total()} parameters ({adam_s:.2f} s, timed on 12.2 M), FP64, "
                              f"extrapolated to the whole step")}
            ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
            if ncores > 1:  # the same oracle on every host core, one process per core
                try:
                    ra = oracle_timing(float(os.environ.get("PRENOM_ORACLE_ALL_CORES_S", "6")), ncores)
                    sa = oracle_step_seconds(ra, ncores, adam_s)
                    cpu["all_cores"] = {"value": n_smp / sa, "unit": "samples/s", "cores": ncores,
                                        "sample": (f"{sum(d for d, _ in ra.values())} rays fwd+bwd over {ncores} "
                                                   f"processes (objects dealt round-robin, spread evenly in the "
                                                   f"extrapolation) + the one-thread Adam pass")}
                except Exception as e:  # the headline line is printed whatever happens here
                    cpu["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
        line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
                "config": {"workload": WORKLOAD,
                           "form": "batched " + FORM[prec] + {"auto": ", fused or split form per group as "
                                                                      "autotuned",
                                                              "fused": ", one fused kernel per group",
                                                              "split": ", split form per group"}[args.form],
                           "objects": BATCHED_OBJECTS, "rays_per_step": n_rays, "samples_per_ray": BATCHED_NR,
                           "samples_per_step": n_smp, "params": n_params, "autotuner": tuning,
                           "groups": groups,
                           "timed_region": "autotuner calls and graph captures ran in set-up (prenom_autotune, "
                                           "at the objects' first step and again after TRAIN_AGE steps); none "
                                           "inside the timed steps (checked by the library's counters)",
                           "training_steps_before_timing": age,
                           "parallelism": (f"{world} ranks, each its own copy of the 32 objects" if world > 1
                                           else "1 GPU, 32 objects"),
                           "l2": "working set > L2: theta, grad, Adam m and v of all objects (4 x %.0f MB) stream "
                                 "every step" % (n_params * 4 / 1e6)},
                "from_init": {"value": n_smp * args.steps * world / (ms_init / 1e3), "unit": "samples/s",
                              "ms_per_step": ms_init / args.steps,
                              "steps": f"the objects' training steps {args.warmup}..{args.warmup + args.steps - 1}"},
                "fp32_per_object_loop": fp32_loop, "speedup_vs_fp32_loop": value / fp32_loop["value"],
                "equal_error": equal,
                "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
                "clocks": clocks.summary(), "compare": compare}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the single-object, Reptile, ablation and "
                                                              "stress comparison runs")
    ap.add_argument("--no-equal-error", action="store_true", help="skip the equal-error training runs")
    ap.add_argument("--equal-error-steps", type=int, default=300)
    ap.add_argument("--precision", default="fp16", choices=list(PRECISION))
    ap.add_argument("--form", default="auto", choices=["auto", "fused", "split"],
                    help="the autotuner's choice per group, the fused kernel, or the three-kernel split form")
    ap.add_argument("--workload", default="batched", choices=["batched", "single"],
                    help="batched: the 32-object headline with its comparisons; single: only the single "
                         "full-size object (FP16 and FP32), for profiling its kernels")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
