"""Benchmark: protect + restore of one 4096 x 4096 RGB uint8 image per GPU, k = 5.

One step = the whole hot path on one image: the fused protect kernel (8x8 DCT-II, exact int16
rounding, zigzag split, AES-128-CTR of the confidential fragment) followed by the fused
restore kernel (CTR decryption, merge, inverse DCT, exact rounding, clamp).  The metric is MB/s
of input pixels (W * H * 3 bytes per step / step time, 10^6 bytes per MB); ranks run
independent images (weak scaling, no collective on the data path).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead, on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WIDTH = HEIGHT = 4096
E2E_STRIPS = 1          # strips of the host-buffer pipeline (1 measured fastest of 1..8 with three lanes)
E2E_LANES = 3           # steps in flight in the end-to-end measurement, one stream each
K_SEL = 5
IMG_SEED, KEY_SEED, IV_SEED = 2, 2005, 3005
METRIC = "protect+restore MB/s of pixels"
UNIT = "MB/s"
WORKLOAD = f"{WIDTH}x{HEIGHT} RGB uint8, protect+restore, k={K_SEL}"
FALLBACK_HBM_GBS = 6800.0


def _config():
    return {"workload": WORKLOAD, "width": WIDTH, "height": HEIGHT, "k": K_SEL,
            "channels": 3, "generator": "20 random 2-D Gaussians + U[-8,8] noise, seed 2",
            "l2": "inputs larger than L2: two fragment buffer sets alternate, so restore reads "
                  "fragments written one step earlier (>= 250 MB of traffic since)"}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
def _oracle_child(args):
    """Runs in a child process with one BLAS/OpenMP thread: oracle protect + restore on
    strips of the workload image until `args.budget` seconds are used."""
    import numpy as np

    from oracle import aes as oaes, dct as odct, fds as ofds
    from paper_1512_02951_gb300 import synth

    img = synth.make_image(WIDTH, HEIGHT, IMG_SEED)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    rows = args.rows
    bx = WIDTH // 8
    done_bytes, t_used, times = 0, 0.0, []
    r0 = args.start_row
    while r0 < HEIGHT // 8 and (t_used < args.budget or not times) and len(times) < args.max_steps:
        r1 = min(HEIGHT // 8, r0 + rows)
        strip = img[8 * r0: 8 * r1]
        t = time.perf_counter()
        q, _ = ofds.quantised_dct(odct.image_to_blocks(strip))
        part1, part2 = ofds.split(q.astype(np.int16), K_SEL)
        off = r0 * bx * 3 * 2 * (K_SEL + 1)
        ct = oaes.ctr_xcrypt(key, iv, np.ascontiguousarray(part1).astype("<i2").tobytes(), offset=off)
        plain = oaes.ctr_xcrypt(key, iv, ct, offset=off)
        p1 = np.frombuffer(plain, dtype="<i2").astype(np.int64).reshape(part1.shape)
        p = ofds.quantised_idct(ofds.merge(p1, part2.astype(np.int64)))
        back = odct.blocks_to_image(np.clip(p, 0, 255).astype(np.uint8))
        dt = time.perf_counter() - t
        assert back.shape == strip.shape
        times.append(dt)
        t_used += dt
        done_bytes += strip.nbytes
        r0 = r1 if r1 < HEIGHT // 8 else 0
    print(json.dumps({"bytes": done_bytes, "seconds": t_used, "steps": len(times),
                      "rows_per_step": rows, "times": times}))


def _oracle_cmd(rows, budget, max_steps, start_row=0):
    return [sys.executable, os.path.abspath(__file__), "--oracle-child", "--rows", str(rows),
            "--budget", str(budget), "--max-steps", str(max_steps), "--start-row", str(start_row)]


def _oracle_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    return env


def _run_oracle(rows, budget, max_steps):
    out = subprocess.run(_oracle_cmd(rows, budget, max_steps), capture_output=True, text=True,
                         env=_oracle_env(), check=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def _run_oracle_all_cores(rows, budget):
    """One single-threaded oracle process per host core, each on its own strips, all at once;
    throughput = all processes' bytes / the longest process time."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    nrows = HEIGHT // 8
    procs = [subprocess.Popen(_oracle_cmd(rows, budget, 10 ** 6, (i * nrows // cores) // rows * rows),
                              stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                              env=_oracle_env()) for i in range(cores)]
    res = []
    for p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle child failed")
        res.append(json.loads(out.strip().splitlines()[-1]))
    total = sum(r["bytes"] for r in res)
    secs = max(r["seconds"] for r in res)
    return total, secs, cores


def cpu_baseline():
    r = _run_oracle(rows=32, budget=20.0, max_steps=10 ** 6)
    mbps = r["bytes"] / r["seconds"] / 1e6
    out = {"value": round(mbps, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{r['steps']} strips of {r['rows_per_step']} block rows "
                     f"({r['bytes'] / 1e6:.1f} MB of pixels) of the workload image, "
                     "float64 numpy oracle, one thread"}
    try:
        total, secs, cores = _run_oracle_all_cores(rows=8, budget=8.0)
        out["all_cores"] = {"value": round(total / secs / 1e6, 3), "unit": UNIT, "cores": cores,
                            "sample": f"{cores} single-threaded oracle processes on strips of 8 block "
                                      f"rows ({total / 1e6:.1f} MB of pixels in all) for ~8 s each"}
    except (OSError, RuntimeError, ValueError) as exc:
        out["all_cores"] = {"unavailable": str(exc)}
    return out


def reference_arm(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    # size each step so that warmup + steps stay within about two minutes
    probe = _run_oracle(rows=1, budget=0.0, max_steps=1)
    per_row = max(probe["seconds"], 1e-3)
    rows = int(max(1, min(64, 120.0 / ((args.steps + args.warmup) * per_row))))
    r = _run_oracle(rows=rows, budget=1e9, max_steps=args.steps + args.warmup)
    times = r["times"][args.warmup:] or r["times"]
    step_bytes = rows * 8 * WIDTH * 3
    ms = 1e3 * sum(times) / len(times)
    value = step_bytes / (sum(times) / len(times)) / 1e6
    sample = f"each step: {rows} block rows ({step_bytes / 1e6:.3f} MB) of the workload image"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": world, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm helpers
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# the sources each kernel is compiled from (its translation unit and the shared headers)
KERNEL_SOURCES = {
    "protect_kernel": ["fds_protect.cu"],
    "restore_kernel": ["fds_restore.cu"],
    "protect_tc_kernel": ["fds_protect_tc.cu"],
    "aes_ctr_full_kernel": ["fds_aes_full.cu"],
}
SHARED_HEADERS = ["fds_tile.cuh", "fds_device.cuh", "fds_cos_limbs.h"]


def kernel_source_sha(kernel):
    """Short hash of the sources of one kernel; a committed ncu summary applies only while it
    matches."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1512_02951_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel] + SHARED_HEADERS:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current
    kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_4096_k{K_SEL}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    tr = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not sha or not tr or sha.group(1) != kernel_source_sha(kernel):
        return None
    return int(tr.group(1))


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index):
        import torch
        self.sel = []
        try:
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            self.sel = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"] + self.sel, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        ClockSampler.log.append(self.out or "")

    log: list = []      # samples of every timed region of this process, for emit()

    def summary(self):
        return clock_summary(self.out)


def clock_summary(text):
    """Median SM clock, max clock and active throttle reasons of nvidia-smi samples."""
    sm, mx, reasons = [], None, set()
    for ln in (text or "").splitlines():
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            mx = float(f[1])
        except ValueError:
            continue
        for name, val in zip(ClockSampler.NAMES, f[4:8]):
            if val.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def emit(line):
    """Print a secondary workload's JSON line with the clocks sampled during its timed regions."""
    line.setdefault("clocks", clock_summary("\n".join(ClockSampler.log)))
    print(json.dumps(line), flush=True)


def gpu_arm(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(local)
    img_np = synth.make_image(WIDTH, HEIGHT, IMG_SEED + rank)
    key, iv = synth.make_key(KEY_SEED + rank), synth.make_iv(IV_SEED + rank)
    img = torch.from_numpy(img_np).to(dev)
    pub_b, priv_b = api.sizes(WIDTH, HEIGHT, K_SEL)
    sets = [(torch.empty((HEIGHT // 8, WIDTH // 8, 3, 63 - K_SEL), dtype=torch.int16, device=dev),
             torch.empty(priv_b, dtype=torch.uint8, device=dev)) for _ in range(2)]
    out = torch.empty_like(img)
    stream = torch.cuda.current_stream(dev)

    def step(i, ev=None):
        pub, priv = sets[i % 2]
        opub, opriv = sets[(i + 1) % 2]
        if ev is not None:
            ev[0].record(stream)
        api.protect_image(img, key, iv, K_SEL, pub, priv)
        if ev is not None:
            ev[1].record(stream)
        api.restore_image(opub, opriv, WIDTH, HEIGHT, K_SEL, key, iv, out)
        if ev is not None:
            ev[2].record(stream)

    # correctness of what is timed: fragments and restored image of this very configuration
    api.counters(reset=True)
    step(0)
    step(1)
    torch.cuda.synchronize()
    back = out.cpu().numpy()
    exact_frac = float(np.mean(back == img_np))
    mse = float(np.mean((back.astype(np.float64) - img_np) ** 2))
    psnr = float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            step(i, evs[i])
        stop.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = start.elapsed_time(stop)
    prot_ms = [e[0].elapsed_time(e[1]) for e in evs]
    rest_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = sorted(a + b for a, b in zip(prot_ms, rest_ms))
    n2, n3, fails = api.counters()

    # end to end through the public API from pinned host memory: E2E_LANES steps in flight,
    # each lane a stream with its own device and host buffers (its own copy streams inside
    # the library), so one step's copies overlap the next step's; every step copies its
    # pixels in and both fragments and the restored pixels out inside the timed region
    host_px = torch.from_numpy(img_np).pin_memory()
    lanes = []
    for j in range(E2E_LANES):
        lanes.append({"s": torch.cuda.Stream(dev), "dpx": torch.empty_like(img), "out": torch.empty_like(img),
                      "pub": sets[j % 2][0] if j < 2 else torch.empty_like(sets[0][0]),
                      "priv": sets[j % 2][1] if j < 2 else torch.empty_like(sets[0][1]),
                      "host_pub": torch.empty(sets[0][0].shape, dtype=torch.int16).pin_memory(),
                      "host_priv": torch.empty(priv_b, dtype=torch.uint8).pin_memory(),
                      "host_out": torch.empty(img_np.shape, dtype=torch.uint8).pin_memory()})
    e2e_steps = max(1, min(args.steps, 200))

    def e2e_step(i):
        # the host-buffer entry points: H2D of the pixels, protect, D2H of both fragments,
        # restore, D2H of the pixels, cut into strips so the copies overlap the kernels
        ln = lanes[i % E2E_LANES]
        with torch.cuda.stream(ln["s"]):
            api.protect_image_host(host_px, ln["dpx"], key, iv, K_SEL, ln["pub"], ln["priv"],
                                   ln["host_pub"], ln["host_priv"], E2E_STRIPS)
            api.restore_image_host(ln["pub"], ln["priv"], ln["out"], ln["host_out"], key, iv, K_SEL, E2E_STRIPS)

    for i in range(max(3, E2E_LANES)):
        e2e_step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for ln in lanes:
        ln["s"].wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    for ln in lanes:
        stream.wait_stream(ln["s"])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    for ln in lanes:
        assert np.array_equal(ln["host_out"].numpy(), back)

    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms, e2e_ms = float(t[0]), float(t[1])
    if rank != 0:
        return

    px_bytes = WIDTH * HEIGHT * 3
    ms_per_step = total_ms / args.steps
    value = world * px_bytes / (ms_per_step * 1e-3) / 1e6
    alg_bytes = px_bytes + pub_b + priv_b          # per launch, protect and restore alike
    peak, peak_kind = _peaks()
    prot_avg, rest_avg = sum(prot_ms) / len(prot_ms), sum(rest_ms) / len(rest_ms)
    kern = {}
    for name, ms in (("protect", prot_avg), ("restore", rest_avg)):
        gbs = alg_bytes / (ms * 1e-3) / 1e9
        kern[name] = {"ms": round(ms, 5), "alg_bytes": alg_bytes, "achieved_gbs": round(gbs, 1),
                      "frac": round(gbs / peak, 4)}
    dom = "protect" if prot_avg >= rest_avg else "restore"
    roof = {"bound": "hbm", "achieved": kern[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": kern[dom]["frac"], "traffic": _profiled_traffic(dom + "_kernel"),
            "kernel": dom, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback 6.8 TB/s"}
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(),
            "latency_ms": {"p50": round(step_ms[len(step_ms) // 2], 5),
                           "p99": round(step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))], 5)},
            "roofline": roof, "kernels": kern,
            "e2e": {"value": round(world * px_bytes / (e2e_ms * 1e-3) / 1e6, 1), "unit": UNIT,
                    "h2d_bytes_per_step": px_bytes,
                    "d2h_bytes_per_step": pub_b + priv_b + px_bytes,
                    "note": f"fds_protect_image_host + fds_restore_image_host: H2D pixels, protect, D2H both fragments, restore, D2H pixels, in {E2E_STRIPS} strip{'s' if E2E_STRIPS > 1 else ''} per call, {E2E_LANES} steps in flight on {E2E_LANES} streams with their own buffers; the D2H bytes bound it (host link measured at 193 GB/s device to host, 211 GB/s host to device, 167 GB/s each way together)"},
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
            "quality": {"exact_restore_fraction": round(exact_frac, 5), "psnr_db": round(psnr, 3),
                        "exact_redecisions": n2, "escalations_256bit": n3, "failures": fails},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# batched form: 2000 uneven images, one persistent launch per direction under a CUDA graph
BATCH_N, BATCH_SEED, BATCH_K = 2000, 1000, 0


def batch_inputs(n=BATCH_N, seed=BATCH_SEED):
    """n images with W, H log-uniform in [64, 2048] (multiples of 8), each cropped from one of
    16 seeded 2048 x 2048 generator images at a seeded offset (the generator is the same as
    for single images; cropping keeps the host set-up to seconds)."""
    import numpy as np

    from paper_1512_02951_gb300 import synth

    sizes = synth.batch_sizes(n, seed)
    bases = [synth.make_image(2048, 2048, seed + 5000 + i) for i in range(16)]
    rng = np.random.default_rng(seed + 1)
    crops = []
    for w, h in sizes:
        b = bases[int(rng.integers(0, 16))]
        y0 = int(rng.integers(0, 2048 - h + 1)) & ~7
        x0 = int(rng.integers(0, 2048 - w + 1)) & ~7
        crops.append((b, y0, x0, w, h))
    return sizes, crops


def batch_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    sizes, crops = batch_inputs()
    keys = [synth.make_key(BATCH_SEED + 7000 + i) for i in range(64)]
    slots = [api.key_register(k) for k in keys]
    descs = [api.ImageDesc(w, h, BATCH_K, slots[i % 64], synth.make_iv(BATCH_SEED + 9000 + i))
             for i, (w, h) in enumerate(sizes)]
    npx, npub, npriv = api.layout(descs)
    host = np.zeros(npx, dtype=np.uint8)
    for d, (b, y0, x0, w, h) in zip(descs, crops):
        host[d.pixel_offset: d.pixel_offset + w * h * 3] = b[y0: y0 + h, x0: x0 + w].reshape(-1)
    px = torch.from_numpy(host).to(dev)
    pub = torch.empty(npub, dtype=torch.uint8, device=dev)
    priv = torch.empty(npriv, dtype=torch.uint8, device=dev)
    out = torch.empty_like(px)
    pix_bytes = sum(w * h * 3 for w, h in sizes)
    stream = torch.cuda.Stream(dev)

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            with ClockSampler(0):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    per_image = timed(lambda: (api.protect(px, pub, priv, descs), api.restore(pub, priv, out, descs)),
                      max(1, min(args.steps, 5)))
    ref = (pub.cpu().numpy().copy(), priv.cpu().numpy().copy(), out.cpu().numpy().copy())
    plan = api.Plan(descs)
    with torch.cuda.stream(stream):
        fixed = {}
        for name, ps in (("default_residency", 0), ("one_cta_per_sm", 1)):
            plan.set_schedule(ps, False, False)
            fixed[name] = timed(lambda: (plan.protect(px, pub, priv), plan.restore(pub, priv, out)), args.steps)
        tuned = plan.tune(px, pub, priv, out, reps=3)
    plain = timed(lambda: (plan.protect(px, pub, priv), plan.restore(pub, priv, out)), args.steps)
    graphed = timed(lambda: (plan.protect(px, pub, priv, graph=True),
                             plan.restore(pub, priv, out, graph=True)), args.steps)
    got = (pub.cpu().numpy(), priv.cpu().numpy(), out.cpu().numpy())
    same = all(np.array_equal(a, b) for a, b in zip(ref, got))
    prot = timed(lambda: plan.protect(px, pub, priv, graph=True), args.steps)
    rest = timed(lambda: plan.restore(pub, priv, out, graph=True), args.steps)
    cands = tuned["candidates"]
    sched = {"size_class": tuned["size_class"], "largest_first": tuned["largest_first"],
             "protect": tuned["protect"], "restore": tuned["restore"], "candidates_timed": len(cands),
             "candidate_ms_range": {d: [round(min(c["ms"] for c in cands if c["direction"] == d), 4),
                                        round(max(c["ms"] for c in cands if c["direction"] == d), 4)]
                                    for d in ("protect", "restore")}}
    line = {"metric": METRIC + " (batched form)", "value": round(pix_bytes / (graphed * 1e-3) / 1e6, 1),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(graphed, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{BATCH_N} RGB uint8 images, W,H log-uniform [64,2048], k={BATCH_K}, "
                                   "protect+restore", "images": BATCH_N, "pixel_bytes": pix_bytes,
                       "schedule": sched},
            "images_per_s": {"graph": round(BATCH_N / (graphed * 1e-3), 1),
                             "plan_no_graph": round(BATCH_N / (plain * 1e-3), 1),
                             "per_image_launches": round(BATCH_N / (per_image * 1e-3), 1)},
            "ms": {"graph": round(graphed, 4), "plan_no_graph": round(plain, 4),
                   "per_image_launches": round(per_image, 4), "protect_graph": round(prot, 4),
                   "restore_graph": round(rest, 4),
                   "untuned_plan": {k: round(v, 4) for k, v in fixed.items()}},
            "bit_identical_to_per_image": same,
            "protect_roofline_frac": round(pix_bytes * 3 / (prot * 1e-3) / 1e9 / _peaks()[0], 4),
            "restore_roofline_frac": round(pix_bytes * 3 / (rest * 1e-3) / 1e9 / _peaks()[0], 4),
            "gpu_launches": 2 * args.steps}
    plan.close()
    emit(line)


# ------------------------------------------------------------------------------------------
# precision form: the 4096 x 4096 image with the DCT on the tensor cores (BF16 / TF32 limbs)
def _fp64_dct(img):
    """float64 DCT-II of every 8x8 block of every channel, [H/8, W/8, 3, 8, 8] (torch on the
    device, straight from the orthonormal basis formula; a measuring stick for the float32
    coefficients, not part of the path)."""
    import math

    import torch
    b = torch.empty((8, 8), dtype=torch.float64)
    for u in range(8):
        for y in range(8):
            b[u, y] = (math.sqrt(0.5) if u == 0 else 1.0) * 0.5 * math.cos((2 * y + 1) * u * math.pi / 16)
    b = b.to(img.device)
    h, w, _ = img.shape
    blk = img.to(torch.float64).reshape(h // 8, 8, w // 8, 8, 3).permute(0, 2, 4, 1, 3)
    return torch.einsum("uy,abcyx,vx->abcuv", b, blk, b)


def _median_launch_ms(fn, args, flush, stream):
    """Median CUDA-event time of args.steps launches of fn after args.warmup, L2 flushed
    between them, nvidia-smi clocks sampled meanwhile."""
    import numpy as np
    import torch

    for _ in range(args.warmup):
        fn()
    ts = []
    with ClockSampler(0):
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def precision_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    img_np = synth.make_image(WIDTH, HEIGHT, IMG_SEED)
    img = torch.from_numpy(img_np).to(dev)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    pub_b, priv_b = api.sizes(WIDTH, HEIGHT, K_SEL)
    pub = torch.empty((HEIGHT // 8, WIDTH // 8, 3, 63 - K_SEL), dtype=torch.int16, device=dev)
    priv = torch.empty(priv_b, dtype=torch.uint8, device=dev)
    out = torch.empty_like(img)
    ref64 = _fp64_dct(img)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    forms = {"f32_cuda_cores": (lambda: api.protect_image(img, key, iv, K_SEL, pub, priv),
                                lambda: api.debug_dct_f32(img)),
             "bf16_3limb_tcgen05": (lambda: api.protect_image_tc(img, key, iv, K_SEL, "bf16", pub, priv),
                                    lambda: api.debug_dct_tc(img, "bf16")),
             "tf32_2limb_tcgen05": (lambda: api.protect_image_tc(img, key, iv, K_SEL, "tf32", pub, priv),
                                    lambda: api.debug_dct_tc(img, "tf32")),
             "f16_3limb_tcgen05_warp_specialised": (
                 lambda: api.protect_image_tc(img, key, iv, K_SEL, "f16", pub, priv),
                 lambda: api.debug_dct_tc(img, "f16"))}
    alg_bytes = WIDTH * HEIGHT * 3 + pub_b + priv_b
    peak, _ = _peaks()
    res, first = {}, None
    for name, (protect, coefs) in forms.items():
        err = (coefs().to(torch.float64) - ref64).abs().max().item()
        api.counters(reset=True)
        protect()
        torch.cuda.synchronize()
        slow, esc, fails = api.counters()
        frags = (pub.clone(), priv.clone())
        if first is None:
            first = frags
        api.restore_image(pub, priv, WIDTH, HEIGHT, K_SEL, key, iv, out)
        exact_frac = (out == img).to(torch.float64).mean().item()
        ms = _median_launch_ms(protect, args, flush, stream)
        gbs = alg_bytes / (ms * 1e-3) / 1e9
        res[name] = {"protect_ms": round(ms, 5), "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                     "max_abs_coef_err_vs_fp64": err, "slow_path_values": slow, "escalations_256bit": esc,
                     "failures": fails, "exact_restore_fraction": round(exact_frac, 6),
                     "bit_identical_to_f32_path": bool(torch.equal(frags[0], first[0]) and
                                                       torch.equal(frags[1], first[1]))}
    api.protect_image(img, key, iv, K_SEL, pub, priv)
    restore = {}
    rforms = {"f32_cuda_cores": lambda: api.restore_image(pub, priv, WIDTH, HEIGHT, K_SEL, key, iv, out),
              "f16_3limb_tcgen05_inverse": lambda: api.restore_image_tc(pub, priv, WIDTH, HEIGHT, K_SEL, key, iv, out)}
    rfirst = None
    for name, fn in rforms.items():
        api.counters(reset=True)
        out.fill_(0)
        fn()
        torch.cuda.synchronize()
        slow, esc, fails = api.counters()
        got = out.clone()
        if rfirst is None:
            rfirst = got
        rms = _median_launch_ms(fn, args, flush, stream)
        rgbs = alg_bytes / (rms * 1e-3) / 1e9
        restore[name] = {"restore_ms": round(rms, 5), "achieved_gbs": round(rgbs, 1), "frac": round(rgbs / peak, 4),
                         "slow_path_values": slow, "escalations_256bit": esc, "failures": fails,
                         "exact_restore_fraction": round((got == img).to(torch.float64).mean().item(), 6),
                         "bit_identical_to_f32_path": bool(torch.equal(got, rfirst))}
    bounds = {f: api.tc_basis(f)[1] for f in ("bf16", "tf32", "f16")}
    bounds["f16_inverse_per_unit_sum_abs_q"] = api.tc_basis("f16_inverse")[1]
    best = max(res.values(), key=lambda r: r["achieved_gbs"])
    # the headline: the fastest tensor-core form
    tc_name = min((n for n in res if n != "f32_cuda_cores"), key=lambda n: res[n]["protect_ms"])
    tc_ms = res[tc_name]["protect_ms"]
    line = {"metric": "protect MB/s of pixels (precision forms)",
            "value": round(WIDTH * HEIGHT * 3 / (tc_ms * 1e-3) / 1e6, 1),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tc_ms, "higher_is_better": True, "headline_form": tc_name,
            "scaling": "weak", "vs_baseline": None,
            "dtype": tc_name.split("_")[0] + " limbs, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": f"{WIDTH}x{HEIGHT} RGB uint8, protect, k={K_SEL}, DCT as tensor-core MMAs",
                       "l2": "256 MB buffer written between timed launches"},
            "forms": res, "restore": restore, "proven_error_bounds": bounds,
            "roofline": {"bound": "hbm", "achieved": best["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": best["frac"], "traffic": None},
            "gpu_launches": args.steps * (len(forms) + len(rforms))}
    emit(line)


# ------------------------------------------------------------------------------------------
# selective vs full encryption (the paper's comparison, Tables 7, 9, 11) on the same GPU
def compare_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    img_np = synth.make_image(WIDTH, HEIGHT, IMG_SEED)
    img = torch.from_numpy(img_np).to(dev)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    px_bytes = WIDTH * HEIGHT * 3
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    full_out = torch.empty_like(img)

    def timed(fn):
        return _median_launch_ms(fn, args, flush, stream)   # L2 flushed between timed launches

    res = {}
    full_ms = timed(lambda: api.encrypt_full(img, key, iv, out=full_out))
    res["full_aes128_ctr"] = {"ms": round(full_ms, 5), "MBps": round(px_bytes / (full_ms * 1e-3) / 1e6, 1)}
    for k in (0, 5):
        pub_b, priv_b = api.sizes(WIDTH, HEIGHT, k)
        pub = torch.empty((HEIGHT // 8, WIDTH // 8, 3, 63 - k), dtype=torch.int16, device=dev)
        priv = torch.empty(priv_b, dtype=torch.uint8, device=dev)
        out = torch.empty_like(img)
        p_ms = timed(lambda: api.protect_image(img, key, iv, k, pub, priv))
        r_ms = timed(lambda: api.restore_image(pub, priv, WIDTH, HEIGHT, k, key, iv, out))
        res[f"selective_k{k}"] = {"protect_ms": round(p_ms, 5), "restore_ms": round(r_ms, 5),
                                  "protect_MBps": round(px_bytes / (p_ms * 1e-3) / 1e6, 1),
                                  "encrypted_bytes": priv_b,
                                  "protect_time_vs_full_encryption": round(p_ms / full_ms, 3)}
    peak, _ = _peaks()
    full_gbs = 2 * px_bytes / (full_ms * 1e-3) / 1e9
    line = {"metric": "selective protection vs full AES-128-CTR of the pixels, MB/s of pixels",
            "value": res["selective_k5"]["protect_MBps"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["selective_k5"]["protect_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{WIDTH}x{HEIGHT} RGB uint8: protect (k=0, 5) vs AES-128-CTR of all "
                                   "pixel bytes", "l2": "256 MB buffer written between timed launches"},
            "results": res,
            "full_encryption_roofline": {"bound": "hbm", "achieved": round(full_gbs, 1), "peak": peak,
                                         "unit": "GB/s", "frac": round(full_gbs / peak, 4)},
            "gpu_launches": args.steps * 5}
    emit(line)


# ------------------------------------------------------------------------------------------
# bit-packed storage (Sect. 6.4.3, Table 5): protect / restore with 11-bit and 8-bit fields
def packed_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    img_np = synth.make_image(WIDTH, HEIGHT, IMG_SEED)
    img = torch.from_numpy(img_np).to(dev)
    img_np = img_np.astype(np.float64)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    px_bytes = WIDTH * HEIGHT * 3
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        return _median_launch_ms(fn, args, flush, stream)   # L2 flushed between timed launches

    res = {}
    pub16_b, priv16_b = api.sizes(WIDTH, HEIGHT, K_SEL)
    pub16 = torch.empty((HEIGHT // 8, WIDTH // 8, 3, 63 - K_SEL), dtype=torch.int16, device=dev)
    priv16 = torch.empty(priv16_b, dtype=torch.uint8, device=dev)
    out = torch.empty_like(img)
    res["int16"] = {"protect_ms": round(timed(lambda: api.protect_image(img, key, iv, K_SEL, pub16, priv16)), 5),
                    "restore_ms": round(timed(lambda: api.restore_image(pub16, priv16, WIDTH, HEIGHT, K_SEL,
                                                                         key, iv, out)), 5),
                    "public_bytes": pub16_b, "private_bytes": priv16_b}
    for form in (11, 8):
        pub_b, priv_b, scr_b = api.sizes_packed(WIDTH, HEIGHT, K_SEL, form)
        scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
        pub = torch.empty(pub_b, dtype=torch.uint8, device=dev)
        priv = torch.empty(max(priv_b, 16), dtype=torch.uint8, device=dev)
        p_ms = timed(lambda: api.protect_image_packed(img, key, iv, K_SEL, form, scratch, pub, priv))
        r_ms = timed(lambda: api.restore_image_packed(pub, priv[:priv_b], WIDTH, HEIGHT, K_SEL, key, iv, form,
                                                      scratch, out))
        back = out.cpu().numpy().astype(np.float64)
        mse = float(np.mean((back - img_np) ** 2))
        res[f"packed{form}"] = {"protect_ms": round(p_ms, 5), "restore_ms": round(r_ms, 5),
                                "restore_psnr_db": round(10.0 * np.log10(255.0 ** 2 / mse), 3) if mse else None,
                                "restore_exact_fraction": round(float((back == img_np).mean()), 5),
                                "public_bytes": pub_b, "private_bytes": priv_b,
                                "stored_fraction_of_pixels": round((pub_b + priv_b) / px_bytes, 4),
                                "private_fraction_of_pixels": round(priv_b / px_bytes, 4)}
    p11 = res["packed11"]["protect_ms"]
    line = {"metric": "protect throughput with 11-bit packed storage, MB/s of pixels",
            "value": round(px_bytes / (p11 * 1e-3) / 1e6, 1), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": p11,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{WIDTH}x{HEIGHT} RGB uint8, k={K_SEL}: int16 vs 11-bit vs 8-bit "
                                   "fragment storage", "l2": "256 MB buffer written between timed launches"},
            "results": res,
            "gpu_launches": args.steps * 6}   # int16 2 + 2 forms x (protect 1 + restore 1)
    emit(line)


# ------------------------------------------------------------------------------------------
# strong level (Sect. 6.3.2, Tables 10, 11): public image XOR SHA-512 of Part 1 per block, vs
# full AES-128-CTR of the pixels on the same GPU
def strong_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    img_np = synth.make_image(WIDTH, HEIGHT, IMG_SEED)
    img = torch.from_numpy(img_np).to(dev)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    px_bytes = WIDTH * HEIGHT * 3
    ncb = px_bytes // 64
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        return _median_launch_ms(fn, args, flush, stream)   # L2 flushed between timed launches

    _, priv_b, scr_b = api.sizes_strong(WIDTH, HEIGHT, K_SEL)
    scratch = torch.empty(scr_b, dtype=torch.uint8, device=dev)
    pub = torch.empty_like(img)
    priv = torch.empty(priv_b, dtype=torch.uint8, device=dev)
    out = torch.empty_like(img)
    full_out = torch.empty_like(img)
    p_ms = timed(lambda: api.protect_image_strong(img, key, iv, K_SEL, scratch, pub, priv))
    r_ms = timed(lambda: api.restore_image_strong(pub, priv, K_SEL, key, iv, scratch, out))
    full_ms = timed(lambda: api.encrypt_full(img, key, iv, out=full_out))
    back = out.cpu().numpy()
    pub16, _ = api.protect_image(img, key, iv, K_SEL)
    pimg = torch.empty_like(img)
    pi_ms = timed(lambda: api.public_image(pub16, WIDTH, HEIGHT, K_SEL, pimg))
    st_ms = timed(lambda: api.image_stats(img))
    r_img = api.correlation(api.image_stats(img)[1])
    r_pub = api.correlation(api.image_stats(pimg)[1])
    r_strong = api.correlation(api.image_stats(pub)[1])
    mse = float(np.mean((back.astype(np.float64) - img_np.astype(np.float64)) ** 2))
    res = {"protect_ms": round(p_ms, 5), "restore_ms": round(r_ms, 5),
           "protect_MBps": round(px_bytes / (p_ms * 1e-3) / 1e6, 1),
           "sha512_hashes_per_protect": ncb,
           "full_aes128_ctr_ms": round(full_ms, 5),
           "protect_time_vs_full_encryption": round(p_ms / full_ms, 3),
           "restore_psnr_db": round(10.0 * np.log10(255.0 ** 2 / mse), 3) if mse else None,
           "restore_exact_fraction": round(float((back == img_np).mean()), 5),
           "public_image_ms": round(pi_ms, 5),
           "public_image_GBps": round((2 * (63 - K_SEL) / 64 + 1) * px_bytes / (pi_ms * 1e-3) / 1e9, 1),
           "image_stats_ms": round(st_ms, 5),
           "adjacent_pixel_correlation": {
               "original": [[round(v, 4) for v in row] for row in r_img],
               "public_image": [[round(v, 4) for v in row] for row in r_pub],
               "strong_public_image": [[round(v, 4) for v in row] for row in r_strong],
               "order": "[right, down, down-right][R, G, B]"}}
    line = {"metric": "strong-level protect throughput, MB/s of pixels",
            "value": res["protect_MBps"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["protect_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{WIDTH}x{HEIGHT} RGB uint8, k={K_SEL}: strong level (public image "
                                   "XOR SHA-512 of Part 1) vs AES-128-CTR of all pixel bytes",
                       "l2": "256 MB buffer written between timed launches"},
            "results": res,
            "gpu_launches": args.steps * (4 + 4 + 1 + 1 + 1)}
    emit(line)


# ------------------------------------------------------------------------------------------
# the DWT scheme (Sect. 6.8-6.12, Table 15): Le Gall 5/3 + AES-CTR + SHA-256/512 masks on a
# byte matrix, vs AES-128-CTR of the same bytes
DWT_W = DWT_H = 4800


def dwt_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth

    build.build()
    api.init(0)
    dev = torch.device("cuda", 0)
    data_np = synth.make_image(DWT_W, DWT_H, IMG_SEED)[..., 0].copy()   # a grey 4800 x 4800 matrix
    data = torch.from_numpy(data_np).to(dev)
    key, iv = synth.make_key(KEY_SEED), synth.make_iv(IV_SEED)
    nbytes = DWT_W * DWT_H
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        return _median_launch_ms(fn, args, flush, stream)   # L2 flushed between timed launches

    outs = tuple(torch.empty(n, dtype=torch.uint8, device=dev) for n in api.dwt_sizes(DWT_W, DWT_H))
    back = torch.empty_like(data)
    full_out = torch.empty_like(data)
    p_ms = timed(lambda: api.dwt_protect(data, key, iv, outs))
    r_ms = timed(lambda: api.dwt_restore(*outs, DWT_W, DWT_H, key, iv, back))
    full_ms = timed(lambda: api.encrypt_full(data, key, iv, out=full_out))
    exact = bool(torch.equal(back, data))
    stored = sum(o.numel() for o in outs)
    res = {"protect_ms": round(p_ms, 5), "restore_ms": round(r_ms, 5),
           "protect_MBps": round(nbytes / (p_ms * 1e-3) / 1e6, 1),
           "restore_MBps": round(nbytes / (r_ms * 1e-3) / 1e6, 1),
           "restore_exact": exact,
           "blocks": nbytes // 64, "sha256_and_sha512_hashes_each": nbytes // 64,
           "private_bytes": outs[0].numel() + outs[1].numel(), "public_bytes": outs[2].numel(),
           "stored_fraction": round(stored / nbytes, 4),
           "full_aes128_ctr_ms": round(full_ms, 5),
           "protect_time_vs_full_encryption": round(p_ms / full_ms, 3)}
    line = {"metric": "DWT selective encryption throughput, MB/s of data",
            "value": res["protect_MBps"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["protect_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"{DWT_W}x{DWT_H} byte matrix: two-level Le Gall 5/3 per 8x8 block, "
                                   "AES-128-CTR level 1, SHA-256 / SHA-512 masks on levels 2 / 3",
                       "l2": "256 MB buffer written between timed launches"},
            "results": res,
            "gpu_launches": args.steps * 3}
    emit(line)


# ------------------------------------------------------------------------------------------
# serving form: Poisson arrivals, mixed protect / restore, continuous batching
SERVE_N, SERVE_RATE, SERVE_SEED = 1500, 500.0, 4242


def serve_arm(args):
    import numpy as np
    import torch

    from paper_1512_02951_gb300 import api, build, synth
    from paper_1512_02951_gb300.serve import Request, Server, run_poisson

    build.build()
    api.init(0)
    sizes, crops = batch_inputs(SERVE_N, SERVE_SEED)
    keys = [synth.make_key(SERVE_SEED + 100 + i) for i in range(64)]
    slots = [api.key_register(k) for k in keys]
    rng = np.random.default_rng(SERVE_SEED)

    def make_requests():
        reqs = []
        for i, (b, y0, x0, w, h) in enumerate(crops):
            img = torch.from_numpy(np.ascontiguousarray(b[y0: y0 + h, x0: x0 + w])).pin_memory()
            slot = slots[int(rng.integers(0, 64))]
            iv = synth.make_iv(SERVE_SEED + 1000 + i)
            if i % 2 == 0:
                reqs.append(Request("protect", w, h, 0, slot, iv, pixels=img))
            else:                                   # restore inputs, protected beforehand
                pub, priv = api.protect_image(img.cuda(), keys[slots.index(slot)], iv, 0)
                reqs.append(Request("restore", w, h, 0, slot, iv, public=pub.cpu().pin_memory(),
                                    private=priv.cpu().pin_memory()))
        torch.cuda.synchronize()
        return reqs

    reqs = make_requests()
    arrivals = synth.poisson_arrivals(len(reqs), SERVE_RATE, SERVE_SEED)
    srv = Server(lanes=3, max_batch=64)

    def outputs(r):
        """Pinned output buffers of the request's result (the caller's, reused across runs)."""
        n, pb, vb = r.sizes()
        return tuple(torch.empty(b, dtype=torch.uint8).pin_memory() for b in ((pb, vb) if r.kind == "protect" else (n,)))

    outs_a = [outputs(r) for r in reqs]             # the Poisson run's results
    outs_b = [outputs(r) for r in reqs]             # the warm-up's and the saturated run's
    for r, o in zip(reqs, outs_a):
        r.out = o
    # warm-up: every request once, all at once, so that the device and pinned-host caching
    # allocators hold blocks of every size the timed runs need
    warm = [Request(r.kind, r.width, r.height, r.k, r.key_slot, r.iv, r.pixels, r.public, r.private, out=o)
            for r, o in zip(reqs, outs_b)]
    run_poisson(srv, warm, np.zeros(len(warm)))
    with ClockSampler(0):
        poisson = run_poisson(srv, reqs, arrivals)
    stats_p = dict(srv.stats)
    again = [Request(r.kind, r.width, r.height, r.k, r.key_slot, r.iv, r.pixels, r.public, r.private, out=o)
             for r, o in zip(reqs, outs_b)]
    with ClockSampler(0):
        burst = run_poisson(srv, again, np.zeros(len(again)))      # all at once: saturation
    srv.close()
    same = all((np.array_equal(a.future.result()[0], b.future.result()[0]) and
                a.future.result()[1] == b.future.result()[1]) if a.kind == "protect"
               else np.array_equal(a.future.result(), b.future.result()) for a, b in zip(reqs, again))
    line = {"metric": "serving p50/p99 ms per request and sustained MB/s of pixels",
            "value": round(poisson["p99_ms"], 3), "unit": "ms (p99)", "n_gpus": 1,
            "steps": len(reqs), "warmup": len(warm), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{SERVE_N} requests, Poisson {SERVE_RATE:g} req/s, 50/50 protect/restore, "
                                   "W,H log-uniform [64,2048], k=0, 64 device-resident keys, "
                                   "memory-based admission, 3 lanes, batches up to 64, pinned inputs, "
                                   "results copied from the device into per-request pinned output buffers"},
            "poisson": {k: round(v, 3) for k, v in poisson.items()},
            "saturation": {k: round(v, 3) for k, v in burst.items()},
            "batches": stats_p["batches"], "max_batch": stats_p["max_batch"],
            "max_lanes_busy": stats_p["max_lanes_busy"],
            "same_results_in_both_runs": same}
    emit(line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["image4096", "precision", "compare", "batch2000", "serve", "packed", "strong", "dwt"],
                    default="image4096")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--rows", type=int, default=32, help=argparse.SUPPRESS)
    ap.add_argument("--budget", type=float, default=20.0, help=argparse.SUPPRESS)
    ap.add_argument("--max-steps", type=int, default=10 ** 6, help=argparse.SUPPRESS)
    ap.add_argument("--start-row", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.oracle_child:
        _oracle_child(args)
    elif args.impl == "reference":
        reference_arm(args)
    elif args.workload == "precision":
        precision_arm(args)
    elif args.workload == "compare":
        compare_arm(args)
    elif args.workload == "batch2000":
        batch_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    elif args.workload == "packed":
        packed_arm(args)
    elif args.workload == "strong":
        strong_arm(args)
    elif args.workload == "dwt":
        dwt_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
