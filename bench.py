"""Benchmark: secondary samples/s and ms per 800x800 frame of the fused renderer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16] [--impl ours|reference]

One step renders one 800x800 frame (N = 128 directions per pixel, M = 8 per
secondary point, L = 16 levels, T = 2^19, resolutions 16..2048, 64x128 env)
through the C ABI, i.e. one launch of the fused kernel; the headline is the
BF16 tensor-core path (FP16 table) and the FP32 path of the same workload is
timed in the same run under "compare".  Four seeded scenes
(tables, MLPs, env maps and G-buffers, about 420 MB in FP32) are rotated
step by step, so every step starts with its inputs out of the 129 MB L2.
Under torchrun each rank renders its own scenes (weak scaling, no data-path
collective); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the only other place this script runs oracle/).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenegen  # noqa: E402

METRIC = "secondary samples/s & ms/frame at 800² (BF16 vs FP32, ≥45 dB PSNR vs FP64)"
UNIT = "samples/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 FFMA peak of a GB300: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_NOTE = "4 scenes rotated, one per step (73 MB each in BF16, 105 MB in FP32; 290-420 MB in total > 129 MB L2)"


def algorithmic_flop_per_sample(cfg) -> int:
    """MLP multiply-adds x 2 per secondary sample, unpadded: (1 + M) I evaluations and one B."""
    lf = cfg.levels * 2
    irt = (lf + 27) * 64 + 64 * 64 + 64 * 2
    brdf = lf * 64 + 64 * 64 + 64 * 7
    return 2 * ((1 + cfg.m_dirs) * irt + brdf)


def workload_name(cfg) -> str:
    return (f"{cfg.name}: {cfg.width}x{cfg.height} px, N={cfg.n_dirs}, M={cfg.m_dirs}, L={cfg.levels}, "
            f"T=2^{cfg.log2_T}, res {cfg.base_res}-{cfg.max_res}, env {cfg.env_h}x{cfg.env_w}, {cfg.precision}")


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu() -> dict:
    """The host's logical CPU count and model name (lscpu; /proc/cpuinfo as a fallback)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    return {"nproc": os.cpu_count(), "model": model}


def cpu_oracle_rate(cfg, seconds: float, seed: int = 0, threads: int = 0, keep: bool = False):
    """Samples/s of the FP64 oracle on a bounded pixel sample of the workload (host cores;
    threads > 0 limits torch's intra-op threads for this call).  Returns (samples/s, pixels,
    seconds, threads) and, with keep=True, also the rendered rows and their radiance."""
    import torch
    if threads > 0:
        saved = torch.get_num_threads()
        torch.set_num_threads(threads)
        try:
            return cpu_oracle_rate(cfg, seconds, seed, keep=keep)
        finally:
            torch.set_num_threads(saved)
    from oracle import render as orender
    sc = scenegen.make_scene(cfg, seed)
    gb = scenegen.make_gbuffer(cfg.n_pixels, seed)
    prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)
    opt = orender.Options.from_config(cfg)
    rows = scenegen.subset_permutation(cfg.n_pixels, cfg.n_pixels, seed=1)
    chunk = max(1, (1 << 15) // cfg.n_dirs)
    done, t0 = 0, time.perf_counter()
    outs = []
    while True:
        o = orender.render(gb, prm, opt, rows=rows[done:done + chunk])
        if keep:
            outs.append(o)
        done += chunk
        el = time.perf_counter() - t0
        if el >= seconds or done >= cfg.n_pixels:
            break
    done = min(done, cfg.n_pixels)
    res = (done * cfg.n_dirs / el, done, el, torch.get_num_threads())
    if keep:
        return res + (rows[:done], np.concatenate(outs, axis=0)[:done])
    return res


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def golden_frame_stats(cfg, seed: int):
    """(peak, p99.9) of the whole FP64 oracle frame from tests/golden, or None."""
    path = os.path.join(GOLDEN_DIR, f"{cfg.name.split('[')[0].replace('_bf16', '')}_seed{seed}_stats.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if not line.startswith("#") and len(line.split()) == 2:
            kv[line.split()[0]] = float(line.split()[1])
    return (kv["peak"], kv["p999"]) if "peak" in kv and "p999" in kv else None


def parity_stats(got: np.ndarray, ref: np.ndarray, precision: str, peaks=None) -> dict:
    """Errors of a rendered sample against the FP64 oracle's radiance of the same pixels."""
    err = np.abs(got - ref)
    amax = float(np.abs(ref).max()) if ref.size else 1.0
    rel = err / np.maximum(np.abs(ref), 1e-6 * amax)
    st = {"pixels": int(ref.shape[0]), "frame_rel_l1": float(err.sum() / max(np.abs(ref).sum(), 1e-300)),
          "max_abs": float(err.max()), "max_rel": float(rel.max()), "median_rel": float(np.median(rel))}
    if precision == "bf16":
        mse = float((err ** 2).mean())
        peak, p999 = peaks if peaks is not None else (amax, float(np.quantile(ref, 0.999)))
        st["psnr_db_peak_max"] = 10.0 * math.log10(peak * peak / mse) if mse > 0 else float("inf")
        st["psnr_db_peak_p999"] = 10.0 * math.log10(p999 * p999 / mse) if mse > 0 else float("inf")
        st["peaks"] = {"max": peak, "p999": p999,
                       "source": "whole-frame FP64 oracle (tests/golden)" if peaks is not None else "the sample"}
    return st


def run_reference(args, cfg):
    rank, _, world = dist_info()
    if rank != 0:
        return
    rate_steps = []
    per_step = max(1.0, args.ref_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_oracle_rate(cfg, 0.2)
    samples, secs = 0, 0.0
    for _ in range(args.steps):
        r, done, el, cores = cpu_oracle_rate(cfg, per_step)
        samples += done * cfg.n_dirs
        secs += el
        rate_steps.append(r)
    value = samples / secs
    ms_frame = cfg.samples / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "ms_per_frame": ms_frame, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(cfg), "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{samples // cfg.n_dirs} pixels of the 800x800 frame over {args.steps} steps "
                                       f"(~{per_step:.0f} s each), extrapolated to samples/s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _setup(cfg, rank, n_scenes=4, **overrides):
    import torch
    from paper_2409_10327_gb300 import binding
    renderers, gbs = [], []
    for s in range(n_scenes):
        seed = rank * n_scenes + s
        sc = scenegen.make_scene(cfg, seed)
        r = binding.Renderer(binding.make_config(cfg, **overrides))
        table = torch.from_numpy(sc.table).cuda()
        if cfg.precision == "bf16":
            table = table.half()
        r.set_params(table, torch.from_numpy(sc.brdf_blob).cuda(), torch.from_numpy(sc.irt_blob).cuda(),
                     torch.from_numpy(sc.env).cuda())
        renderers.append(r)
        gbs.append({k: torch.from_numpy(v).cuda() for k, v in scenegen.make_gbuffer(cfg.n_pixels, seed).items()})
    return renderers, gbs


def _time_frames(renderers, gbs, out, steps, warmup, barrier, clocks=None):
    """Kernel-time the fused render over `steps` frames rotating the scenes; returns (total ms, per-launch ms)."""
    import torch
    stream = torch.cuda.current_stream()
    n = len(renderers)
    for w in range(warmup):
        renderers[w % n].render_frame(gbs[w % n], out=out)
    barrier()
    if clocks is not None:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        renderers[k % n].render_frame(gbs[k % n], out=out)
        ev[k][1].record(stream)
    t1.record(stream)
    barrier()
    clk = clocks.stop() if clocks is not None else None
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev], clk


# Per-launch DRAM traffic of the timed kernels, from one ncu pass over a whole
# frame (dram__bytes_read.sum + dram__bytes_write.sum).  Each record names the
# SHA-256 of the kernel's sources at capture time; a kernel changed since then
# reports null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_frame800.txt")
KERNEL_SOURCES = {
    "bf16": ["render_bf16.cu", "render_bf16_kernel.cuh", "tc_common.cuh", "fast_math.cuh", "mis.cuh", "mbarrier.cuh",
             "device_common.cuh", "rt_internal.h"],
    "fp32": ["render_fp32.cu", "warp_gemm.cuh", "mis.cuh", "device_common.cuh", "rt_internal.h"],
}


def kernel_source_hash(precision: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[precision]:
        with open(os.path.join(ROOT, "paper_2409_10327_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(cfg):
    """DRAM bytes per launch for this precision at the 800x800 workload, or None."""
    if cfg.n_pixels != 800 * 800 or not os.path.exists(TRAFFIC_FILE):
        return None
    want = kernel_source_hash(cfg.precision)
    with open(TRAFFIC_FILE) as fh:
        for line in fh:
            if line.startswith("#") or "=" not in line:
                continue
            kv = dict(item.split("=", 1) for item in line.split())
            if kv.get("precision") == cfg.precision and kv.get("source_sha256") == want:
                return int(kv["bytes_per_launch"])
    return None


def measured_l2_sectors_per_sample(cfg):
    """L2 sectors read per secondary sample by the frame kernel (ncu lts__t_sectors_srcunit_tex_op_read
    over a capture, divided by its samples), recorded beside the traffic for the current sources, or None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    want = kernel_source_hash(cfg.precision)
    for line in open(TRAFFIC_FILE):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(item.split("=", 1) for item in line.split())
        if kv.get("precision") == cfg.precision and kv.get("source_sha256") == want and "l2_sectors_per_sample" in kv:
            return float(kv["l2_sectors_per_sample"])
    return None


def measure_probe_peaks(table_bytes: int = 32 << 20, reps: int = 5) -> dict:
    """Live ceilings from the library's probe kernels, timed with CUDA events on the current stream:
    random 4- and 8-byte gathers over an L2-resident table of the FP16 frame table's size (32 MiB), and
    FP32 FMA throughput.  Each figure is the best of `reps` launches after two warm-ups (a burst rate)."""
    import torch
    from paper_2409_10327_gb300 import binding
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 4 * sms                     # 2048 threads per SM
    stream = torch.cuda.current_stream()
    table = torch.randint(0, 1 << 30, (table_bytes // 4,), dtype=torch.int32, device="cuda")
    sink = torch.empty(blocks * 512, dtype=torch.float32, device="cuda")
    isink = sink.view(torch.int32)

    def best_ms(fn):
        for _ in range(2):
            fn()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return min(times)
    out = {"how": f"rt_probe_gather / rt_probe_ffma, {blocks} blocks x 512 threads, best of {reps} after 2 warm-ups"}
    iters = 512
    for bpl in (4, 8):
        ms = best_ms(lambda: binding.probe_gather(table, bpl, iters, blocks, sink=isink))
        loads = blocks * 512 * iters * 8
        out[f"l2_gather_{bpl}B"] = {"table_MiB": table_bytes >> 20, "ms": ms, "loads_per_s": loads / (ms / 1e3),
                                    "useful_GBps": loads * bpl / (ms / 1e3) / 1e9}
    f_iters = 4096
    ms = best_ms(lambda: binding.probe_ffma(f_iters, blocks, sink=sink))
    out["ffma_tflops"] = blocks * 512 * f_iters * 256 / (ms / 1e3) / 1e12
    out["ffma_ms"] = ms
    del table, sink
    return out


def _roofline(cfg, launch_ms, peaks, probes=None):
    flop = algorithmic_flop_per_sample(cfg) * cfg.samples
    avg_s = sum(launch_ms) / len(launch_ms) / 1e3
    if cfg.precision == "fp32":
        if probes and probes.get("ffma_tflops"):
            roof = {"bound": "alu", "achieved": flop / avg_s / 1e12, "peak": probes["ffma_tflops"], "unit": "TFLOP/s",
                    "peak_source": "of measured (rt_probe_ffma, burst, same run)"}
        else:
            roof = {"bound": "alu", "achieved": flop / avg_s / 1e12, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_source": "nominal: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"}
    else:
        # one launch of tens of ms timed alone is a burst: the burst cuBLAS figure is its denominator
        pk = peaks.get("bf16_tflops")
        roof = {"bound": "tensor", "achieved": flop / avg_s / 1e12, "peak": pk if pk else 1900.0, "unit": "TFLOP/s",
                "peak_source": "of measured (bf16_tflops, burst)" if pk else "of fallback (1.9 PFLOP/s burst)"}
        if peaks.get("bf16_tflops_sustained"):
            roof["frac_of_sustained"] = roof["achieved"] / peaks["bf16_tflops_sustained"]
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = measured_traffic(cfg)
    roof["algorithmic_per_launch"] = flop
    roof["kernel_ms"] = avg_s * 1e3
    bpl = 4 if cfg.precision == "bf16" else 8          # bytes of one table entry (one hash-grid corner)
    gather_bytes = cfg.samples * cfg.levels * 8 * bpl
    corners_per_s = cfg.samples * cfg.levels * 8 / avg_s
    hbm = peaks.get("hbm_gbs")
    g = {"algorithmic_bytes_per_launch": gather_bytes, "algorithmic_bytes_per_sample": cfg.levels * 8 * bpl,
         "achieved_GBps": gather_bytes / avg_s / 1e9, "hbm_peak_GBps": hbm,
         "frac_of_hbm": (gather_bytes / avg_s / 1e9 / hbm) if hbm else None}
    probe = (probes or {}).get(f"l2_gather_{bpl}B")
    if probe:
        # the table is L2-resident, so the binding roof is the L2 random-gather rate of loads this size
        g["l2_gather_peak_GBps"] = probe["useful_GBps"]
        g["frac_of_l2_gather"] = gather_bytes / avg_s / 1e9 / probe["useful_GBps"]
        g["corner_loads_per_s"] = corners_per_s
        sectors = measured_l2_sectors_per_sample(cfg)
        if sectors is not None:
            g["l2_sectors_per_sample"] = sectors
            g["l2_sector_rate_frac"] = sectors * cfg.samples / avg_s / probe["loads_per_s"]
    roof["gather"] = g
    return roof


def backward_flop_per_sample(cfg) -> int:
    """Algorithmic FLOPs of one secondary sample's adjoint: the forward recomputed plus, per
    layer, the input gradient and the weight gradient (each as many MACs as the forward)."""
    return 3 * algorithmic_flop_per_sample(cfg)


def time_backward(steps: int, warmup: int, barrier, rays: int = 0, precision: str = "fp32"):
    """One distillation step on the 65,536-ray x 64-direction batch: the student's forward,
    dLoss/dL = (L_s - L_t) / (3 P) against a random-weight teacher of the same architecture
    (teacher seed 1, student seed 2), and rt_backward into zeroed gradient buffers.  precision 'bf16'
    runs the tensor-core forward and adjoint on an FP16 table."""
    import dataclasses
    import torch
    from paper_2409_10327_gb300 import binding
    cfg = dataclasses.replace(scenegen.CONFIGS["grad65k"], precision=precision)
    if rays:
        cfg = dataclasses.replace(cfg, width=rays, height=1)
    gb = {k: torch.from_numpy(v).cuda() for k, v in scenegen.make_gbuffer(cfg.n_pixels, 3).items()}

    def renderer(seed):
        sc = scenegen.make_scene(cfg, seed, bias_scale=0.1)
        r = binding.Renderer(binding.make_config(cfg))
        table = torch.from_numpy(sc.table).cuda()
        r.set_params(table.half() if precision == "bf16" else table, torch.from_numpy(sc.brdf_blob).cuda(),
                     torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(sc.env).cuda())
        return r, sc
    teacher, _ = renderer(1)
    student, sc = renderer(2)
    target = teacher.render_frame(gb)
    g_t = torch.zeros(sc.table.size, device="cuda")
    g_b = torch.zeros(sc.brdf_blob.size, device="cuda")
    g_i = torch.zeros(sc.irt_blob.size, device="cuda")
    out = torch.empty_like(target)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        student.render_frame(gb, out=out)
        d = (out - target) / (3.0 * cfg.n_pixels)
        d[:, 3] = 0.0
        g_t.zero_(), g_b.zero_(), g_i.zero_()
        if ev is not None:
            ev[0].record(stream)
        student.backward(gb, d, g_t, g_b, g_i)
        if ev is not None:
            ev[1].record(stream)
    for _ in range(warmup):
        step()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0.record(stream)
    for k in range(steps):
        step(evs[k])
    t1.record(stream)
    barrier()
    total = t0.elapsed_time(t1)
    bwd = [a.elapsed_time(b) for a, b in evs]
    avg_s = sum(bwd) / len(bwd) / 1e3
    flop = backward_flop_per_sample(cfg) * cfg.samples
    teacher.close()
    student.close()
    if precision == "bf16":
        # the MLP contractions run on the tensor cores: the measured bf16 GEMM rate (burst)
        pk = (json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}).get("bf16_tflops")
        roof = {"bound": "tensor", "peak": pk if pk else 1900.0,
                "peak_source": "of measured (bf16_tflops, burst)" if pk else "of fallback (1.9 PFLOP/s burst)"}
    else:
        roof = {"bound": "alu", "peak": FP32_ALU_PEAK_TFLOPS,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz (nominal FFMA rate)"}
    roof.update({"achieved": flop / avg_s / 1e12, "unit": "TFLOP/s", "frac": flop / avg_s / 1e12 / roof["peak"],
                 "algorithmic_per_launch": flop, "traffic": None})
    return {"workload": f"grad65k: {cfg.n_pixels:,} rays x 64 directions, M=8, L=16, T=2^19, {precision}, L2 distillation",
            "ms_per_step": total / steps, "backward_ms": statistics.median(bwd),
            "value": cfg.samples * steps / (total / 1e3), "unit": UNIT, "steps": steps, "roofline": roof}


def time_distill(steps: int, warmup: int, barrier, rays: int = 2048, K: int = 1024):
    """One online per-head distillation step (Sec. 3.3; supplementary "Training Details": 2,048 rays x
    1,024 stratified directions): directions, the teacher's heads, the student's adjoint, Adam on the
    table and both MLPs, and the rebinding of the student (which synchronises)."""
    import dataclasses
    import torch
    from paper_2409_10327_gb300 import binding, distill
    cfg = dataclasses.replace(scenegen.CONFIGS["grad65k"], width=rays, height=1)

    def renderer(seed):
        sc = scenegen.make_scene(cfg, seed, bias_scale=0.1)
        r = binding.Renderer(binding.make_config(cfg))
        r.set_params(torch.from_numpy(sc.table).cuda(), torch.from_numpy(sc.brdf_blob).cuda(),
                     torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(sc.env).cuda())
        return r, sc
    teacher, _ = renderer(1)
    student, sc = renderer(2)
    d = distill.Distiller(student, teacher, torch.from_numpy(sc.table).cuda(), torch.from_numpy(sc.brdf_blob).cuda(),
                          torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(sc.env).cuda(), K=K)
    gb = scenegen.make_gbuffer(rays, 9)
    pos = torch.from_numpy(gb["pos"]).cuda()
    nrm = torch.from_numpy(gb["normal"]).cuda()
    first = None
    for w in range(warmup):
        loss = d.step(pos, nrm, ray_offset=w * rays)
        if first is None:
            first = float(loss.sum())
    barrier()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        loss = d.step(pos, nrm, ray_offset=(warmup + k) * rays)
    t1.record(stream)
    barrier()
    ms = t0.elapsed_time(t1) / steps
    last = float(loss.sum())
    # the step's parts, each timed alone with CUDA events on the launching stream (own gradient buffers)
    scratch_loss = torch.zeros_like(d.loss)
    scratch_grads = [torch.zeros_like(g) for g in d.grads]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    dirs = student.distill_dirs(rays, K, 0)
    ev[1].record(stream)
    feat = teacher.encode(pos)
    brdf_t = teacher.decode(feat)
    vis_t, depth_t = teacher.trace(feat, dirs)
    ev[2].record(stream)
    student.distill_backward(pos, nrm, dirs, brdf_t, vis_t, depth_t, scratch_loss, *scratch_grads)
    ev[3].record(stream)
    torch.cuda.synchronize()
    parts = {"dirs": ev[0].elapsed_time(ev[1]), "teacher_stage_kernels": ev[1].elapsed_time(ev[2]),
             "distill_backward": ev[2].elapsed_time(ev[3])}
    out = {"workload": f"{rays} rays x {K} stratified directions, L=16, T=2^19, fp32 student and teacher",
           "ms_per_step": ms, "value": rays * K / (ms / 1e3), "unit": "ray-direction pairs/s", "steps": steps,
           "loss_first_last": [first, last], "parts_ms": parts}
    teacher.close()
    student.close()
    return out


def backward_gradient_check(n_rays: int = 256, precision: str = "fp32") -> dict:
    """The FP64 oracle's gradient of the L2 distillation loss on the 256-ray check subset of the
    differentiation workload (timed on the host cores: the backward's CPU baseline), against the
    GPU adjoint's gradient on the same rays: per-tensor ||g - g_ref|| / ||g_ref|| and cosine.  For
    'bf16' both sides use the FP16-rounded table the BF16 context reads."""
    import dataclasses
    import torch
    from oracle import render as orender
    from paper_2409_10327_gb300 import binding
    cfg = dataclasses.replace(scenegen.CONFIGS["grad65k"], precision=precision)
    student = scenegen.make_scene(cfg, 2, bias_scale=0.1)
    teacher = scenegen.make_scene(cfg, 1, bias_scale=0.1)
    if precision == "bf16":
        student.table = student.table.astype(np.float16).astype(np.float32)
    full = scenegen.make_gbuffer(cfg.n_pixels, 3)
    rows = np.sort(scenegen.subset_permutation(cfg.n_pixels, n_rays, seed=0))
    gb = {k: np.ascontiguousarray(v[rows]) for k, v in full.items()}
    opt = orender.Options.from_config(cfg)
    idx = np.arange(n_rays)
    t0 = time.perf_counter()
    t_prm = orender.Params.from_arrays(teacher.table, teacher.brdf, teacher.irt, student.env)
    s_prm = orender.Params.from_arrays(student.table, student.brdf, student.irt, student.env, requires_grad=True)
    with torch.no_grad():
        target = orender.render(gb, t_prm, opt, rows=idx)
        l_s = orender.render(gb, orender.Params.from_arrays(student.table, student.brdf, student.irt, student.env),
                             opt, rows=idx)
    up = orender.upstream_gradient(l_s, target)
    _, g_table, g_brdf, g_irt = orender.distill_gradient(gb, idx, s_prm, torch.from_numpy(target), opt)
    el = time.perf_counter() - t0
    r = binding.Renderer(binding.make_config(cfg))
    table = torch.from_numpy(student.table).cuda()
    r.set_params(table.half() if precision == "bf16" else table, torch.from_numpy(student.brdf_blob).cuda(),
                 torch.from_numpy(student.irt_blob).cuda(), torch.from_numpy(student.env).cuda())
    dgb = {k: torch.from_numpy(v).cuda() for k, v in gb.items()}
    g4 = torch.zeros(n_rays, 4, device="cuda")
    g4[:, :3] = torch.from_numpy(up.astype(np.float32)).cuda()
    gt = torch.zeros(student.table.shape, device="cuda")
    gbw = torch.zeros(student.brdf_blob.size, device="cuda")
    giw = torch.zeros(student.irt_blob.size, device="cuda")
    r.backward(dgb, g4, gt, gbw, giw)
    torch.cuda.synchronize()
    r.close()
    lf = cfg.levels * 2
    parts = {"table": (gt.cpu().numpy(), g_table.numpy())}
    for name, got, ref, ind, outd in (("brdf", gbw.cpu().numpy(), g_brdf.numpy(), lf, 7),
                                      ("irt", giw.cpu().numpy(), g_irt.numpy(), lf + 27, 2)):
        for k, ((wg, bg), (wr, br)) in enumerate(zip(scenegen.unpack_mlp(got, ind, outd),
                                                     scenegen.unpack_mlp(ref, ind, outd))):
            parts[f"{name}.W{k + 1}"] = (wg, wr)
            parts[f"{name}.b{k + 1}"] = (bg, br)
    stats = {}
    for k, (a, b) in parts.items():
        nb = float(np.linalg.norm(b))
        if nb > 0:
            stats[k] = {"relnorm": float(np.linalg.norm(a.ravel() - b.ravel()) / nb),
                        "cosine": float(np.dot(a.ravel(), b.ravel()) / max(np.linalg.norm(a) * nb, 1e-300))}
    return {"rays": n_rays, "precision": precision, "reference": "FP64 oracle autograd gradient (directions held fixed)",
            "per_tensor": stats, "max_relnorm": max(v["relnorm"] for v in stats.values()),
            "cpu_baseline": {"value": n_rays * cfg.n_dirs / el, "unit": "ray-direction samples/s", "seconds": el,
                             "kind": "oracle", "sample": f"{n_rays} rays x {cfg.n_dirs} directions (forward + gradient)"}}


def run_ours(args, cfg):
    import dataclasses
    import torch
    import torch.distributed as dist
    rank, local, world = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2409_10327_gb300.parallel import max_over_ranks

    from paper_2409_10327_gb300 import binding
    main_modes = {"visibility": binding.RT_VIS_HARD if args.visibility == "hard" else binding.RT_VIS_SOFT,
                  "sampling": binding.RT_SAMPLE_MIS if args.sampling == "mis" else binding.RT_SAMPLE_COSINE}
    renderers, gbs = _setup(cfg, rank, **main_modes)
    if cfg.precision == "bf16":
        for r in renderers:   # the frame kernel's launch shape (single light)
            r.set_launch_shape(r.launch_shape()[0], args.warpgroups)
            r.set_tile_shape(args.dirs_per_tile)
    out = torch.empty(cfg.n_pixels, 4, device="cuda")
    total_ms, launch_ms, clk = _time_frames(renderers, gbs, out, args.steps, args.warmup, barrier,
                                            ClockSampler(local))
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = world * cfg.samples * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host G-buffer -> device, render, radiance -> host
    host_gb = [{k: v.cpu().pin_memory() for k, v in g.items()} for g in gbs]
    host_out = torch.empty(cfg.n_pixels, 4).pin_memory()
    staging = {k: torch.empty_like(v) for k, v in gbs[0].items()}
    n = len(renderers)
    for w in range(max(1, args.warmup)):
        renderers[w % n].render_frame_host(host_gb[w % n], host_out, staging, out)
    barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        renderers[k % n].render_frame_host(host_gb[k % n], host_out, staging, out)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    h2d = sum(v.numel() * v.element_size() for v in host_gb[0].values())
    d2h = host_out.numel() * host_out.element_size()
    # scene 0's frame in the timed launch configuration, kept for the parity block
    frames = {cfg.precision: renderers[0].render_frame(gbs[0]).cpu().numpy()[:, :3]}
    # live ceilings for the rooflines: L2 random-gather rates and FP32 FMA throughput
    probes = measure_probe_peaks()

    # the spatial SVGF denoiser (Sec. 4.1) on the rendered frame; depth = distance to a camera at (0, 0, -3)
    den = None
    if not args.no_denoise and cfg.width * cfg.height == cfg.n_pixels:
        from paper_2409_10327_gb300 import binding
        depth = (gbs[0]["pos"][:, :3] - torch.tensor([0.0, 0.0, -3.0], device="cuda")).norm(dim=1).contiguous()
        d_out = torch.empty_like(out)
        d_work = torch.empty_like(out)
        for _ in range(3):
            binding.denoise(out, depth, gbs[0]["normal"], cfg.width, cfg.height, out=d_out, work=d_work)
        reps = 20
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(reps):
            binding.denoise(out, depth, gbs[0]["normal"], cfg.width, cfg.height, out=d_out, work=d_work)
        d1.record(stream)
        barrier()
        den = {"ms": d0.elapsed_time(d1) / reps, "iterations": 5, "launches": 6,
               "image": f"{cfg.width}x{cfg.height}", "note": "spatial SVGF, L2-resident image, CUDA events over 20 runs"}
    for r in renderers:
        r.close()
    del renderers, gbs, host_gb, staging

    # the other precision of the same workload, for the BF16-vs-FP32 comparison
    compare = None
    if not args.no_compare:
        other = dataclasses.replace(cfg, precision="fp32" if cfg.precision == "bf16" else "bf16")
        rs, gs = _setup(other, rank)
        steps = max(3, args.steps // 4)
        o_total, o_launch, _ = _time_frames(rs, gs, out, steps, args.warmup, barrier)
        o_total = max_over_ranks(o_total)
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        compare = {"precision": other.precision, "value": world * other.samples * steps / (o_total / 1e3),
                   "unit": UNIT, "ms_per_frame": o_total / steps, "steps": steps,
                   "roofline": _roofline(other, o_launch, peaks, probes)}
        if args.visibility == "soft" and args.sampling == "cosine":
            frames[other.precision] = rs[0].render_frame(gs[0]).cpu().numpy()[:, :3]
        for r in rs:
            r.close()

    # the paper's inference mode: hard visibility, only shadow directions bounce (compacted in the kernel)
    hard = None
    if not args.no_hard and cfg.precision == "bf16":
        from paper_2409_10327_gb300 import binding
        rs, gs = _setup(cfg, rank, visibility=binding.RT_VIS_HARD)
        steps = max(3, args.steps // 4)
        h_total, h_launch, _ = _time_frames(rs, gs, out, steps, args.warmup, barrier)
        h_total = max_over_ranks(h_total)
        # share of primary directions that are shadow rays (v = 0), from the stage kernels on 16,384 pixels
        sub = {k: v[:16384].contiguous() for k, v in gs[0].items()}
        dirs = rs[0].sample(sub["normal"], 0)
        vis, _ = rs[0].trace(rs[0].encode(sub["pos"]), dirs)
        shadow = float((vis <= 0.5).float().mean().item())
        hard = {"visibility": "hard", "value": world * cfg.samples * steps / (h_total / 1e3), "unit": UNIT,
                "ms_per_frame": h_total / steps, "steps": steps, "shadow_fraction": shadow,
                "kernel_ms": {"min": min(h_launch), "median": statistics.median(h_launch)},
                "note": "v, v' = 1[sigmoid(z0) > 0.5] (Sec. 3.2 overview); shadow rows are queued per warpgroup and "
                        "run in compacted 128-row tiles; samples/s counts all P*N primary directions"}
        for r in rs:
            r.close()

    # MIS primary directions (light + GGX visible normals, balance heuristic; Sec. 4.1)
    mis_line = None
    if not args.no_mis:
        from paper_2409_10327_gb300 import binding
        rs, gs = _setup(cfg, rank, sampling=binding.RT_SAMPLE_MIS)
        steps = max(3, args.steps // 4)
        m_total, m_launch, _ = _time_frames(rs, gs, out, steps, args.warmup, barrier)
        m_total = max_over_ranks(m_total)
        mis_line = {"sampling": "mis", "value": world * cfg.samples * steps / (m_total / 1e3), "unit": UNIT,
                    "ms_per_frame": m_total / steps, "steps": steps,
                    "kernel_ms": {"min": min(m_launch), "median": statistics.median(m_launch)}}
        for r in rs:
            r.close()

    # row a10: one distillation step (forward + hand-written adjoint)
    bwd = None if args.no_backward else time_backward(max(3, args.steps // 4), args.warmup, barrier)
    dst = None if args.no_distill else time_distill(max(3, args.steps // 4), args.warmup, barrier)
    if bwd is not None:
        r = bwd["roofline"]
        r["peak"], r["frac"] = probes["ffma_tflops"], r["achieved"] / probes["ffma_tflops"]
        r["peak_source"] = "of measured (rt_probe_ffma, burst, same run)"
        # the BF16 tensor-core adjoint of the same batch
        bwd["bf16"] = time_backward(max(3, args.steps // 4), args.warmup, barrier, precision="bf16")
    # batched serving (16 views x 8 lights at 1920x1080, one CUDA graph per batch)
    srv = None if args.no_serve else time_serve(args.views, args.lights, args.serve_steps, 1, rank, local)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    cpu = None
    parity = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle timed on the host cores; the pixels it renders (a seeded sample of scene 0, the
        # first timed scene) are also the reference of the parity block
        rate, done, el, cores, rows, ref = cpu_oracle_rate(cfg, args.cpu_seconds, keep=True)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
               "sample": f"{done} pixels ({done * cfg.n_dirs} secondary samples) of one 800x800 frame, {el:.1f} s"}
        r1, d1, e1, _ = cpu_oracle_rate(cfg, max(1.0, args.cpu_seconds / 3), threads=1)
        cpu["single_core"] = {"value": r1, "unit": UNIT, "cores": 1,
                              "sample": f"{d1} pixels of the same frame, {e1:.1f} s"}
        if args.visibility == "soft" and args.sampling == "cosine" and cfg.n_pixels == 800 * 800:
            parity = {"reference": f"FP64 oracle, the same {done} seeded pixels of scene 0 as cpu_baseline",
                      **{prec: parity_stats(fr[rows], ref, prec, golden_frame_stats(cfg, 0) if prec == "bf16" else None)
                         for prec, fr in frames.items()}}
        if bwd is not None and not args.no_grad_check:
            bwd["gradient_check"] = backward_gradient_check()
            if "bf16" in bwd:
                bwd["bf16"]["gradient_check"] = backward_gradient_check(precision="bf16")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "ms_per_frame": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if cfg.precision == "fp32" else "bf16",
            "data": "synthetic",
            "config": {"workload": workload_name(cfg), "l2": L2_NOTE, "scenes_per_rank": 4,
                       "visibility": args.visibility, "sampling": args.sampling,
                       "warpgroups": args.warpgroups, "dirs_per_tile": args.dirs_per_tile},
            "roofline": _roofline(cfg, launch_ms, peaks, probes), "cpu_baseline": cpu, "parity": parity,
            "probes": probes, "serve": srv,
            "e2e": {"value": world * cfg.samples * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps},
            "gpu_launches": args.steps, "clocks": clk, "compare": compare, "hard_visibility": hard, "mis": mis_line, "denoise": den, "backward": bwd, "distill": dst,
            "launch_ms": {"min": min(launch_ms), "median": statistics.median(launch_ms), "max": max(launch_ms),
                          "all": [round(x, 3) for x in launch_ms]}}
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def time_serve(views: int, lights: int, steps: int, warmup: int, rank: int = 0, local: int = 0) -> dict:
    """Batched serving: V views x E lights at 1920x1080 (N=256, L=16, T=2^20, BF16), one CUDA-graph launch
    per batch after rt_tune picked the launch shape; per-view latencies from events inside the graph."""
    import torch
    from paper_2409_10327_gb300 import binding, serve
    cfg = scenegen.CONFIGS["serve1080"]
    V, E = views, lights
    sc = scenegen.make_scene(cfg, 0)
    r = binding.Renderer(binding.make_config(cfg))
    r.set_params(torch.from_numpy(sc.table).cuda().half(), torch.from_numpy(sc.brdf_blob).cuda(),
                 torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(sc.env).cuda())
    gbs = [{k: torch.from_numpy(v).cuda() for k, v in scenegen.make_gbuffer(cfg.n_pixels, rank * V + v).items()}
           for v in range(V)]
    envs = torch.from_numpy(np.stack([scenegen.make_env(cfg.env_h, cfg.env_w, 100 + e) for e in range(E)])).cuda()
    srv = serve.BatchedServer(r, gbs, envs)
    tune_pixels = cfg.n_pixels // 8            # the search runs on the first eighth of view 0
    tuned_ms = srv.tune(pixels=tune_pixels)
    shape = r.launch_shape()
    dpt = r.tile_shape()
    srv.capture()
    for _ in range(warmup):
        srv.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    lats = []
    t0.record()
    for _ in range(steps):
        srv.replay()
        t1.record()
        torch.cuda.synchronize()
        lats += srv.view_latencies_ms()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    frames = V * E * steps
    samples = cfg.samples * V * steps          # secondary samples of the geometry passes
    lat = np.array(lats)
    out = {"workload": f"serve1080: {V} views x {E} env maps, 1920x1080, N=256, M=8, L=16, T=2^20, bf16",
           "value": samples / (total_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_batch": total_ms / steps, "frames_per_s": frames / (total_ms / 1e3),
           "lit_samples_per_s": samples * E / (total_ms / 1e3),
           "view_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "views": int(lat.size)},
           "frame_latency_ms_amortised": {"p50": float(np.percentile(lat, 50)) / E,
                                          "p99": float(np.percentile(lat, 99)) / E},
           "graph": "one CUDA graph per batch (one rt_render_frame_multi per view)",
           "launch_shape": {"lights_per_launch": shape[0], "warpgroups": shape[1], "dirs_per_tile": dpt,
                            "tuned_ms": tuned_ms, "tuned_on_pixels": tune_pixels},
           "gpu_launches": steps * V * max(1, E // shape[0]), "clocks": clk}
    del srv, gbs, envs
    r.close()
    return out


def run_serve(args):
    """Batched serving as its own bench line (--mode serve)."""
    import torch
    rank, local, world = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    res = time_serve(args.views, args.lights, args.steps, args.warmup, rank, local)
    if rank != 0:
        return
    line = {"metric": "batched serving: secondary samples/s and frame latency (16 views x 8 env maps, 1920x1080)",
            "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": res["workload"], "graph": res["graph"], "launch_shape": res["launch_shape"]},
            "frames_per_s": res["frames_per_s"], "lit_samples_per_s": res["lit_samples_per_s"],
            "view_latency_ms": res["view_latency_ms"], "frame_latency_ms_amortised": res["frame_latency_ms_amortised"],
            "gpu_launches": res["gpu_launches"], "clocks": res["clocks"]}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="bf16")
    ap.add_argument("--no-compare", action="store_true", help="skip the other precision's comparison timing")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="frame800")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hard", action="store_true", help="skip the hard-visibility timing")
    ap.add_argument("--no-denoise", action="store_true", help="skip the denoiser timing")
    ap.add_argument("--no-backward", action="store_true", help="skip the backward (distillation step) timing")
    ap.add_argument("--no-mis", action="store_true", help="skip the MIS-sampling timing")
    ap.add_argument("--no-distill", action="store_true", help="skip the distillation-step timing")
    ap.add_argument("--mode", choices=["frame", "serve", "backward", "distill"], default="frame")
    ap.add_argument("--visibility", choices=["soft", "hard"], default="soft",
                    help="visibility of the main frame leg (the headline is soft)")
    ap.add_argument("--sampling", choices=["cosine", "mis"], default="cosine",
                    help="primary directions of the main frame leg (the headline is cosine)")
    ap.add_argument("--no-serve", action="store_true", help="skip the batched-serving leg")
    ap.add_argument("--serve-steps", type=int, default=2, help="timed batches of the serving leg")
    ap.add_argument("--no-grad-check", action="store_true",
                    help="skip the backward's FP64 gradient check (part of the cpu_baseline leg)")
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--lights", type=int, default=8)
    ap.add_argument("--warpgroups", type=int, choices=[2, 3, 4], default=4,
                    help="BF16 frame kernel: warpgroups per CTA")
    ap.add_argument("--dirs-per-tile", type=int, choices=[32, 64, 128], default=128,
                    help="BF16 frame kernel: directions of a pixel per 128-row tile (rt_set_tile_shape)")
    ap.add_argument("--pixels", type=int, default=0,
                    help="render only the first P pixel rows of each frame (a smaller case for profilers)")
    args = ap.parse_args()
    import dataclasses
    cfg = dataclasses.replace(scenegen.CONFIGS[args.config], precision=args.precision)
    if args.pixels:
        cfg = dataclasses.replace(cfg, name=cfg.name + f"[{args.pixels} px]", width=args.pixels, height=1)
    if args.impl == "reference":
        run_reference(args, cfg)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "backward":
        import torch
        torch.cuda.set_device(0)
        line = time_backward(args.steps, args.warmup, torch.cuda.synchronize, rays=args.pixels,
                             precision=args.precision)
        print(json.dumps({"metric": "backward (distillation step) secondary samples/s", "n_gpus": 1,
                          "warmup": args.warmup, "dtype": "bf16" if args.precision == "bf16" else "f32",
                          "data": "synthetic", **line}))
    elif args.mode == "distill":
        import torch
        torch.cuda.set_device(0)
        line = time_distill(args.steps, args.warmup, torch.cuda.synchronize, rays=args.pixels or 2048)
        print(json.dumps({"metric": "per-head distillation step, ray-direction pairs/s", "n_gpus": 1,
                          "warmup": args.warmup, "dtype": "f32", "data": "synthetic", **line}))
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
