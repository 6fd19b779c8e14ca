"""Pyramid-WFS frames/s at ELT scale on GB300, with the roofline of the
dominant kernel and the FP64 oracle timed on the host cores as a baseline.

One step = one frame of the 39 m single-pyramid system (480 px pupil, 960^2
FFT, 48 modulation points, 96 x 96 subapertures, 35 layers, 4000-mode MVM):
layer extraction -> modulated pyramid image -> slopes -> reconstructor,
through the C ABI of libspecula_gb300.  Inputs are resident in HBM before
the timed region; L2 is flushed (a 256 MB write) between timed frames, outside
the frame's CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl specula|reference]

Under torchrun each rank runs an independent replica (its own seeded
atmosphere); value = frames of all ranks / max over ranks of the timed span.
"""
import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

# the oracle baselines are timed single-threaded per process (BLAS included)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pwfs39m"
METRIC = "pyramid-WFS frames/s (ELT scale) + roofline %, mixed vs plain FP32 at stated err"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x clock
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def fft_flops(n):
    return 5.0 * n * math.log2(n)


def kernel_flops(wl):
    """Algorithmic FLOPs per frame of each pyramid pass (benchFFT convention
    5 N log2 N per N-point transform, pruned inputs counted as full
    transforms; element-wise work not counted).  Two-pass form: the row
    filter transforms the n_pix pupil rows forward and back once per distinct
    cosine of the modulation angles (n_mod / 2 + 1 of them: points m and
    n_mod - m share the row filter), the column filter all N columns forward
    and back for every modulation point; three-pass form: n_pix forward rows,
    N columns forward and back, N inverse rows, per modulation point."""
    s = wl.sensors[0]
    n = s.pupil.n_pix
    N = s.pwfs.pad * n
    n_mod = s.pwfs.n_mod
    nc = n_mod // 2 + 1
    return {"pwfs_rowfilt": nc * 2 * n * fft_flops(N),
            "pwfs_colfilt_bin": n_mod * 2 * N * fft_flops(N),
            "pwfs_rows_fwd": n_mod * n * fft_flops(N),
            "pwfs_cols": n_mod * 2 * N * fft_flops(N),
            "pwfs_rows_inv": n_mod * N * fft_flops(N)}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 20 ms, started before
    the timed region (the first sample is awaited) and kept for the samples
    whose timestamps fall inside it (mark_start / mark_end)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None
        self._thread = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.lines.append(line.strip())

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self
        self._thread = threading.Thread(target=self._read, daemon=True)
        self._thread.start()
        end = time.time() + 3.0
        while not self.lines and time.time() < end and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self._thread is not None:
            self._thread.join(timeout=2)

    def summary(self):
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in list(self.lines):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[1]), float(f[2]),
                             {n for k, n in enumerate(names) if f[4 + k].lower().startswith("active")}))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None
                  and self.t0 - 0.02 <= r[0] <= self.t1 + 0.02]
        use = inside or rows
        reasons = set().union(*[r[3] for r in use])
        return {"sm_mhz": statistics.median(r[1] for r in use),
                "sm_max_mhz": max(r[2] for r in use), "reasons": sorted(reasons),
                "samples": len(use), "samples_in_timed_region": len(inside),
                "interval_ms": 20}


def read_traffic():
    """dram bytes per launch of the dominant kernel from the committed ncu
    summary (a line 'traffic_bytes_per_launch <kernel> <workload> <bytes>')."""
    out = {}
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return out
    for f in os.listdir(d):
        if not f.endswith((".txt", ".md")):
            continue
        for line in open(os.path.join(d, f)):
            m = re.match(r"\s*traffic_bytes_per_launch\s+(\S+)\s+(\S+)\s+([0-9.eE+]+)", line)
            if m:
                out[(m.group(1), m.group(2))] = float(m.group(3))
    return out


def aggregate_ranks(total_ms, steps, ws, dist=None, device="cpu"):
    """(ms per step, whole-job frames/s): the slowest rank's timed span over
    the frames all ranks processed (each rank runs its own replica)."""
    if dist is not None and ws > 1:
        import torch
        t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms / steps, ws * steps / (total_ms / 1e3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU oracle

def _mod_points_sum(E, ms, mask, n, mod_amp, n_mod):
    """Summed |IDFT(mask DFT(pad(E tilt_m)))|^2 over the modulation points ms:
    the oracle's pyramid steps, point by point."""
    from oracle import geometry
    from oracle.dft import centred_coords, centred_dft2, centred_idft2
    N = 2 * n
    off = (N - n) // 2
    x = centred_coords(n)
    cs, sn = geometry.mod_angles(n_mod)
    I = np.zeros((N, N))
    for m in ms:
        tilt = np.exp(2j * np.pi * mod_amp * (x[None, :] * cs[m] + x[:, None] * sn[m]) / n)
        P = np.zeros((N, N), dtype=np.complex128)
        P[off:off + n, off:off + n] = E * tilt
        I += np.abs(centred_idft2(centred_dft2(P) * mask)) ** 2
    return I


_POOL = {}


def _pool_init(mask, n, mod_amp, n_mod):
    _POOL.update(mask=mask, n=n, mod_amp=mod_amp, n_mod=n_mod)


def _pool_mod_points(args):
    E, ms = args
    return _mod_points_sum(E, ms, _POOL["mask"], _POOL["n"], _POOL["mod_amp"], _POOL["n_mod"])


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class OracleFrame:
    """The FP64 oracle on whole frames of the ELT workload: all 35 layers
    extracted, all 48 modulation points imaged, binning, slopes and the
    4000-mode MVM, nothing scaled.  Two oracle screens are cycled over the 35
    layers (the timing does not depend on screen values).  frame() runs in
    this process, or with the modulation points spread over a pool of
    spawned processes (one per host core; every process single-threaded)."""

    def __init__(self):
        import synth
        from oracle import geometry, pyramid, screens
        wl = synth.workload(WORKLOAD)
        s = wl.sensors[0]
        self.wl, self.s, self.n = wl, s, s.pupil.n_pix
        base = [screens.fft_screen(l.side, l.pitch_m, l.r0_m, l.L0_m,
                                   synth.screen_noise(l.seed, l.side),
                                   synth.subharmonic_noise(l.seed)).astype(np.float32)
                for l in wl.layers[:2]]
        self.scr = [base[k % 2].astype(np.float64) for k in range(len(wl.layers))]
        self.amp = geometry.pupil_mask(self.n, s.pupil.obsc_frac).astype(np.float64)
        self.valid = geometry.valid_subaps(self.amp.astype(np.uint8), s.pwfs.n_sub)
        self.n_slopes = 2 * len(self.valid)
        self.R = synth.normal_draws(7, (wl.n_modes, self.n_slopes)) / np.sqrt(self.n_slopes)
        self.mask = pyramid.pyramid_mask(2 * self.n, self.n)
        self.pool = None
        self.cores = 1

    def open_pool(self):
        import multiprocessing as mp
        self.cores = host_cores()
        s = self.s
        self.pool = mp.get_context("spawn").Pool(
            self.cores, initializer=_pool_init,
            initargs=(self.mask, self.n, s.pwfs.mod_amp, s.pwfs.n_mod))
        self.chunks = [list(range(k, s.pwfs.n_mod, self.cores))
                       for k in range(min(self.cores, s.pwfs.n_mod))]

    def close_pool(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def describe(self, pooled):
        where = (f"the {self.s.pwfs.n_mod} modulation points spread over {self.cores} spawned "
                 f"single-threaded processes, the rest in the parent"
                 if pooled else "all in one single-threaded process")
        return (f"whole {WORKLOAD} frames (35-layer extraction, {self.s.pwfs.n_mod} modulation "
                f"points, binning, slopes, {self.wl.n_modes}x{self.n_slopes} MVM), {where}; "
                f"FP64 NumPy oracle, nothing scaled")

    def frame(self, t=0.001):
        """Seconds of one whole frame."""
        from oracle import atmo, pyramid, recon, slopes
        s, n = self.s, self.n
        t0 = time.perf_counter()
        phi = atmo.atmo_extract(self.scr, self.wl.layers, s.source, n, s.pupil.pitch_m, t)
        E = self.amp * np.exp(1j * phi)
        if self.pool is None:
            I = _mod_points_sum(E, range(s.pwfs.n_mod), self.mask, n, s.pwfs.mod_amp,
                                s.pwfs.n_mod)
        else:
            parts = self.pool.map_async(_pool_mod_points,
                                        [(E, c) for c in self.chunks]).get(timeout=600)
            I = parts[0]
            for q in parts[1:]:
                I = I + q
        det = pyramid.bin_image(I / s.pwfs.n_mod, n // s.pwfs.n_sub)
        sl = slopes.pyr_slopes(det, s.pwfs.n_sub, self.valid)
        recon.mvm(self.R, sl)
        return time.perf_counter() - t0


def cpu_baselines(n_pooled=3):
    """The oracle's frame rate on the host: whole frames with the points over
    all cores (1 warm-up, n_pooled timed, mean), and one whole frame in one
    process."""
    sample = OracleFrame()
    sample.open_pool()
    try:
        sample.frame(0.001)
        tp = [sample.frame(0.001 * (k + 2)) for k in range(n_pooled)]
    finally:
        sample.close_pool()
    pooled = {"value": n_pooled / sum(tp), "unit": "frames/s", "cores": sample.cores,
              "kind": "oracle",
              "sample": sample.describe(True) + f"; mean of {n_pooled} after one warm-up"}
    t1 = sample.frame(0.001)
    single = {"value": 1.0 / t1, "unit": "frames/s", "cores": 1, "kind": "oracle",
              "sample": sample.describe(False) + "; one frame"}
    return pooled, single


def reference_leg(args, ws, rank):
    """The reference arm: the oracle (the paper ships no program to run) on
    whole frames, each step one frame with the points over all host cores."""
    if rank != 0:
        return
    sample = OracleFrame()
    sample.open_pool()
    try:
        times = []
        for k in range(args.warmup + args.steps):
            t = sample.frame(0.001 * (k + 1))
            if k >= args.warmup:
                times.append(t)
    finally:
        sample.close_pool()
    per = sum(times) / len(times)
    value = 1.0 / per
    desc = sample.describe(True)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": sample.cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ learned

def learned_leg(ctx, n_train=200000, n_test=5000, epochs=12):
    """The learned-reconstructor configuration (8 m pyramid geometry, 2512 ->
    1024 -> 1024 -> 500): pairs generated by the GPU simulator, network
    trained by the library's kernels, residual compared with the calibrated
    linear MVM on held-out frames (disjoint sample indices)."""
    import torch
    import synth
    from paper_2602_06688_gb300.learned import LearnedPipeline
    wl = synth.workload("learned8m")
    t0 = time.perf_counter()
    p = LearnedPipeline(ctx, wl)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    Xtr, Ttr = p.make_pairs(n_train, 0)
    Xte, Tte = p.make_pairs(n_test, 10 ** 6)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    hist = p.fit(Xtr, Ttr, epochs=epochs)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    res = p.evaluate(Xte, Tte)
    # batched inference throughput of the reconstructors on the test set
    # (each warmed once: the split-bf16 product sizes its workspace on its
    # first call at a batch size)
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    mlp_ms = timed(lambda: p.predict(Xte))
    lin_ms = timed(lambda: p.linear(Xte))
    split_ms = timed(lambda: p.linear(Xte, split_bf16=True))
    return {"workload": "learned8m", "net": "2512-1024-1024-500 GELU (bf16 tcgen05, FP32 acc)",
            "train_pairs": n_train, "test_pairs": n_test, "epochs": epochs, "batch": 256,
            "r0_range_m": [0.06, 0.20],
            "residual_rms_rad": {"linear_mvm": res["linear"],
                                 "linear_mvm_split_bf16": res["linear_split_bf16"],
                                 "learned": res["learned"], "true_modes_rms": res["labels"]},
            "learned_gain": res["linear"] / res["learned"],
            "calibration_s": t1 - t0, "pair_generation_s": t2 - t1, "training_s": t3 - t2,
            "final_train_loss": hist[-1],
            "inference_frames_per_s": {
                "learned_batched": n_test / (mlp_ms / 1e3),
                "linear_batched": n_test / (split_ms / 1e3),
                "linear_batched_path": "split-bf16 R on the tensor cores (one 3-term tcgen05 "
                                       "GEMM over the slopes' bf16 halves)",
                "linear_batched_fp32_cuda_cores": n_test / (lin_ms / 1e3)}}


def closed_loop_leg(ctx, steps=400, settle=150):
    """The closed loop on the 8 m pyramid (160 px pupil, 24 points, three
    layers, 500 calibrated Zernike modes, integrator gain 0.4): one step
    (extraction, mirror shape, residual statistics, pyramid, slopes, MVM,
    integrator update) per replay of a CUDA graph, steps back to back as a
    running loop.  Reports the step rate and, averaged after `settle` steps,
    the residual RMS over the whole pupil (edge pixels outside every valid
    subaperture included: the sensor never sees them) and the H-band
    (1650 nm) Strehl ratio, with the leaky integrator (leak 0.01, the
    default), without leak, and open (gain 0), over the same atmosphere; and
    the largest command every 100 steps (bounded commands: no mode drifts)."""
    import torch
    import synth
    import paper_2602_06688_gb300 as sp
    from paper_2602_06688_gb300.loop import ClosedLoop, LoopNetwork
    st = torch.cuda.Stream()
    out = {"workload": "pwfs8m", "gain": 0.4, "sci_wavelength_nm": 1650.0}
    cl = ClosedLoop(ctx, synth.workload("pwfs8m"), gain=0.4)
    # pixels the sensor sees: inside a valid subaperture and the pupil
    fr = cl.fr
    g = synth.workload("pwfs8m").sensors[0].pwfs
    b = fr.n_pix // g.n_sub
    seen = np.zeros((fr.n_pix, fr.n_pix), dtype=bool)
    for v in sp.specula_valid_subaps_host(fr.pupil, g.n_sub):
        a, c = divmod(int(v), g.n_sub)
        seen[a * b:(a + 1) * b, c * b:(c + 1) * b] = True
    seen &= fr.amp.cpu().numpy() > 0
    seen_t = torch.tensor(seen, device="cuda")
    n_seen = float(seen.sum())
    nets = {}
    for label, gain, leak in (("closed", 0.4, 0.01), ("closed_no_leak", 0.4, 0.0),
                              ("open", 0.0, 0.0), ("closed_learned_correction", 0.4, 0.01),
                              ("closed_learned_direct", 0.4, 0.01)):
        cl.gain, cl.leak = gain, leak
        cl.net = None
        if label.startswith("closed_learned"):
            net = LoopNetwork(cl, residual=label.endswith("correction"))
            nets[label] = net.train()
            cl.net = net
        cl.reset()
        cl.close()
        cl.capture(st)
        hist = torch.zeros(steps, 2, dtype=torch.float64, device="cuda")
        cmax = torch.zeros(steps, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            e0.record()
            for k in range(steps):
                cl.replay(k * cl.fr.dt, st)
                hist[k].copy_(cl.stats)
            e1.record()
        torch.cuda.synchronize()
        # the command trajectory and the residual over the seen pixels, from a
        # second (untimed) run of the same steps
        cl.reset()
        seen_ms = torch.zeros(steps, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(st):
            for k in range(steps):
                cl.replay(k * cl.fr.dt, st)
                cmax[k] = cl.cmd.abs().max()
                r = cl.resid.double()[seen_t]
                seen_ms[k] = ((r - r.mean()) ** 2).sum() / n_seen
        torch.cuda.synchronize()
        h = hist.cpu().numpy()[settle:]
        c = cmax.cpu().numpy()
        out[label] = {"leak": leak, "strehl": float(h[:, 1].mean()),
                      "resid_rms_rad_wfs_full_pupil": float(h[:, 0].mean()),
                      "resid_rms_rad_wfs_seen_pixels":
                          float(np.sqrt(seen_ms.cpu().numpy()[settle:]).mean()),
                      "max_abs_cmd_every_100": [float(c[k]) for k in range(99, steps, 100)]}
        if label in nets:
            out[label]["training"] = nets[label]
        if label == "closed":
            ms = e0.elapsed_time(e1)
            out.update({"frames_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps,
                        "n_modes": cl.n_modes, "rank": cl.rank,
                        "graph_kernels": cl.graph.kernel_count(),
                        "timing": "back-to-back steps, each with a 16-byte copy of its "
                                  "statistics; L2 not flushed"})
    cl.net = None
    cl.close()
    out["learned_note"] = ("closed_learned_correction: m = R s + f(s), f the 2512-1024-1024-500 "
                           "network trained on synthetic modal phases with 16x the loop's own "
                           "residual spectrum (targets: what R s misses); closed_learned_direct: "
                           "m = f(s) alone, same training phases")
    return out


def fma_peaks_leg(ctx):
    """Measured fused multiply-add rates (the library's probe kernel, 8 CTAs
    of 256 threads per SM, 8 independent chains per thread), best of 3
    event-timed launches after one warm-up: the check on the derived FP32
    peak, and the float64 rate of the set-up paths."""
    import torch
    import paper_2602_06688_gb300 as sp
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n_ctas = 8 * n_sm
    out = {}
    for bits, n_iter, dt in ((32, 20000, torch.float32), (64, 1000, torch.float64)):
        sink = torch.empty(n_ctas * 256, dtype=dt, device="cuda")
        sp.specula_fma_probe(ctx, bits, n_ctas, n_iter, sink)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sp.specula_fma_probe(ctx, bits, n_ctas, n_iter, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        flops = 2.0 * 8 * n_iter * 256 * n_ctas
        out["fp%d_fma_tflops" % bits] = flops / (best / 1e3) / 1e12
        assert bool(torch.isfinite(sink).all())
    out["sms"] = n_sm
    return out


def infinite_leg(ctx, st, flush, steps):
    """The 8 m pyramid frame on infinite screens: 256 px rings, two stencil
    lines; before each frame the host picks the lines the footprints need and
    the line kernel grows them, then the captured frame runs.  Timed from
    10 s of flow on (every layer growing), growth inside the events."""
    import torch
    import synth
    import paper_2602_06688_gb300 as sp
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload("pwfs8m")
    fi = PwfsFrame(ctx, wl, infinite=dict(side=256, n_st=2, seed=4))
    g = fi.capture(st)
    t0 = 10.0
    with torch.cuda.stream(st):
        for k in range(5):
            fi.replay(t0 + k * wl.dt_s, st)
    torch.cuda.synchronize()
    n0 = fi.inf.lines_grown
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    launches = 0
    with torch.cuda.stream(st):
        for k in range(steps):
            flush.zero_()
            fi.t_dev.fill_(t0 + (k + 5) * wl.dt_s)
            ev[k][0].record(st)
            launches += fi.inf.advance(t0 + (k + 5) * wl.dt_s, stream=st)
            g.launch(st)
            ev[k][1].record(st)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    lines = fi.inf.lines_grown - n0
    # the line kernel alone: one line in each of the three rings per call,
    # 20 calls captured in a graph (device time without host issue)
    A, B, _ = next(iter(fi.inf.ops.values()))
    tasks = [(fi.screens[i], A, B, 1.0, 0, 1, 100 + i, 10 ** 6) for i in range(3)]
    torch.cuda.synchronize()
    sp.specula_graph_begin(ctx, st)
    try:
        for k in range(20):
            sp.specula_infscreen_lines(ctx, 256, 2, tasks, seed=9, stream=st)
    finally:
        gl = sp.specula_graph_end(ctx, st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        for k in range(3):
            gl.launch(st)
        e0.record(st)
        for k in range(10):
            gl.launch(st)
        e1.record(st)
    torch.cuda.synchronize()
    gl.close()
    g.close()
    return {"config": "pwfs8m frame (3 layers) on 256 px infinite rings, 2 stencil lines, "
                      "from t = 10 s",
            "frames_per_s": steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
            "lines_per_frame": lines / steps, "line_calls_per_frame": launches / steps,
            "line_call_us_3_rings": e0.elapsed_time(e1) / 200 * 1e3,
            "note": "the periodic pwfs8m frame (1024 px screens) is systems.pwfs8m"}


def systems_leg(ctx, steps=50):
    """The other systems of the paper's scale list, one frame per step from a
    CUDA graph, L2 flushed between frames outside the events: the 8 m single
    pyramid (FP32 / split-BF16 / BF16 reconstructor) and the 39 m
    multi-sensor system (6 laser-star SH + 3 pyramids + MVM) in one
    persistent launch against the same frame as per-sensor launches."""
    import torch
    import synth
    import paper_2602_06688_gb300 as sp
    from paper_2602_06688_gb300.frame import PwfsFrame
    from paper_2602_06688_gb300.system import System
    st = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def time_graph(g, set_t, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        with torch.cuda.stream(st):
            for k in range(n):
                flush.zero_()
                set_t(k)
                ev[k][0].record(st)
                g.launch(st)
                ev[k][1].record(st)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    out = {}
    wl = synth.workload("pwfs8m")
    fr = PwfsFrame(ctx, wl, autotune=True)
    res = {}
    for name, prec in (("fp32", sp.PREC_FP32), ("bf16x2", sp.PREC_BF16X2), ("bf16", sp.PREC_BF16)):
        fr.set_precision(prec)
        g = fr.capture(st)
        time_graph(g, lambda k: fr.t_dev.fill_(wl.dt_s * k), 5)
        ms = time_graph(g, lambda k: fr.t_dev.fill_(wl.dt_s * k), steps)
        res[name] = {"frames_per_s": steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps}
        g.close()
    # the batched form: B consecutive open-loop frames per graph launch
    def batched(name, B):
        w = synth.workload(name)
        fb = PwfsFrame(ctx, w, autotune=True, batch=B)
        g = fb.capture(st)
        ar = torch.arange(B, dtype=torch.float64, device="cuda") * w.dt_s
        set_t = lambda k: fb.t_dev.copy_(ar + k * B * w.dt_s)
        time_graph(g, set_t, 5)
        ms = time_graph(g, set_t, steps)
        g.close()
        res = {"batch": B, "frames_per_s": B * steps / (sum(ms) / 1e3),
               "ms_per_step": sum(ms) / steps,
               "tiles": {"chunk": fb.tiles[0], "ka": fb.tiles[1], "passes": fb.tiles[2]}}
        del fb
        torch.cuda.empty_cache()
        return res

    out["pwfs8m"] = {"config": "8.4 m, 160 px pupil, 320^2 FFT, 24 mod points, 40x40 subaps, "
                               "3 layers, 500 modes",
                      "tiles": {"chunk": fr.tiles[0], "ka": fr.tiles[1], "passes": fr.tiles[2]},
                      "recon_variants": res, "batched_fp32": batched("pwfs8m", 16)}
    del fr
    out["pwfs39m_batched_fp32"] = batched("pwfs39m", 8)
    # the paper's SOUL example geometry: 40 x 40 subapertures, images 48 px
    # apart on a 120 px detector (80 px pupil padded three times, 2 x 2 bins)
    ws = synth.workload("soul8m")
    fs = PwfsFrame(ctx, ws, autotune=True)
    gs = fs.capture(st)
    time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), 5)
    mss = time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), steps)
    out["soul8m"] = {"config": "8.2 m, 80 px pupil padded 3x (240^2 FFT), 16 mod points, "
                               "40x40 subaps, images 48 px apart on a 120 px detector, "
                               "%d modes, FP32" % fs.n_modes,
                     "tiles": {"chunk": fs.tiles[0], "ka": fs.tiles[1], "passes": fs.tiles[2]}
                     if fs.tiles else None,
                     "frames_per_s": steps / (sum(mss) / 1e3), "ms_per_step": sum(mss) / steps}
    gs.close()
    del fs
    # the same example as the paper states it: 220 px pupil oversampled 3x
    # (660^2 FFT, Tab. 2's 24 x 660 x 660), detector pixels of 5.5 x 5.5 grid
    # pixels (area-weighted rebinning in the column pass), 500 modes
    ws = synth.workload("soul220")
    fs = PwfsFrame(ctx, ws, autotune=True)
    gs = fs.capture(st)
    time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), 5)
    mss = time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), steps)
    out["soul220"] = {"config": "8.2 m, 220 px pupil padded 3x (660^2 FFT = 30 x 22), 24 mod "
                                "points, 40x40 subaps of 5.5 px, images 48 px apart on a 120 px "
                                "detector (area-weighted rebinning), %d modes, FP32" % fs.n_modes,
                      "tiles": {"chunk": fs.tiles[0], "ka": fs.tiles[1], "passes": fs.tiles[2]}
                      if fs.tiles else None,
                      "frames_per_s": steps / (sum(mss) / 1e3), "ms_per_step": sum(mss) / steps,
                      "paper_context": "SOUL full loop 162.2 Hz (6.2 ms per step) on one GPU, "
                                       "Sect. 6 Tab. 1"}
    gs.close()
    del fs
    # the ANDES pyramid (Tab. 2's 24 x 1600 x 1600): 400 px pupil oversampled
    # 4x on the ELT, 100 x 100 subapertures, 35 layers, 4000 modes
    ws = synth.workload("andes400")
    fs = PwfsFrame(ctx, ws, autotune=True)
    gs = fs.capture(st)
    time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), 5)
    mss = time_graph(gs, lambda k: fs.t_dev.fill_(ws.dt_s * k), steps)
    out["andes400"] = {"config": "39 m, 400 px pupil padded 4x (1600^2 FFT = 32 x 50), 24 mod "
                                 "points, 100x100 subaps of 4 px, images 120 subaps apart on a "
                                 "400 px detector, 35 layers, 4000 x %d MVM, FP32"
                                 % fs.R.shape[1],
                       "tiles": {"chunk": fs.tiles[0], "ka": fs.tiles[1], "passes": fs.tiles[2]}
                       if fs.tiles else None,
                       "frames_per_s": steps / (sum(mss) / 1e3), "ms_per_step": sum(mss) / steps,
                       "paper_context": "ANDES full loop 19.6 Hz (50.9 ms per step) on one GPU, "
                                        "Sect. 6 Tab. 1"}
    gs.close()
    del fs
    torch.cuda.empty_cache()
    out["infinite8m"] = infinite_leg(ctx, st, flush, steps)
    wl = synth.workload("mwfs39m")
    S = System(ctx, wl)
    res = {}
    for name, sep in (("one_persistent_launch", False), ("per_sensor_launches", True)):
        g = S.capture(st, separate=sep)
        time_graph(g, lambda k: S.t_dev.fill_(wl.dt_s * k), 5)
        ms = time_graph(g, lambda k: S.t_dev.fill_(wl.dt_s * k), steps)
        res[name] = {"frames_per_s": steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
                     "kernels_per_frame": g.kernel_count()}
        g.close()
    sched = S.m.schedule()
    out["mwfs39m"] = {"config": "39 m: 6 laser-star SH (68x68 x 12 px, 24^2 FFT) + 3 pyramids "
                                "(120 px, 240^2 FFT, 16 mod), 10 layers, 4000 x %d MVM, FP32"
                                % S.n_slopes,
                      "tasks_per_frame": sched["n_tasks"], "ctas": sched["grid"], **res,
                      "speedup_persistent": res["per_sensor_launches"]["ms_per_step"]
                      / res["one_persistent_launch"]["ms_per_step"]}
    S.m.close()
    del S
    torch.cuda.empty_cache()
    return out


def gemm_leg(ctx, pk, n=8192, reps=10):
    """The tcgen05 BF16 GEMM (C = A B^T, FP32 accumulate) on an n^3 problem,
    against the measured cuBLAS BF16 burst peak."""
    import torch
    import paper_2602_06688_gb300 as sp
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn(n, n, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(n, n, device="cuda", generator=g).to(torch.bfloat16)
    Cm = torch.empty(n, n, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, tot = float("inf"), 0.0
    for _ in range(3):
        sp.specula_gemm_bf16(ctx, A, B, Cm)
    for _ in range(reps):
        e0.record()
        sp.specula_gemm_bf16(ctx, A, B, Cm)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        tot += e0.elapsed_time(e1)
    tf = 2.0 * n ** 3 / (best / 1e3) / 1e12
    peak = pk.get("bf16_tflops")
    out = {"kernel": "k_gemm_tn<bf16, 256> (persistent, one CTA per SM; TMA ring of 4 x 48 KB; "
                     "tcgen05 128x256x16 MMAs; two TMEM accumulators, epilogue overlapped)",
           "shape": [n, n, n], "best_ms": best, "mean_ms": tot / reps, "achieved_tflops": tf,
           "achieved_tflops_mean": 2.0 * n ** 3 / (tot / reps / 1e3) / 1e12,
           "peak_tflops": peak, "frac": (tf / peak) if peak else None,
           "peak_source": "measured cuBLAS bf16 burst" if peak else None}
    del A, B, Cm
    return out


def elt_calibrated_leg(ctx, fr, variants):
    """The ELT pyramid's 4000-mode reconstructor calibrated on the GPU (basis,
    push-pull interaction matrix, float64 pseudo-inverse) and compared at
    equal wavefront accuracy: the residual wavefront RMS left by the float32,
    split-bf16 and bf16 MVMs and by the 13344-2048-2048-4000 network (trained
    on synthetic modal phases) on held-out scaled atmospheric phases, next to
    each form's frame rate from the headline frame's variants."""
    import torch
    from paper_2602_06688_gb300.calibrated import CalibratedRecon
    t0 = time.perf_counter()
    cr = CalibratedRecon(ctx, fr)
    torch.cuda.synchronize()
    t_cal = time.perf_counter() - t0
    res = cr.compare()
    out = {"calibration_s": t_cal, "n_modes": cr.n_modes, "rank": res.pop("rank"),
           "residual_rms_rad": {k: res[k] for k in ("no_correction", "fp32", "bf16x2", "bf16",
                                                     "learned", "learned_correction")},
           "test": {"n_test": res["n_test"], "phase_rms_rad": res["phase_rms_rad"]},
           "learned_train": res["learned_train"],
           "frames_per_s": {"fp32": variants.get("fp32", {}).get("frames_per_s"),
                            "bf16x2": variants.get("bf16x2", {}).get("frames_per_s"),
                            "bf16": variants.get("bf16", {}).get("frames_per_s"),
                            "learned": variants.get("learned_mlp", {}).get("frames_per_s"),
                            "learned_correction":
                                variants.get("learned_mlp_correction", {}).get("frames_per_s")}}
    f = out["residual_rms_rad"]["fp32"]
    out["within_1pct_of_fp32"] = {k: abs(v - f) <= 0.01 * f
                                  for k, v in out["residual_rms_rad"].items()
                                  if k not in ("no_correction", "fp32")}
    del cr
    torch.cuda.empty_cache()
    return out


def recon_batched_leg(ctx, nb=2048, n_modes=4000, n_slopes=13344):
    """The ELT-size reconstructor applied to a batch of slope vectors: float32
    R on the CUDA cores against the split-bf16 and bf16 copies on the tensor
    cores (one multi-term GEMM), each with its relative error against a
    float64 product."""
    import torch
    import paper_2602_06688_gb300 as sp
    g = torch.Generator(device="cuda").manual_seed(17)
    R = torch.randn(n_modes, n_slopes, device="cuda", generator=g) / n_slopes ** 0.5
    X = torch.randn(nb, n_slopes, device="cuda", generator=g)
    hi = torch.empty(n_modes, n_slopes, dtype=torch.int16, device="cuda")
    lo = torch.empty_like(hi)
    sp.specula_recon_convert(ctx, R, sp.PREC_BF16X2, hi, lo)
    recs = {"fp32_cuda_cores": sp.recon_desc(n_modes, n_slopes, sp.PREC_FP32, R),
            "bf16x2_tensor": sp.recon_desc(n_modes, n_slopes, sp.PREC_BF16X2, hi, lo),
            "bf16_tensor": sp.recon_desc(n_modes, n_slopes, sp.PREC_BF16, hi)}
    ref = X.double() @ R.double().t()
    out = torch.empty(nb, n_modes, device="cuda")
    res = {"shape": [n_modes, n_slopes], "batch": nb}
    for name, rec in recs.items():
        sp.specula_recon(ctx, rec, X, out)
        torch.cuda.synchronize()
        err = float((out.double() - ref).norm() / ref.norm())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2 if name.startswith("fp32") else 10
        e0.record()
        for _ in range(reps):
            sp.specula_recon(ctx, rec, X, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"frames_per_s": nb / ms * 1e3, "ms_per_batch": ms,
                     "tflops": 2.0 * n_modes * n_slopes * nb / ms / 1e9, "rel_err_vs_fp64": err}
    del R, X, hi, lo, ref, out
    torch.cuda.empty_cache()
    return res


def gemm_rate(ctx, M, N, K, tf32, reps=10):
    """Best event-timed rate of the library's tcgen05 GEMM (TFLOP/s)."""
    import torch
    import paper_2602_06688_gb300 as sp
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    if not tf32:
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda")
    run = (lambda: sp.specula_gemm_tf32(ctx, A, B, C)) if tf32 else \
        (lambda: sp.specula_gemm_bf16(ctx, A, B, C))
    for _ in range(3):
        run()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del A, B, C
    return 2.0 * M * N * K / (best / 1e3) / 1e12


def dftgemm_leg(ctx, reps=20):
    """The DFT-as-GEMM pyramid forms (bf16 x 3, tf32 x 3) on the 8 m system
    (pwfs8m: 160 px pupil, 320^2 grid, 24 points, 40 x 40 subapertures, its
    3-layer atmosphere extracted on the GPU) against the register-FFT tilt
    form (autotuned): time per image and the normalised-intensity deviation
    from the FFT form (the error against the FP64 oracle is asserted by the
    parity tests)."""
    import torch
    import paper_2602_06688_gb300 as sp
    import synth
    from paper_2602_06688_gb300.frame import PwfsFrame
    fr = PwfsFrame(ctx, synth.workload("pwfs8m"))
    fr.frame(0.05)
    torch.cuda.synchronize()
    pu, pw, amp = fr.pupil, fr.pwfs, fr.amp
    ph = fr.phase.reshape(1, fr.n_pix, fr.n_pix).clone()
    nd = 2 * pw.n_sub
    det = torch.empty(1, nd, nd, device="cuda")
    ch, ka, ps = sp.specula_pwfs_autotune(ctx, pu, pw, amp, ph, det, reps=5)

    def timed():
        for _ in range(3):
            sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts) * 1e3, det[0].double().clone()

    flat = torch.zeros_like(ph)

    def slopes_rel():
        """Reference-subtracted slopes of the current form (its own flat
        reference)."""
        fdet = torch.empty_like(det)
        sp.specula_pwfs_image(ctx, pu, pw, amp, flat, fdet)
        r = torch.empty(fr.n_slopes, device="cuda")
        sp.specula_slopes(ctx, fr.slopec, fdet, None, r)
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        sl = torch.empty(fr.n_slopes, device="cuda")
        sp.specula_slopes(ctx, fr.slopec, det, r, sl)
        torch.cuda.synchronize()
        return sl.double()

    out = {"geometry": "pwfs8m: 160 px pupil, 320^2 grid, 24 modulation points, 40x40 "
                       "subapertures", "bound": "normalised intensity within 1e-5 of FP64; "
                                                "slope RMS deviation within 1e-3 of the slope RMS"}
    us, ref = timed()
    out["fft_tilt"] = {"us_per_image": us, "tiles": {"chunk": ch, "ka": ka, "passes": ps}}
    s_fft = slopes_rel()
    rn = ref / ref.sum()
    for form, name in ((sp.PWFS_FORM_DFTGEMM_BF16, "dftgemm_bf16x3"),
                       (sp.PWFS_FORM_DFTGEMM_TF32, "dftgemm_tf32x3")):
        sp.specula_pwfs_set_form(ctx, pu, pw, form)
        us, d = timed()
        dn = d / d.sum()
        sp.specula_prof_enable(ctx, 4096)
        for _ in range(10):
            sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        prof = sp.specula_prof_read(ctx)
        sp.specula_prof_enable(ctx, 0)
        s_g = slopes_rel()
        out[name] = {"us_per_image": us,
                     "norm_dev_vs_fft_form": float((dn - rn).abs().max() / rn.max()),
                     "slope_rms_dev_over_slope_rms": float((s_g - s_fft).norm() / s_fft.norm()),
                     "kernels_us": {k: v[0] / 10 * 1e3 for k, v in prof.items()}}
    sp.specula_pwfs_set_form(ctx, pu, pw, sp.PWFS_FORM_TILT)
    best = min(out["dftgemm_bf16x3"]["us_per_image"], out["dftgemm_tf32x3"]["us_per_image"])
    out["kept_in_frame"] = best < out["fft_tilt"]["us_per_image"]
    n, n_mod = fr.n_pix, pw.n_mod
    out["gemm_tflops_stage_shape"] = {
        "shape": [n_mod * 2 * n, 4 * n, 6 * n],
        "bf16": gemm_rate(ctx, n_mod * 2 * n, 4 * n, 6 * n, False),
        "tf32": gemm_rate(ctx, n_mod * 2 * n, 4 * n, 6 * n, True)}
    return out


# ------------------------------------------------------------------ GPU leg

def gpu_leg(args, ws, rank, local):
    import torch
    from paper_2602_06688_gb300 import build
    build.build()
    import paper_2602_06688_gb300 as sp
    from paper_2602_06688_gb300.frame import PwfsFrame
    import synth

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = synth.workload(WORKLOAD)
    ctx = sp.Context(local)
    fr = PwfsFrame(ctx, wl, seed_offset=1000 * rank, autotune=True)
    dt = wl.dt_s
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    K, W = args.steps, args.warmup

    st = torch.cuda.Stream()

    def timed(nsteps, t0_step, graph=True, with_flush=True):
        """Per-frame CUDA events on the launch stream; the L2 flush runs
        between frames, outside the events."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        with torch.cuda.stream(st):
            for k in range(nsteps):
                if with_flush:
                    flush.zero_()
                ev[k][0].record(st)
                if graph:
                    fr.replay((t0_step + k) * dt, st)
                else:
                    fr.frame((t0_step + k) * dt, stream=st)
                ev[k][1].record(st)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for k in range(W):
        fr.frame(k * dt)
    torch.cuda.synchronize()
    fr.capture(st)
    graph_kernels = fr.graph.kernel_count()
    timed(W, 0)

    # ---- headline: plain FP32 path, whole frame replayed as one CUDA graph
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.mark_start()
        wall0 = time.perf_counter()
        ms = timed(K, W)
        wall1 = time.perf_counter()
        clk.mark_end()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = graph_kernels * K
    ms_per_step, value = aggregate_ranks(sum(ms), K, ws, dist, "cuda")
    ms_eager = timed(K, W, graph=False)
    if args.quick:
        # headline frames only (used for profiler launch lists)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "frames/s",
                              "ms_per_step": ms_per_step, "quick": True,
                              "gpu_launches": launches}), flush=True)
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return
    fp32_slopes = fr.slopes.clone()

    # ---- precision variants of the reconstructor (same frame otherwise)
    variants = {}
    # FP64 reference product on the host for the error report
    ref_modes = fr.R.cpu().numpy().astype(np.float64) @ fp32_slopes.cpu().numpy().astype(np.float64)
    for name, prec in (("fp32", sp.PREC_FP32), ("bf16x2", sp.PREC_BF16X2), ("bf16", sp.PREC_BF16)):
        fr.set_precision(prec)
        fr.graph.close()
        fr.capture(st)
        timed(3, W)
        msv = timed(K, W)
        # modal error of this reconstructor on the FP32 slopes, vs FP64 R s
        out = torch.empty_like(fr.modes)
        sp.specula_recon(ctx, fr.rec, fp32_slopes, out)
        torch.cuda.synchronize()
        err = float(np.linalg.norm(out.cpu().numpy().astype(np.float64) - ref_modes) /
                    np.linalg.norm(ref_modes))
        variants[name] = {"frames_per_s": K / (sum(msv) / 1e3), "ms_per_step": sum(msv) / K,
                          "modal_rel_rms_err_vs_fp64": err}
    fr.set_precision(sp.PREC_FP32)
    # learned reconstructor at ELT scale in place of the MVM (frame timing;
    # its accuracy is measured on the 8 m configuration below)
    import synth as _synth
    sizes = (fr.n_slopes, 2048, 2048, fr.n_modes)
    mlp = sp.MLP(ctx, sizes, 128)
    for l in range(3):
        bnd = 1.0 / math.sqrt(sizes[l])
        mlp.set_layer(l, _synth.uniform_draws(300 + 2 * l, (sizes[l + 1], sizes[l]), -bnd, bnd),
                      _synth.uniform_draws(301 + 2 * l, (sizes[l + 1],), -bnd, bnd))
    fr.use_learned(mlp)
    fr.graph.close()
    fr.capture(st)
    timed(3, W)
    msl = timed(K, W)
    variants["learned_mlp"] = {"frames_per_s": K / (sum(msl) / 1e3), "ms_per_step": sum(msl) / K,
                               "net": "%d-2048-2048-%d GELU, batch 1: bf16 weight rows streamed by k_mlp_gemv on CUDA cores (tcgen05 GEMMs serve batches above 4)"
                                      % (fr.n_slopes, fr.n_modes)}
    # the network as a correction on top of the MVM (m = R s + f(s))
    fr.use_learned(mlp, correction=True)
    fr.graph.close()
    fr.capture(st)
    timed(3, W)
    msc = timed(K, W)
    variants["learned_mlp_correction"] = {
        "frames_per_s": K / (sum(msc) / 1e3), "ms_per_step": sum(msc) / K,
        "net": "FP32 MVM, then the same network by k_mlp_gemv, its output added to the modes"}
    fr.use_learned(None)
    fr.graph.close()
    fr.capture(st)
    mlp.close()

    # shifted-mask modulation (one forward transform per image, the mask moved
    # per point): its frame rate, and its deviation from the tilt form on the
    # same phase (detector and reference-subtracted slopes)
    t_cmp = 5 * fr.dt
    fr.frame(t_cmp)
    torch.cuda.synchronize()
    det_t, sl_t, ref_t = fr.det.clone(), fr.slopes.clone(), fr.ref.clone()
    sp.specula_pwfs_set_form(ctx, fr.pupil, fr.pwfs, sp.PWFS_FORM_SHIFTED)
    flat, fdet = torch.zeros_like(fr.phase), torch.empty_like(fr.det)
    sp.specula_pwfs_image(ctx, fr.pupil, fr.pwfs, fr.amp, flat, fdet)
    sp.specula_slopes(ctx, fr.slopec, fdet, None, fr.ref)      # flat reference, this form
    fr.frame(t_cmp)
    torch.cuda.synchronize()
    a = det_t.double() / det_t.double().sum()
    b = fr.det.double() / fr.det.double().sum()
    dev_img = float((a - b).abs().max() / a.abs().max())
    dev_sl = float((fr.slopes.double() - sl_t.double()).norm() / sl_t.double().norm())
    fr.graph.close()
    fr.capture(st)
    timed(3, W)
    mss = timed(K, W)
    sp.specula_prof_enable(ctx, 64 * (K + 4))
    timed(K, W, graph=False)
    prof_s = sp.specula_prof_read(ctx)
    sp.specula_prof_enable(ctx, 0)
    variants["shifted_mask"] = {
        "frames_per_s": K / (sum(mss) / 1e3), "ms_per_step": sum(mss) / K,
        "detector_norm_max_dev_vs_tilt": dev_img, "slope_rel_rms_dev_vs_tilt": dev_sl,
        "kernels_us": {k: 1e3 * v[0] / K for k, v in prof_s.items()},
        "form": "one forward 2D FFT per image; per point the analytic mask at the shifted "
                "frequencies, inverse FFT, |.|^2 (a different discretisation of the modulation)"}
    sp.specula_pwfs_set_form(ctx, fr.pupil, fr.pwfs, sp.PWFS_FORM_TILT)
    fr.ref.copy_(ref_t)
    # detector photon and readout noise in the frame (CCD call after the
    # image): frame rate, and the slope noise against the noise-free frame
    noise = {"photons": 2.0e6, "qe": 0.8, "ron": 0.5, "seed": 7}
    fr.noise = noise
    fr.noise_scale = noise["photons"] * noise["qe"] / float(
        sp.specula_pupil_mask_host(fr.pupil).sum())
    fr.frame(t_cmp)
    torch.cuda.synchronize()
    dev_noise = float((fr.slopes.double() - sl_t.double()).norm() / sl_t.double().norm())
    fr.graph.close()
    fr.capture(st)
    timed(3, W)
    msn = timed(K, W)
    variants["ccd_noise"] = {"frames_per_s": K / (sum(msn) / 1e3), "ms_per_step": sum(msn) / K,
                             "photons_per_frame": noise["photons"], "qe": noise["qe"],
                             "ron_e": noise["ron"],
                             "slope_rel_rms_noise": dev_noise}
    fr.noise = None
    fr.graph.close()
    fr.capture(st)

    # ---- live per-kernel roofline (library event tracing on the launch
    # stream; tracing brackets eager launches, so this pass runs eagerly)
    sp.specula_prof_enable(ctx, 64 * (K + 4))
    timed(K, W, graph=False)
    prof = sp.specula_prof_read(ctx)
    sp.specula_prof_enable(ctx, 0)
    pk, how = peaks()
    flops = kernel_flops(wl)
    n_frames = K
    kern = {}
    for name, (tms, n) in prof.items():
        kern[name] = {"total_ms": tms, "launches": n, "share": 0.0}
    tot = sum(v["total_ms"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["total_ms"] / tot if tot else 0.0
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    clocks = clk.summary()
    sm_max = (clocks or {}).get("sm_max_mhz") or pk.get("sm_max_mhz", 2070.0)
    peak_alu = fp32_peak_tflops(sm_max)
    roof = None
    traffic = read_traffic()
    # The FFT/mask/accumulate stage (the pyramid's 2D filter and |E|^2, one
    # launch of each of its kernels per frame) is the dominant work.  Its
    # algorithmic FLOPs per frame count two full N x N transforms per
    # modulation point, 5 N^2 log2(N^2) each, pruning
    # and shared row filters not subtracted (so the rate compares with a
    # plain implementation); achieved = that count / the summed time of the
    # stage's kernels.
    s0 = wl.sensors[0]
    N = s0.pwfs.pad * s0.pupil.n_pix
    stage_flops = s0.pwfs.n_mod * 2 * 5.0 * N * N * math.log2(N * N)
    stage = [k for k in ("pwfs_rowfilt", "pwfs_colfilt_bin") if k in kern] or \
            [k for k in ("pwfs_rows_fwd", "pwfs_cols", "pwfs_rows_inv") if k in kern]
    if stage:
        st_ms = sum(kern[k]["total_ms"] for k in stage)
        achieved = stage_flops * n_frames / (st_ms / 1e3) / 1e12
        trs = [traffic.get((k, WORKLOAD)) for k in stage]
        tr = sum(trs) if all(t is not None for t in trs) else None
        roof = {"bound": "alu", "kernel": "+".join(stage), "achieved": achieved, "peak": peak_alu,
                "unit": "TFLOP/s", "frac": achieved / peak_alu,
                "traffic": tr * 1.0 if tr is not None else None,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (derived)",
                "flops_per_launch": stage_flops,
                "flops_convention": "n_mod x 2 x 5 N^2 log2(N^2) per frame (two full 2D FFTs "
                                    "per modulation point)",
                "dominant_kernel": dom}
    for name in flops:
        if name in kern:
            kern[name]["achieved_tflops"] = flops[name] * n_frames / (kern[name]["total_ms"] / 1e3) / 1e12
    if "recon" in kern:
        rb = fr.n_modes * fr.n_slopes * 4.0
        gbs = rb * kern["recon"]["launches"] / (kern["recon"]["total_ms"] / 1e3) / 1e9
        kern["recon"]["achieved_gbs"] = gbs
        kern["recon"]["hbm_frac"] = gbs / pk["hbm_gbs"]
        kern["recon"]["traffic"] = traffic.get(("recon", WORKLOAD))

    # ---- each stage of the frame captured as its own CUDA graph and
    # replayed after an L2 flush: per-stage device time without the tracing
    # events that bracket every eager launch above
    def stage_us(enqueue, n=max(K, 20)):
        torch.cuda.synchronize()
        sp.specula_graph_begin(ctx, st)
        try:
            enqueue()
        finally:
            g = sp.specula_graph_end(ctx, st)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n + 3)]
        with torch.cuda.stream(st):
            for a, b in ev:
                flush.zero_()
                a.record(st)
                g.launch(st)
                b.record(st)
        torch.cuda.synchronize()
        kernels = g.kernel_count()
        g.close()
        t = [a.elapsed_time(b) * 1e3 for a, b in ev[3:]]
        return {"us": sum(t) / len(t), "kernels": kernels}

    fr.t_dev.fill_(W * dt)
    stages = {
        "extraction": stage_us(lambda: sp.specula_atmo_extract(
            ctx, fr.layers, fr.screens, fr.src, fr.pupil, 0.0, fr.phase, t_dev=fr.t_dev,
            stream=st)),
        "image": stage_us(lambda: sp.specula_pwfs_image(ctx, fr.pupil, fr.pwfs, fr.amp,
                                                        fr.phase, fr.det, stream=st)),
        "slopes": stage_us(lambda: sp.specula_slopes(ctx, fr.slopec, fr.det, fr.ref, fr.slopes,
                                                     stream=st)),
        "reconstructor": stage_us(lambda: sp.specula_recon(ctx, fr.rec, fr.slopes, fr.modes,
                                                           stream=st)),
    }
    stages["sum_us"] = sum(v["us"] for v in stages.values())
    stages["whole_frame_graph_us"] = ms_per_step * 1e3
    stages["note"] = ("each stage captured alone and replayed after an L2 flush (so each "
                      "starts cold); the whole frame's graph chains them")

    # ---- end to end through the public API with host buffers: per frame the
    # time goes host -> device, the captured frame runs, the modes come back.
    # Synchronous: the host waits for every frame's modes before the next.
    t_host = torch.empty(1, dtype=torch.float64).pin_memory()
    modes_host = torch.empty(fr.n_modes, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    with torch.cuda.stream(st):
        for k in range(K):
            t_host[0] = (W + k) * dt
            fr.t_dev.copy_(t_host, non_blocking=True)
            fr.graph.launch(st)
            modes_host.copy_(fr.modes, non_blocking=True)
            st.synchronize()
    e1 = time.perf_counter()
    e2e_sync = ws * K / (e1 - e0)
    # Pipelined (the open-loop frame does not feed the next one): the same
    # copies every frame, from and into a ring of pinned slots; the host waits
    # only before reusing a slot (for the copy-back of the frame that last
    # used it), and once at the end.
    R = 8
    t_ring = torch.empty(R, dtype=torch.float64).pin_memory()
    m_ring = torch.empty(R, fr.n_modes, dtype=torch.float32).pin_memory()
    evs = [torch.cuda.Event() for _ in range(R)]
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    with torch.cuda.stream(st):
        for k in range(K):
            sl = k % R
            if k >= R:
                evs[sl].synchronize()
            t_ring[sl] = (W + k) * dt
            fr.t_dev.copy_(t_ring[sl:sl + 1], non_blocking=True)
            fr.graph.launch(st)
            m_ring[sl].copy_(fr.modes, non_blocking=True)
            evs[sl].record(st)
        st.synchronize()
    e1 = time.perf_counter()
    e2e = ws * K / (e1 - e0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws,
                "steps": K, "warmup": W, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded von Karman screens, seeded stand-in R)",
                "config": {"workload": WORKLOAD, "pupil_px": 480, "fft": 960, "n_mod": 48,
                           "n_sub": 96, "layers": 35, "n_modes": fr.n_modes,
                           "n_slopes": fr.n_slopes, "l2": "flushed between timed frames",
                           "pwfs_tiles": {"chunk": fr.tiles[0], "ka": fr.tiles[1],
                                          "passes": fr.tiles[2]} if fr.tiles else None,
                           "frame": "one CUDA graph per frame (%d kernels)" % graph_kernels,
                           "eager_frames_per_s": K / (sum(ms_eager) / 1e3),
                           "wall_ms_per_step_incl_flush": (wall1 - wall0) * 1e3 / K},
                "roofline": roof, "kernels": kern, "stages_graph": stages,
                "variants": variants,
                "e2e": {"value": e2e, "unit": "frames/s", "h2d_bytes_per_step": 8,
                        "d2h_bytes_per_step": 4 * fr.n_modes,
                        "note": "per step: pinned host time -> device, frame, modes -> pinned "
                                "host, in a ring of 8 pinned slots (host waits before reusing a "
                                "slot, and at the end)",
                        "synchronous_value": e2e_sync,
                        "synchronous_note": "the host waits for every frame's modes"},
                "gpu_launches": launches, "clocks": clocks,
                "peaks": {"source": how, "hbm_gbs": pk.get("hbm_gbs")}}
        meas = fma_peaks_leg(ctx)
        meas["fp32_derived_tflops"] = peak_alu
        meas["fp32_measured_over_derived"] = meas["fp32_fma_tflops"] / peak_alu
        meas["fft_stage_frac_of_measured_fp32"] = (roof["achieved"] / meas["fp32_fma_tflops"]
                                                   if roof else None)
        line["peaks"]["measured_fma"] = meas
        if not args.no_systems:
            line["systems"] = systems_leg(ctx)
        if not args.no_loop:
            line["closed_loop"] = closed_loop_leg(ctx)
        if not args.no_learned:
            line["learned"] = learned_leg(ctx)
            line["gemm_bf16"] = gemm_leg(ctx, pk)
        meas["tf32_gemm_tflops_8192"] = gemm_rate(ctx, 8192, 8192, 8192, True)
        line["variants"]["elt_calibrated"] = elt_calibrated_leg(ctx, fr, line["variants"])
        line["variants"]["dftgemm_8m"] = dftgemm_leg(ctx)
        line["variants"]["recon_batched_elt"] = recon_batched_leg(ctx)
        if not args.no_cpu_baseline:
            line["cpu_baseline"], line["cpu_baseline_single_core"] = cpu_baselines()
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="specula", choices=["specula", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the 8 m and 39 m multi-sensor system timings")
    ap.add_argument("--no-loop", action="store_true",
                    help="skip the closed-loop run on the 8 m system")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-reconstructor training run on the 8 m system")
    ap.add_argument("--quick", action="store_true",
                    help="headline frames only (no variants, tracing pass, e2e or baseline)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        reference_leg(args, ws, rank)
        return
    gpu_leg(args, ws, rank, local)


if __name__ == "__main__":
    main()
