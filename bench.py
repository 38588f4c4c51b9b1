"""Benchmark: least-misfit gridding + degridding throughput on one GB300 (or N replicas).

One step = the whole hot path on one batch of visibilities: bin the positions, grid,
FFT (+i), correct and crop to the dirty image; pad and correct a model image, FFT (-i),
degrid to predicted visibilities. The model's pad and transform, which do not depend on the
positions, run on a second stream while the positions are binned and gridded, and the
degridding runs on a third while the dirty image is transformed and cropped. Workload: 64-antenna Earth-rotation tracks (6 h,
2048 samples, 1.4 GHz; 4,128,768 visibilities), 4096^2 grid, 2048^2 image (x0 = 0.5),
W = 7, linear table at M_s = 1000, complex64.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle instead.

Two further workloads print their own line (not the headline):
  --workload channels  96 frequency channels of uneven visibility counts (log-uniform in
                       1e5-2e6), grid sizes drawn from {1024^2, 2048^2, 4096^2} and W from
                       {4, 6, 8}: gridding + degridding as a tuned, graph-captured batch
                       (one persistent sweep per W) against 96 sequential single-plan calls.
  --workload autograd  differentiable imaging, L = ||P I - V||^2 with 49.5e6 visibilities
                       (64 channels x 384 samples over 0.95-1.05 GHz), 4096^2 grid, W = 8:
                       forward + backward with all channels in one plan against one plan
                       per channel.
  --workload precision float64 sweeps on the 4.1M-visibility tracks (Section 5.2): W = 7 with linear
                       (M_s = 1000) and cubic (M_s = 20000) tables and with the direct calculation of
                       the weights, W = 14 with a cubic table; next to the float32 W = 7 sweeps.
  --workload large     high accuracy at scale: 128 antennas x 768 samples (8 h) x 32
                       channels = 2.0e8 visibilities, 8192^2 grid, W = 12: float32 gridding
                       with plain and with compensated (two-float) accumulation, errors
                       against the float64 path and FP64-oracle spot checks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mvis/s grid+degrid at W=7, 4096² grid; fraction of roofline; RMS error vs FP64"
WORKLOAD = dict(n_ant=64, hours=6.0, n_times=2048, freq_hz=1.4e9, n_src=200, noise_sigma=0.1,
                N=4096, n_image=2048, x0=0.5, W=7, oversample=1000, interp="linear")
# positions are stored sample-major (one sample of every baseline, then the next sample), as a
# correlator writes them; the binning is told the number of tracks (lmg_plan_bin_tracks)
WORKLOAD["tracks"] = WORKLOAD["n_ant"] * (WORKLOAD["n_ant"] - 1) // 2
WORKLOAD_NAME = ("64-antenna 6 h Earth-rotation tracks (2048 samples, 1.4 GHz, dec -30), 4,128,768 vis, "
                 "200 point sources + noise, 4096^2 grid, 2048^2 image, W=7, linear table M_s=1000, complex64")
L2_FLUSH_BYTES = 256 << 20
CLOCK_WINDOW_S = 2.2  # the clock record spans the timed steps plus identical steps up to this long
VALUE_DEFINITION = ("value = visibilities / time of one whole step (bin + grid + image transform with correction "
                    "and crop + model transform with pad and correction + degrid); grid_degrid_mvis_s = visibilities / "
                    "(grid + degrid kernel time), the narrower figure of the metric's name")
KERNELS_PER_STEP = 12  # bin 5, grid sweep + spill 2, image transform 2, model transform 2, degrid sweep 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="tracks", choices=["tracks", "channels", "autograd", "large", "precision"])
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run this many untimed steps only (for ncu launch lists) and exit")
    return ap.parse_args()


def max_over_ranks(ms, device):
    """The slowest rank's time: replicas run the same work, the job ends with the last one
    (all-reduce MAX over the process group; the value itself on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mvis(nvis_per_rank, world, ms):
    """Visibilities processed by all ranks per second, in millions."""
    return world * nvis_per_rank / (ms * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs():
    from paper_1906_07102_gb300 import synthetic as S
    w = WORKLOAD
    uv = S.array_tracks(n_ant=w["n_ant"], hours=w["hours"], n_times=w["n_times"], freqs_hz=(w["freq_hz"],), seed=0)
    dl = S.pixel_scale_for(uv)
    l, m, f = S.point_source_sky(w["n_src"], 0.45 * w["n_image"] * dl, seed=0)
    vis = S.visibilities(uv, l, m, f, noise_sigma=w["noise_sigma"], seed=0).astype(np.complex64)
    model = S.gaussian_blob_image(w["n_image"], 64, seed=0).astype(np.complex64)
    return uv, dl, vis, model


# ---------------------------------------------------------------------------------------
# oracle (CPU) timing: the reference arm and the cpu_baseline leg
# ---------------------------------------------------------------------------------------
_ORACLE_SETUP = {}


def oracle_setup():
    """The oracle's table and correction factors for the workload (built once, untimed)."""
    if not _ORACLE_SETUP:
        from oracle import design as D
        from oracle import imaging as I
        w = WORKLOAD
        N, n_img, W, Ms = w["N"], w["n_image"], w["W"], w["oversample"]
        h = D.least_misfit_h(W, w["x0"] / 2)
        T = D.lm_table(h, W, w["x0"] / 2, Ms)
        _ORACLE_SETUP["T"] = T
        _ORACLE_SETUP["hv"] = D.correction_factors(T, Ms, D.INTERP_LINEAR, W, I.pixel_coords(n_img, N))
    return _ORACLE_SETUP["T"], _ORACLE_SETUP["hv"]


def oracle_step(uv, dl, vis, model, T, hv):
    """One oracle step on the given visibilities with the full grid: grid, FFT (+i), correct
    and crop; pad and correct the model, FFT (-i), degrid. Returns seconds per stage."""
    from oracle import imaging as I
    w = WORKLOAD
    N, n_img, W, Ms = w["N"], w["n_image"], w["W"], w["oversample"]
    t0 = time.perf_counter()
    uc = I.cells_from_wavelengths(uv, N, dl)
    plan = I.Plan(uc[:, 0], uc[:, 1], W, N)
    G = I.grid(plan, T, Ms, 1, np.asarray(vis, dtype=np.complex128))
    t1 = time.perf_counter()
    img = I.correct_crop(I.fft_image(G), hv, n_img)
    del G
    Gm = I.model_grid(I.pad_correct(np.asarray(model, dtype=np.complex128), hv, N))
    t2 = time.perf_counter()
    pv = I.degrid(plan, T, Ms, 1, Gm)
    t3 = time.perf_counter()
    assert np.isfinite(img).all() and np.isfinite(pv).all()
    return {"grid": t1 - t0, "fft_correct": t2 - t1, "degrid": t3 - t2, "total": t3 - t0}


def _oracle_worker(idx, uv, dl, vis, model, T, hv, n_steps, barrier, queue):
    """One host core of the all-core oracle: n_steps steps on its share of the visibilities,
    each started together with the other workers' at a barrier."""
    for k in range(n_steps):
        barrier.wait()
        st = oracle_step(uv, dl, vis, model, T, hv)
        queue.put((idx, k, int(uv.shape[0]), st))


def oracle_workers():
    """Worker count for the all-core oracle: every host core, as far as memory allows
    (a worker holds about 2.5 GB at the 4096^2 grid)."""
    cores = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        cores = max(1, min(cores, int(mem // (2.5 * 2 ** 30))))
    except (ValueError, OSError, AttributeError):
        pass
    return cores


def oracle_allcore(uv, dl, vis, model, n_steps, every=1):
    """The oracle on every host core: the visibilities sel = every `every`-th are dealt to P
    spawned worker processes (one core each), each runs a whole oracle step on its share
    (its own full-size grid and FFTs). Returns (P, visibilities per step, list of wall
    seconds per step from the common start to the last worker's result, per-stage
    seconds of the slowest worker of the last step)."""
    import multiprocessing as mp
    T, hv = oracle_setup()
    P = oracle_workers()
    sel = np.arange(0, uv.shape[0], every)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(P + 1)
    queue = ctx.Queue()
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    procs = []
    try:
        for p in range(P):
            part = sel[p::P]
            procs.append(ctx.Process(target=_oracle_worker,
                                     args=(p, np.ascontiguousarray(uv[part]), dl, np.ascontiguousarray(vis[part]),
                                           model, T, hv, n_steps, barrier, queue), daemon=True))
            procs[-1].start()
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    walls, last = [], None
    for k in range(n_steps):
        barrier.wait()
        t0 = time.perf_counter()
        res = [queue.get() for _ in range(P)]
        walls.append(time.perf_counter() - t0)
        last = max((r[3] for r in res), key=lambda st: st["total"])
    for pr in procs:
        pr.join(timeout=60)
    return P, int(sel.size), walls, last


def oracle_single(uv, dl, vis, model, every):
    """The oracle on one core (this process) on every `every`-th visibility."""
    T, hv = oracle_setup()
    sel = np.arange(0, uv.shape[0], every)
    st = oracle_step(uv[sel], dl, vis[sel], model, T, hv)
    return int(sel.size), st


ALLCORE_TEXT = ("the FP64 oracle (numpy) on {P} host cores: the {n} visibilities ({frac}) dealt to {P} spawned "
                "processes, each running a whole oracle step (grid, FFT, crop, pad, FFT, degrid) on its share with "
                "its own 4096^2 grid; value = visibilities per second from the common start to the last result "
                "(the {P} partial dirty images are not summed)")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    uv, dl, vis, model = make_inputs()
    nv = uv.shape[0]
    P, n, walls, last = oracle_allcore(uv, dl, vis, model, args.warmup + args.steps)
    timed = walls[args.warmup:]
    step_s = float(np.mean(timed))
    value = n / step_s / 1e6
    sample = ALLCORE_TEXT.format(P=P, n=n, frac="all of them")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvis/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "parallelism": f"{P} host processes"},
            "value_definition": VALUE_DEFINITION,
            "oracle_stage_s_slowest_worker": last,
            "cpu_baseline": {"value": value, "unit": "Mvis/s", "cores": P, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mvis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region: start() waits for the sampler's first
    line, mark() notes where the timed region begins, stop() keeps the samples taken from
    there on (at least one, waiting briefly for it when the region was shorter than the
    sampling interval)."""

    def __init__(self, index):
        import tempfile
        self.proc = None
        self.index = index
        fd, self.path = tempfile.mkstemp(prefix=f"lmg_clocks_rank{index}_", suffix=".csv")
        os.close(fd)
        self.first = 0

    def _lines(self):
        with open(self.path) as f:
            return [ln for ln in f.read().splitlines() if ln.count(",") >= 8]

    def _wait_lines(self, n, timeout):
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < timeout:
            if len(self._lines()) >= n:
                return
            time.sleep(0.01)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            self._wait_lines(1, 2.0)
        except (OSError, FileNotFoundError):
            self.proc = None
            if getattr(self, "f", None) is not None:
                self.f.close()

    def mark(self):
        if self.proc is not None:
            self.first = len(self._lines())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._wait_lines(self.first + 1, 1.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        lines = self._lines()[self.first:]
        try:
            os.remove(self.path)
        except OSError:
            pass
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(np.max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


SWEEP_SOURCES = ("sweep.cu", "sweep_body.cuh", "device_common.cuh")


def sweep_sources_sha256():
    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1906_07102_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_record(pass_name):
    """DRAM traffic per launch of the gridding ("grid") or degridding ("degrid") sweep from
    the committed ncu summary, if the pass's record holds for the current sweep sources
    (the SHA-256 of the sources it was taken on, or of later sources that left that pass's
    kernel code unchanged, listed in the record with the reason)."""
    p = os.path.join(ROOT, "profiles", "sweeps_config2_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
        valid = rec[pass_name].get("sources_sha256", [rec.get("sweep_sources_sha256")])
        if sweep_sources_sha256() not in valid:
            return None
        return float(rec[pass_name]["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def accuracy(uv, dl, vis, model, img, pv):
    """Relative RMS error against the FP64 oracle on sampled outputs: 24 dirty-image pixels
    (direct per-pixel evaluation) and 2000 predicted visibilities (full FP64 model grid)."""
    from oracle import design as D
    from oracle import imaging as I
    w = WORKLOAD
    N, n_img, W, Ms = w["N"], w["n_image"], w["W"], w["oversample"]
    h = D.least_misfit_h(W, w["x0"] / 2)
    T = D.lm_table(h, W, w["x0"] / 2, Ms)
    x = I.pixel_coords(n_img, N)
    g = np.random.default_rng(123)
    py, px = g.integers(0, n_img, 24), g.integers(0, n_img, 24)
    hx = D.correction_factors(T, Ms, 1, W, x[px])
    hy = D.correction_factors(T, Ms, 1, W, x[py])
    uc = I.cells_from_wavelengths(uv, N, dl)
    plan = I.Plan(uc[:, 0], uc[:, 1], W, N)
    ref_px = I.dirty_pixels_direct(plan, T, Ms, 1, hx, hy, vis.astype(np.complex128), None, x[px], x[py])
    e_img = np.sqrt(np.mean(np.abs(img[py, px] - ref_px) ** 2) / np.mean(np.abs(ref_px) ** 2))
    sel = g.integers(0, uv.shape[0], 2000)
    hv = D.correction_factors(T, Ms, 1, W, x)
    Gm = I.model_grid(I.pad_correct(model.astype(np.complex128), hv, N))
    sub = I.Plan(uc[sel, 0], uc[sel, 1], W, N)
    ref_pv = I.degrid(sub, T, Ms, 1, Gm)
    e_pv = np.sqrt(np.mean(np.abs(pv[sel] - ref_pv) ** 2) / np.mean(np.abs(ref_pv) ** 2))
    return {"dirty_image_rel_rms": float(e_img), "predicted_vis_rel_rms": float(e_pv),
            "sample": "24 random pixels of the 2048^2 dirty image; 2000 random predicted visibilities"}


class OverlappedStep:
    """One step of the hot path through the public calls, with work that does not depend on
    other work on separate streams: the prediction's model grid (pad, correction and
    transform: lmg_grid_from_image) runs on a side stream from the step's start,
    concurrently with the binning and gridding on the caller's stream; after the gridding,
    the degridding of the model grid runs on a third stream while the caller's stream
    transforms, corrects and crops the dirty image (lmg_image_from_grid); the caller's
    stream ends the step when both are done. The two transforms have scratch arrays of their
    own; the predictions' buffer is zeroed on the side stream at the start and the
    degridding adds into it (lmg_degrid_add), so that no zeroing precedes it. Nothing of step k + 1 starts on any stream before step k has ended on the caller's
    stream. Measured on the 4.1M-visibility workload with the library transforms: 0.982 ms
    per step against 1.024 ms with the same calls in series."""

    def __init__(self, plan, N, dev, tracks):
        import torch
        self.torch = torch
        self.plan = plan
        self.tracks = tracks
        self.side = torch.cuda.Stream(device=dev)
        self.side2 = torch.cuda.Stream(device=dev)
        self.work = torch.empty((N, N), dtype=torch.complex64, device=dev)
        self.model_grid = torch.empty((N, N), dtype=torch.complex64, device=dev)
        nb = plan.transform_scratch_bytes() // 8
        self.scratch_model = torch.empty(nb, dtype=torch.complex64, device=dev) if nb else None
        self.scratch_image = torch.empty(nb, dtype=torch.complex64, device=dev) if nb else None
        self.start = torch.cuda.Event()
        self.model_ready = torch.cuda.Event()
        self.gridded = torch.cuda.Event()
        self.predicted = torch.cuda.Event()

    def __call__(self, uv, vis, model, img, pv, main, img_ready=None):
        torch, plan = self.torch, self.plan
        self.start.record(main)
        self.side.wait_event(self.start)
        with torch.cuda.stream(self.side):
            pv.zero_()   # the degridding adds into it (lmg_degrid_add): no zeroing on the critical path
            plan.grid_from_image(model, out=self.model_grid, scratch=self.scratch_model)
            self.model_ready.record(self.side)
        plan.bin(uv, tracks=self.tracks)
        plan.grid(vis, out=self.work)
        self.gridded.record(main)
        self.side2.wait_event(self.gridded)
        self.side2.wait_event(self.model_ready)
        with torch.cuda.stream(self.side2):
            plan.degrid(self.model_grid, out=pv, add=True)
            self.predicted.record(self.side2)
        plan.image_from_grid(self.work, out=img, scratch=self.scratch_image)
        if img_ready is not None:
            img_ready.record(main)
        main.wait_event(self.predicted)


def run_native(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1906_07102_gb300 import lmg
    w = WORKLOAD
    uv, dl, vis, model = make_inputs()
    nv = uv.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    table = lmg.Table(w["W"], w["x0"], w["oversample"], w["interp"])
    plan = lmg.Plan(table, w["n_image"], dl, nv, "c64")
    uv_d = torch.from_numpy(uv).to(dev)
    vis_d = torch.from_numpy(vis).to(dev)
    model_d = torch.from_numpy(model).to(dev)
    img_d = torch.empty((w["n_image"], w["n_image"]), dtype=torch.complex64, device=dev)
    pv_d = torch.empty(nv, dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    ostep = OverlappedStep(plan, w["N"], dev, w["tracks"])

    def step():
        ostep(uv_d, vis_d, model_d, img_d, pv_d, stream)

    if args.profile_steps:
        for _ in range(args.profile_steps):
            step()
        torch.cuda.synchronize()
        return

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed before each (outside the step's events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    step_ms = max_over_ranks(float(np.mean([s.elapsed_time(e) for s, e in zip(starts, ends)])), dev)
    value = whole_job_mvis(nv, world, step_ms)
    # the K timed steps last about K ms: the clock record continues over identical steps
    clk = soak(step, flush, stream, torch, t_wall, clocks, args.steps)

    # per-stage breakdown (outside the timed steps; same stream, events per stage)
    stages = {}

    def timed(name, fn, reps=max(3, min(args.steps, 10))):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        stages[name] = float(np.mean(ts))

    work = torch.empty((w["N"], w["N"]), dtype=torch.complex64, device=dev)
    timed("bin_plain", lambda: plan.bin(uv_d))     # the same binning without the layout hint
    timed("bin", lambda: plan.bin(uv_d, tracks=w["tracks"]))
    timed("grid", lambda: plan.grid(vis_d, out=work))
    timed("image_transform", lambda: plan.image_from_grid(work, out=img_d))     # fused, leaves work
    timed("model_transform", lambda: plan.grid_from_image(model_d, out=work))
    timed("degrid", lambda: plan.degrid(work, out=pv_d))
    # the library path of the same two transforms, for comparison (not in the step)
    timed("fft_image_library", lambda: plan.fft(work, "image", pruned=True))
    timed("crop_correct_library", lambda: plan.crop_correct(work, out=img_d))
    timed("pad_correct_library", lambda: plan.pad_correct(model_d, out=work))
    timed("fft_model_library", lambda: plan.fft(work, "model", pruned=True))
    # the two public calls of a step, as a whole (prediction pads only the kept rows)
    timed("dirty_image", lambda: plan.dirty_image(vis_d, out=img_d))
    timed("predict_vis", lambda: plan.predict_vis(model_d, out=pv_d))

    # end to end through the public API with pinned host buffers: every step uploads its
    # uv, visibilities and model and downloads its image and predictions. Two sets of device
    # buffers let step k+1's uploads and step k's downloads run on copy streams while step k
    # computes; every reuse of a buffer waits (stream-order events) for the work that last
    # used it, so each step reads its own inputs.
    uv_h = torch.from_numpy(uv).pin_memory()
    vis_h = torch.from_numpy(vis).pin_memory()
    model_h = torch.from_numpy(model).pin_memory()
    img_h = torch.empty(img_d.shape, dtype=img_d.dtype).pin_memory()
    pv_h = torch.empty(pv_d.shape, dtype=pv_d.dtype).pin_memory()
    bufs = [dict(uv=uv_d, vis=vis_d, model=model_d, img=img_d, pv=pv_d),
            dict(uv=torch.empty_like(uv_d), vis=torch.empty_like(vis_d), model=torch.empty_like(model_d),
                 img=torch.empty_like(img_d), pv=torch.empty_like(pv_d))]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def ev():
        return torch.cuda.Event()

    def e2e_run(k_steps):
        up = [ev(), ev()]          # inputs of the set uploaded
        used = [ev(), ev()]        # compute done with the set's inputs and outputs
        down = [ev(), ev()]        # outputs of the set downloaded
        for e in used + down:
            e.record(stream)

        def upload(b):
            s_in.wait_event(used[b])
            with torch.cuda.stream(s_in):
                bufs[b]["uv"].copy_(uv_h, non_blocking=True)
                bufs[b]["vis"].copy_(vis_h, non_blocking=True)
                bufs[b]["model"].copy_(model_h, non_blocking=True)
                up[b].record(s_in)

        upload(0)
        for k in range(k_steps):
            b = k % 2
            if k + 1 < k_steps:
                upload(1 - b)
            stream.wait_event(up[b])
            stream.wait_event(down[b])
            d = bufs[b]
            img_ready = ev()
            ostep(d["uv"], d["vis"], d["model"], d["img"], d["pv"], stream, img_ready)
            used[b].record(stream)
            s_out.wait_event(img_ready)
            with torch.cuda.stream(s_out):
                img_h.copy_(d["img"], non_blocking=True)
                s_out.wait_event(used[b])
                pv_h.copy_(d["pv"], non_blocking=True)
                down[b].record(s_out)
        stream.wait_stream(s_out)              # the last results are on the host
        stream.wait_stream(s_in)

    e2e_run(2)
    torch.cuda.synchronize()
    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ek = max(3, min(args.steps, 10))
    es.record(stream)
    e2e_run(ek)
    ee.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(es.elapsed_time(ee) / ek, dev)
    h2d = uv_h.numel() * 8 + vis_h.numel() * 8 + model_h.numel() * 8
    d2h = img_h.numel() * 8 + pv_h.numel() * 8

    # roofline of the dominant sweep pass (gridding = sweep + spill, degridding = zeroing +
    # sweep; whichever took longer): algorithmic bytes per launch and the arithmetic side
    # 4 W^2 flops per visibility per pass, against the measured HBM copy bandwidth and the
    # float32 FMA rate measured here on this device
    pass_bytes = nv * (16 + 8) + w["N"] * w["N"] * 8
    pass_flops = 4 * w["W"] ** 2 * nv
    peak, peak_src = measured_peak_hbm()
    fp32 = lmg.fp32_fma_rate() / 1e12
    dom = "grid" if stages["grid"] >= stages["degrid"] else "degrid"
    t_dom = stages[dom] * 1e-3
    achieved = pass_bytes / t_dom / 1e9
    t_hbm = pass_bytes / (peak * 1e9)
    t_alu = pass_flops / (fp32 * 1e12)
    roof = {"kernel": ("k_grid_sweep + k_grid_spill (gridding pass)" if dom == "grid"
                       else "k_degrid_sweep with its output zeroing (degridding pass)"),
            "bound": "hbm" if t_hbm >= t_alu else "alu", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_record(dom),
            "algorithmic_bytes": pass_bytes, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, burst)",
            "fp32_side": {"flops": pass_flops, "peak_tflops": fp32, "achieved_tflops": pass_flops / t_dom / 1e12,
                          "frac": pass_flops / t_dom / 1e12 / fp32,
                          "peak_source": "measured in this process: lmg_fp32_fma_rate (fmaf chains on every SM)",
                          "derivation": "4 W^2 flops per visibility per pass (8 W^2 for gridding plus degridding); "
                                        f"time at peak {1e6 * t_alu:.1f} us against {1e6 * t_hbm:.1f} us for the "
                                        "algorithmic bytes at the HBM peak"}}
    other = "degrid" if dom == "grid" else "grid"
    extra = {"stages_ms": stages, "value_definition": VALUE_DEFINITION,
             "grid_degrid_mvis_s": nv / ((stages["grid"] + stages["degrid"]) * 1e-3) / 1e6,
             "bin_grid_degrid_mvis_s": nv / ((stages["bin"] + stages["grid"] + stages["degrid"]) * 1e-3) / 1e6,
             f"{other}_roofline_frac": pass_bytes / (stages[other] * 1e-3) / 1e9 / peak,
             "timed_wall_s": t_wall}

    line = {"metric": METRIC, "value": value, "unit": "Mvis/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "nvis": nv, "grid": w["N"], "image": w["n_image"], "W": w["W"],
                       "oversample": w["oversample"], "interp": w["interp"],
                       "layout": f"sample-major over {w['tracks']} baselines; binned with that hint "
                                 "(lmg_plan_bin_tracks; stages_ms.bin_plain is the binning without it)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed before every timed step (256 MB write, outside the step's events)"},
            "roofline": roof, "clocks": clk,
            "e2e": {"value": whole_job_mvis(nv, world, e2e_ms), "unit": "Mvis/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": KERNELS_PER_STEP * args.steps}
    line.update(extra)
    if rank == 0 and not args.no_accuracy:
        torch.cuda.synchronize()
        step()
        torch.cuda.synchronize()
        line["accuracy_vs_fp64"] = accuracy(uv, dl, vis, model, img_d.cpu().numpy(), pv_d.cpu().numpy())
    if rank == 0 and not args.no_cpu_baseline:
        P, n, walls, last = oracle_allcore(uv, dl, vis, model, 1, every=2)
        n1, st1 = oracle_single(uv, dl, vis, model, every=8)
        line["cpu_baseline"] = {
            "value": n / walls[0] / 1e6, "unit": "Mvis/s", "cores": P, "kind": "oracle",
            "sample": ALLCORE_TEXT.format(P=P, n=n, frac="every 2nd") + f"; {walls[0]:.1f} s",
            "os_cpu_count": os.cpu_count(), "stage_s_slowest_worker": last,
            "single_core": {"value": n1 / st1["total"] / 1e6, "unit": "Mvis/s", "cores": 1,
                            "grid_degrid_mvis_s": n1 / (st1["grid"] + st1["degrid"]) / 1e6, "stage_s": st1,
                            "sample": f"one oracle step in this process on every 8th visibility ({n1}) with the "
                                      f"full 4096^2 grid; {st1['total']:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------------------
# further workloads: batched channels, differentiable imaging
# ---------------------------------------------------------------------------------------
CHANNELS = dict(n_chan=96, n_ant=64, hours=6.0, f_lo=0.95e9, f_hi=1.05e9, nv_lo=1e5, nv_hi=2e6,
                sizes=(1024, 2048, 4096), Ws=(4, 6, 8), x0=0.5, oversample=1000, n_src=4, noise_sigma=0.1)
CHANNELS_NAME = ("96 frequency channels (0.95-1.05 GHz) of 64-antenna 6 h tracks, visibility counts log-uniform "
                 "in 1e5-2e6, grids drawn from {1024^2, 2048^2, 4096^2}, W from {4, 6, 8}, x0 = 0.5, linear "
                 "tables M_s = 1000, complex64, 4 point sources + noise")


def make_channels():
    from paper_1906_07102_gb300 import synthetic as S
    c = CHANNELS
    g = np.random.default_rng(2024)
    nvs = np.exp(g.uniform(np.log(c["nv_lo"]), np.log(c["nv_hi"]), c["n_chan"])).astype(np.int64)
    Ns = g.choice(c["sizes"], c["n_chan"])
    Ws = g.choice(c["Ws"], c["n_chan"])
    freqs = np.linspace(c["f_lo"], c["f_hi"], c["n_chan"])
    nbl = c["n_ant"] * (c["n_ant"] - 1) // 2
    chans = []
    for k in range(c["n_chan"]):
        n_times = int(-(-nvs[k] // nbl))
        uv = S.array_tracks(n_ant=c["n_ant"], hours=c["hours"], n_times=n_times, freqs_hz=(freqs[k],), seed=0)
        uv = np.ascontiguousarray(uv[:nvs[k]])
        dl = S.pixel_scale_for(uv)
        n_img = int(Ns[k]) // 2
        l, m, f = S.point_source_sky(c["n_src"], 0.45 * n_img * dl, seed=k)
        vis = S.visibilities(uv, l, m, f, noise_sigma=c["noise_sigma"], seed=k).astype(np.complex64)
        chans.append(dict(uv=uv, dl=dl, vis=vis, N=int(Ns[k]), n_img=n_img, W=int(Ws[k])))
    return chans


def _events_ms(step, steps, flush, stream, torch):
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([s.elapsed_time(e) for s, e in zip(starts, ends)]))


def soak(step, flush, stream, torch, t_wall, clocks, steps):
    """Timed steps are often shorter than a useful clock record (nvidia-smi samples every
    100 ms or so): identical steps (L2 flushed the same way) continue after them until the
    window is CLOCK_WINDOW_S long. Stops the clock sampler and returns its record with the
    window and the soak's own time per step."""
    n, per = 0, []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 + t_wall < CLOCK_WINDOW_S:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 0
        a.record(stream)
        while reps < 50 and time.perf_counter() - t0 + t_wall < CLOCK_WINDOW_S:
            flush.zero_()
            step()
            reps += 1
        b.record(stream)
        torch.cuda.synchronize()
        per.append(a.elapsed_time(b) / reps)
        n += reps
    clk = clocks.stop()
    clk["window"] = (f"{steps} timed steps followed by {n} identical steps "
                     f"({t_wall + time.perf_counter() - t0:.2f} s of steps)")
    clk["soak_ms_per_step"] = float(np.mean(per)) if per else None
    return clk


def run_channels(args):
    """Batched channels: tuned, graph-captured batch against sequential single plans."""
    import torch
    from paper_1906_07102_gb300 import lmg
    torch.cuda.set_device(0)
    c = CHANNELS
    chans = make_channels()
    nv_total = int(sum(ch["uv"].shape[0] for ch in chans))
    dev = torch.device("cuda", 0)
    tabs = {W: lmg.Table(W, c["x0"], c["oversample"], "linear") for W in c["Ws"]}
    uvs = [torch.from_numpy(ch["uv"]).to(dev) for ch in chans]
    vis = [torch.from_numpy(ch["vis"]).to(dev) for ch in chans]
    batch = lmg.Batch([tabs[ch["W"]] for ch in chans], [ch["n_img"] for ch in chans], [ch["dl"] for ch in chans],
                      [ch["uv"].shape[0] for ch in chans])
    batch.bin(uvs)
    chosen = batch.tune(vis)
    grids = [torch.empty((ch["N"], ch["N"]), dtype=torch.complex64, device=dev) for ch in chans]
    vout = [torch.empty_like(v) for v in vis]
    plans = []
    for ch, u in zip(chans, uvs):
        p = lmg.Plan(tabs[ch["W"]], ch["n_img"], ch["dl"], ch["uv"].shape[0], "c64")
        p.bin(u)
        plans.append(p)
    grids_s = [torch.empty_like(g) for g in grids]
    vout_s = [torch.empty_like(v) for v in vis]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def batched():
        batch.grid(vis, out=grids)
        batch.degrid(grids, out=vout)

    def sequential():
        for p, v, g, o in zip(plans, vis, grids_s, vout_s):
            p.grid(v, out=g)
            p.degrid(g, out=o)

    for _ in range(max(3, args.warmup)):
        batched()
        sequential()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    clocks.mark()
    t_wall = time.perf_counter()
    ms_b = _events_ms(batched, args.steps, flush, stream, torch)
    t_wall = time.perf_counter() - t_wall
    clk = soak(batched, flush, stream, torch, t_wall, clocks, args.steps)
    ms_s = _events_ms(sequential, args.steps, flush, stream, torch)
    # same accuracy: the batched outputs against the sequential ones
    batched()
    sequential()
    torch.cuda.synchronize()
    d_grid = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(grids, grids_s))
    d_vis = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(vout, vout_s))
    # end to end: visibilities in from pinned host memory, predictions out, every step
    vis_h = [v.cpu().pin_memory() for v in vis]
    out_h = [torch.empty(v.shape, dtype=v.dtype).pin_memory() for v in vis]

    def e2e():
        for d, h in zip(vis, vis_h):
            d.copy_(h, non_blocking=True)
        batched()
        for h, d in zip(out_h, vout):
            h.copy_(d, non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    ms_e = _events_ms(e2e, max(3, min(args.steps, 10)), flush, stream, torch)
    # the batch's imaging and prediction calls as a whole (gridding + pruned transforms +
    # crop, pad + pruned transforms + degridding), for reference beside the sweeps alone
    images = [torch.empty((ch["n_img"], ch["n_img"]), dtype=torch.complex64, device=dev) for ch in chans]
    models = [torch.zeros((ch["n_img"], ch["n_img"]), dtype=torch.complex64, device=dev) for ch in chans]
    for m in models:
        m[m.shape[0] // 2, m.shape[1] // 2] = 1.0
    reps = max(3, min(args.steps, 10))
    batch.dirty_image(vis, out=images)
    batch.predict_vis(models, out=vout)
    ms_dirty = _events_ms(lambda: batch.dirty_image(vis, out=images), reps, flush, stream, torch)
    ms_pred = _events_ms(lambda: batch.predict_vis(models, out=vout), reps, flush, stream, torch)
    sizes = [ch["N"] for ch in chans]
    algo = sum(ch["uv"].shape[0] * 48 + 2 * ch["N"] ** 2 * 8 for ch in chans)
    peak, src = measured_peak_hbm()
    achieved = algo / (ms_b * 1e-3) / 1e9
    n_w = len(set(ch["W"] for ch in chans))
    line = {"metric": "Mvis/s grid+degrid, 96 channels batched (graph-captured, tuned) vs 96 sequential plain calls",
            "value": nv_total / (ms_b * 1e-3) / 1e6, "unit": "Mvis/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CHANNELS_NAME, "nvis": nv_total, "channels": len(chans),
                       "grids": {str(n): sizes.count(n) for n in sorted(set(sizes))},
                       "W": {str(w): sum(ch["W"] == w for ch in chans) for w in sorted(set(ch["W"] for ch in chans))},
                       "tuned": {"rows_per_bin": chosen[0], "records_per_item": chosen[1], "warps": chosen[2],
                                 "tables_in_shared_memory": bool(chosen[3])},
                       "parallelism": "single GPU",
                       "l2": "flushed before every timed step (256 MB write, outside the step's events)"},
            "sequential": {"value": nv_total / (ms_s * 1e-3) / 1e6, "ms_per_step": ms_s,
                           "form": "96 x (lmg_grid + lmg_degrid), one plan per channel"},
            "speedup_vs_sequential": ms_s / ms_b,
            "calls_ms": {"dirty_image": ms_dirty, "predict_vis": ms_pred,
                         "form": "lmg_batch_dirty_image / lmg_batch_predict_vis over all channels (graph replay)"},
            "batched_vs_sequential_rel_diff": {"grid_max_rel_l2": d_grid, "vis_max_rel_l2": d_vis},
            "roofline": {"kernel": "batched step (sweeps + spill + output zeroing, all channels)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_bytes": algo,
                         "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"},
            "clocks": clk, "timed_wall_s": t_wall,
            "e2e": {"value": nv_total / (ms_e * 1e-3) / 1e6, "unit": "Mvis/s",
                    "h2d_bytes_per_step": nv_total * 8, "d2h_bytes_per_step": nv_total * 8},
            "gpu_launches": 4 * n_w * args.steps}
    print(json.dumps(line), flush=True)


AUTOGRAD = dict(n_ant=64, hours=6.0, n_times=384, n_chan=64, f_lo=0.95e9, f_hi=1.05e9, N=4096, n_image=2048,
                x0=0.5, W=8, oversample=1000, n_src=4, noise_sigma=0.1)


def run_autograd(args):
    """Differentiable imaging: forward + backward with all channels in one plan against one
    plan per channel (same loss, same gradient)."""
    import torch
    from paper_1906_07102_gb300 import lmg
    from paper_1906_07102_gb300 import synthetic as S
    torch.cuda.set_device(0)
    a = AUTOGRAD
    freqs = np.linspace(a["f_lo"], a["f_hi"], a["n_chan"])
    uv = S.array_tracks(n_ant=a["n_ant"], hours=a["hours"], n_times=a["n_times"], freqs_hz=freqs, seed=0)
    dl = S.pixel_scale_for(uv)
    l, m, f = S.point_source_sky(a["n_src"], 0.45 * a["n_image"] * dl, seed=0)
    V = S.visibilities(uv, l, m, f, noise_sigma=a["noise_sigma"], seed=0).astype(np.complex64)
    image = S.gaussian_blob_image(a["n_image"], 64, seed=0).astype(np.float32)
    nv = uv.shape[0]
    per = nv // a["n_chan"]
    dev = torch.device("cuda", 0)
    tab = lmg.Table(a["W"], a["x0"], a["oversample"], "linear")
    uv_d = torch.from_numpy(uv).to(dev)
    V_d = torch.from_numpy(V).to(dev)
    img_d = torch.from_numpy(image).to(dev)
    one = lmg.Plan(tab, a["n_image"], dl, nv, "c64")
    one.bin(uv_d)
    plans = []
    for k in range(a["n_chan"]):
        p = lmg.Plan(tab, a["n_image"], dl, per, "c64")
        p.bin(uv_d[k * per:(k + 1) * per])
        plans.append(p)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    grads = {}

    def batched():
        x = img_d.clone().requires_grad_(True)
        r = lmg.predict(x, one) - V_d
        (r.real.double() ** 2 + r.imag.double() ** 2).sum().backward()
        grads["batched"] = x.grad

    def per_channel():
        x = img_d.clone().requires_grad_(True)
        L = 0
        for k, p in enumerate(plans):
            r = lmg.predict(x, p) - V_d[k * per:(k + 1) * per]
            L = L + (r.real.double() ** 2 + r.imag.double() ** 2).sum()
        L.backward()
        grads["per_channel"] = x.grad

    for _ in range(max(3, args.warmup)):
        batched()
        per_channel()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    clocks.mark()
    t_wall = time.perf_counter()
    ms_b = _events_ms(batched, args.steps, flush, stream, torch)
    t_wall = time.perf_counter() - t_wall
    clk = soak(batched, flush, stream, torch, t_wall, clocks, args.steps)
    ms_p = _events_ms(per_channel, args.steps, flush, stream, torch)
    gb, gp = grads["batched"].double(), grads["per_channel"].double()
    diff = float(torch.linalg.vector_norm(gb - gp) / torch.linalg.vector_norm(gp))
    # end to end: image and visibilities in from pinned memory, gradient out
    img_h = torch.from_numpy(image).pin_memory()
    V_h = torch.from_numpy(V).pin_memory()
    g_h = torch.empty(image.shape, dtype=torch.float32).pin_memory()

    def e2e():
        img_d.copy_(img_h, non_blocking=True)
        V_d.copy_(V_h, non_blocking=True)
        batched()
        g_h.copy_(grads["batched"], non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    ms_e = _events_ms(e2e, max(3, min(args.steps, 10)), flush, stream, torch)
    algo = nv * 48 + 2 * a["N"] ** 2 * 8
    peak, src = measured_peak_hbm()
    achieved = algo / (ms_b * 1e-3) / 1e9
    line = {"metric": "Mvis/s forward+backward of ||P I - V||^2 (degrid + grid), all channels in one plan vs one "
                      "plan per channel",
            "value": nv / (ms_b * 1e-3) / 1e6, "unit": "Mvis/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64-antenna tracks, 384 samples x 64 channels (0.95-1.05 GHz), 49.5e6 vis, "
                                   "4096^2 grid, 2048^2 float32 Gaussian-blob image, W=8, M_s=1000",
                       "nvis": nv, "parallelism": "single GPU",
                       "l2": "flushed before every timed step (256 MB write, outside the step's events)"},
            "per_channel": {"value": nv / (ms_p * 1e-3) / 1e6, "ms_per_step": ms_p,
                            "form": "64 plans, loss summed over channels"},
            "speedup_vs_per_channel": ms_p / ms_b,
            "gradient_rel_diff_vs_per_channel": diff,
            "roofline": {"kernel": "forward + backward step", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None, "algorithmic_bytes": algo,
                         "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"},
            "clocks": clk,
            "e2e": {"value": nv / (ms_e * 1e-3) / 1e6, "unit": "Mvis/s",
                    "h2d_bytes_per_step": image.nbytes + V.nbytes, "d2h_bytes_per_step": image.nbytes},
            "gpu_launches": 5 * args.steps}
    print(json.dumps(line), flush=True)


LARGE = dict(n_ant=128, hours=8.0, n_times=768, n_chan=32, f_lo=0.95e9, f_hi=1.05e9, N=8192, n_image=4096, x0=0.5,
             W=12, oversample=1000, n_src=4, noise_sigma=0.1, crop=512, spot=100000)


def run_large(args):
    """Plain against compensated float32 accumulation at W = 12 on an 8192^2 grid."""
    import torch
    from oracle import design as D
    from oracle import imaging as I
    from paper_1906_07102_gb300 import lmg
    from paper_1906_07102_gb300 import synthetic as S
    torch.cuda.set_device(0)
    a = LARGE
    freqs = np.linspace(a["f_lo"], a["f_hi"], a["n_chan"])
    uv = S.array_tracks(n_ant=a["n_ant"], hours=a["hours"], n_times=a["n_times"], freqs_hz=freqs, seed=0)
    dl = S.pixel_scale_for(uv)
    l, m, f = S.point_source_sky(a["n_src"], 0.45 * a["n_image"] * dl, seed=0)
    vis = S.visibilities(uv, l, m, f, noise_sigma=a["noise_sigma"], seed=0)
    model = S.gaussian_blob_image(a["n_image"], 64, seed=0).astype(np.complex128)
    nv = uv.shape[0]
    dev = torch.device("cuda", 0)
    tab = lmg.Table(a["W"], a["x0"], a["oversample"], "linear")
    uv_d = torch.from_numpy(uv).to(dev)
    v64 = torch.from_numpy(vis.astype(np.complex64)).to(dev)
    m64 = torch.from_numpy(model.astype(np.complex64)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    p32 = lmg.Plan(tab, a["n_image"], dl, nv, "c64")
    p32.bin(uv_d)
    grid = torch.empty((a["N"], a["N"]), dtype=torch.complex64, device=dev)
    out = torch.empty_like(v64)
    for _ in range(max(2, args.warmup)):
        p32.grid(v64, out=grid)
        p32.grid(v64, accum="compensated", out=grid)
        p32.degrid(grid, out=out)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 10))
    clocks = Clocks(0)
    clocks.start()
    clocks.mark()
    t_wall = time.perf_counter()
    ms_plain = _events_ms(lambda: p32.grid(v64, out=grid), steps, flush, stream, torch)
    ms_comp = _events_ms(lambda: p32.grid(v64, accum="compensated", out=grid), steps, flush, stream, torch)
    ms_degrid = _events_ms(lambda: p32.degrid(grid, out=out), steps, flush, stream, torch)
    t_wall = time.perf_counter() - t_wall

    def large_step():
        p32.grid(v64, out=grid)
        p32.degrid(grid, out=out)

    clk = soak(large_step, flush, stream, torch, t_wall, clocks, 3 * steps)
    c = a["crop"]
    sl = slice(a["n_image"] // 2 - c // 2, a["n_image"] // 2 + c // 2)
    img_plain = p32.dirty_image(v64)[sl, sl].cpu().numpy()
    img_comp = p32.dirty_image(v64, accum="compensated")[sl, sl].cpu().numpy()
    pv32 = p32.predict_vis(m64).cpu().numpy()
    del p32, grid, out
    torch.cuda.empty_cache()
    # float64 path of the library (kernel parity with the oracle: 1e-12 on shared tables)
    p64 = lmg.Plan(tab, a["n_image"], dl, nv, "c128")
    p64.bin(uv_d)
    img64 = p64.dirty_image(torch.from_numpy(vis).to(dev))[sl, sl].cpu().numpy()
    pv64 = p64.predict_vis(torch.from_numpy(model).to(dev)).cpu().numpy()
    del p64
    torch.cuda.empty_cache()

    def rel(x, ref):
        return float(np.sqrt(np.mean(np.abs(x - ref) ** 2) / np.mean(np.abs(ref) ** 2)))

    # FP64 oracle spot check: predicted visibilities at sampled positions
    k = np.sort(np.random.default_rng(5).choice(nv, a["spot"], replace=False))
    T = D.lm_table(D.least_misfit_h(a["W"], a["x0"] / 2), a["W"], a["x0"] / 2, a["oversample"])
    hv = D.correction_factors(T, a["oversample"], 1, a["W"], I.pixel_coords(a["n_image"], a["N"]))
    uc = I.cells_from_wavelengths(uv[k], a["N"], dl)
    op = I.Plan(uc[:, 0], uc[:, 1], a["W"], a["N"], single_precision_s=False)
    ref_pv = I.degrid(op, T, a["oversample"], 1, I.model_grid(I.pad_correct(model, hv, a["N"])))
    algo = nv * 48 + 2 * a["N"] ** 2 * 8
    peak, src = measured_peak_hbm()
    ms = ms_plain + ms_degrid
    line = {"metric": "Mvis/s grid+degrid at W=12, 8192^2 grid (float32 plain vs compensated accumulation); "
                      "relative RMS error vs FP64",
            "value": nv / (ms * 1e-3) / 1e6, "unit": "Mvis/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "128-antenna 8 h tracks, 768 samples x 32 channels (0.95-1.05 GHz), "
                                   f"{nv} vis, 4 point sources + noise, 8192^2 grid, 4096^2 image, W=12 (QR table), "
                                   "linear table M_s=1000, complex64", "nvis": nv, "parallelism": "single GPU",
                       "l2": "flushed before every timed pass (256 MB write, outside the events)"},
            "stages_ms": {"grid_plain": ms_plain, "grid_compensated": ms_comp, "degrid": ms_degrid},
            "compensated_grid_degrid_mvis_s": nv / ((ms_comp + ms_degrid) * 1e-3) / 1e6,
            "accuracy": {
                "dirty_image_plain_vs_fp64_path": rel(img_plain, img64),
                "dirty_image_compensated_vs_fp64_path": rel(img_comp, img64),
                "predicted_vis_vs_fp64_path": rel(pv32, pv64),
                "predicted_vis_vs_fp64_oracle": rel(pv32[k], ref_pv),
                "fp64_path_predicted_vis_vs_fp64_oracle": rel(pv64[k], ref_pv),
                "sample": f"central {c}^2 of the 4096^2 dirty image against the library's float64 path; "
                          f"{a['spot']} predicted visibilities against the FP64 oracle (full 8192^2 model grid)"},
            "roofline": {"kernel": "grid (plain) + degrid passes", "bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": algo / (ms * 1e-3) / 1e9 / peak, "traffic": None,
                         "algorithmic_bytes": algo, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"},
            "clocks": clk, "gpu_launches": 4 * steps}
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Sweep throughput of the float64 path against the float32 one (Section 5.2: the direct
    calculation of the weights against table lookups, and the W = 14 double-precision
    design), on the 4.1M-visibility tracks; L2 flushed before every timed launch."""
    import torch
    from paper_1906_07102_gb300 import lmg
    torch.cuda.set_device(0)
    uv, dl, vis, model = make_inputs()
    nv = uv.shape[0]
    dev = torch.device("cuda", 0)
    uv_d = torch.from_numpy(uv).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    cases = [("c64", 7, "linear", 1000), ("c128", 7, "linear", 1000), ("c128", 7, "cubic", 20000),
             ("c128", 7, "direct", 4), ("c128", 14, "cubic", 20000)]
    out = []
    ref = {}
    for dt, W, interp, Ms in cases:
        tab = lmg.Table(W, 0.5, Ms, interp)
        plan = lmg.Plan(tab, WORKLOAD["n_image"], dl, nv, dt)
        plan.bin(uv_d)
        cd = torch.complex64 if dt == "c64" else torch.complex128
        v = torch.from_numpy(vis.astype(np.complex64 if dt == "c64" else np.complex128)).to(dev)
        g = torch.empty((WORKLOAD["N"], WORKLOAD["N"]), dtype=cd, device=dev)
        vo = torch.empty_like(v)
        reps = max(3, min(args.steps, 10))
        plan.grid(v, out=g)
        plan.degrid(g, out=vo)
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        clocks.mark()
        t_wall = time.perf_counter()
        tg = _events_ms(lambda: plan.grid(v, out=g), reps, flush, stream, torch)
        plan.grid(v, out=g)
        td = _events_ms(lambda: plan.degrid(g, out=vo), reps, flush, stream, torch)
        t_wall = time.perf_counter() - t_wall

        def case_step():
            plan.grid(v, out=g)
            plan.degrid(g, out=vo)

        clk = soak(case_step, flush, stream, torch, t_wall, clocks, 2 * reps)
        plan.grid(v, out=g)
        plan.degrid(g, out=vo)
        torch.cuda.synchronize()
        gi = g.cpu().numpy()[::64, ::64].astype(np.complex128)
        key = (W,)
        row = {"dtype": dt, "W": W, "interp": interp, "oversample": Ms, "grid_ms": tg, "degrid_ms": td,
               "grid_degrid_mvis_s": nv / ((tg + td) * 1e-3) / 1e6, "clocks": clk}
        if key in ref:  # agreement of the grid with the first float64 case of the same W
            r = ref[key]
            row["grid_rel_diff_vs_" + r[0]] = float(np.sqrt(np.mean(np.abs(gi - r[1]) ** 2) / np.mean(np.abs(r[1]) ** 2)))
        elif dt == "c128":
            ref[key] = (f"{interp}{Ms}", gi)
        out.append(row)
        del plan, g, vo, v
        torch.cuda.empty_cache()
    line = {"workload": "precision", "config": {"workload": WORKLOAD_NAME + " (values used as complex128 for the "
                                                                        "float64 rows)"},
            "unit": "ms per launch pass; Mvis/s", "cases": out}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "channels":
        run_channels(args)
    elif args.workload == "autograd":
        run_autograd(args)
    elif args.workload == "large":
        run_large(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
