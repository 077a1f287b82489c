#!/usr/bin/env python
"""Benchmark: 720p scale-hyperprior encode + decode frames/s on B300.

One step = encode then decode of a batch of 8 synthetic 1280x720 frames
(replicate-padded to 1280x768 inside the codec), N=128, M=192, FP32 chain,
inputs resident in HBM, timed with CUDA events on the codec's stream, with
an L2 flush (a 512 MB write) before every step outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica (frames are independent, the
path has no exchange step); rank 0 prints one JSON line.  --impl reference
times the FP64 CPU oracle on a bounded crop of the same workload.
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

METRIC = "720p hyperprior enc+dec frames/s (FP32 plain vs BF16/FP8/student) at PSNR; p99 ms"
N_CH, M_CH = 128, 192
PAD_H, PAD_W = 768, 1280


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--height", type=int, default=720)
    ap.add_argument("--width", type=int, default=1280)
    ap.add_argument("--conv", default="auto", choices=["auto", "simt"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp8"],
                    help="arithmetic of the timed chain (the precision forms run in any case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision / student / pipelined forms")
    ap.add_argument("--forms", default="all",
                    help="comma-separated forms to run after the FP32 chain (all, or any of: precision (BF16, "
                         "FP8, FP32 with 1DN), substreams, format2, wide, two_streams, student, serving)")
    ap.add_argument("--student-steps", type=int, default=20000, help="training steps of the student form (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of the serving form's workload (0: skip)")
    return ap.parse_args()


def want(args, form):
    """Whether the run includes `form` (--no-forms: none; --forms: a comma list or all)."""
    if args.no_forms:
        return False
    names = {f.strip() for f in args.forms.split(",")}
    return "all" in names or form in names


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- clocks

class _NvmlCtypes:
    """The five read-only NVML calls the clock sampler makes, through ctypes on
    the driver's libnvidia-ml (for hosts without the pynvml package); the
    constants are NVML's public ones."""
    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, r):
        if r != 0:
            raise RuntimeError(f"NVML error {r}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2())

    def nvmlDeviceGetHandleByUUID(self, uuid):
        h = self.c.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByUUID(self.c.c_char_p(uuid.encode()), self.c.byref(h)))
        return h

    def _clock(self, fn, h, kind):
        v = self.c.c_uint()
        self._ok(fn(h, self.c.c_int(kind), self.c.byref(v)))
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h, kind)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h, kind)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        if fn is None:
            fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.c.byref(v)))
        return v.value


class ClockSampler:
    """SM clock and clock-event (throttle) reasons while running, read only.

    NVML (pynvml, else the driver's library through ctypes) polled every 10 ms
    from a thread, the device found by the UUID the CUDA runtime reports (so the
    samples are of the GPU the work runs on, whatever CUDA_VISIBLE_DEVICES says);
    without NVML, nvidia-smi every 50 ms. Nothing is set: only clocks and
    reasons are queried."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.010
    # the reasons a run is judged by, with their NVML bit names
    REASONS = (("hw_slowdown", "HwSlowdown"), ("hw_thermal_slowdown", "HwThermalSlowdown"),
               ("sw_thermal_slowdown", "SwThermalSlowdown"), ("sw_power_cap", "SwPowerCap"))

    def __init__(self, gpu_index, tag="main", nvml=None, uuid=None):
        self.gpu = gpu_index
        self.proc = None
        self.thread = None
        self.nvml = nvml          # a module with pynvml's interface (tests pass a fake)
        self.uuid = uuid
        self.samples = []         # (sm MHz, max sm MHz, reasons bitmask)
        self.source = None
        self.path = os.path.join(tempfile.gettempdir(),
                                 f"lic_bench_clocks_gpu{gpu_index}_{os.getpid()}_{tag}.csv")

    def _nvml_open(self):
        nv = self.nvml
        if nv is None:
            try:
                import pynvml as nv
            except ImportError:
                nv = _NvmlCtypes()
            self.nvml = nv
        nv.nvmlInit()
        uuid = self.uuid
        if uuid is None:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.gpu).uuid)
        h = nv.nvmlDeviceGetHandleByUUID(uuid)
        return nv, h

    def _poll(self, nv, h):
        get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        smax = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while True:
            try:
                self.samples.append((nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM), smax, get_reasons(h)))
            except Exception:
                pass
            if self.stop.wait(self.PERIOD_S):
                break

    def __enter__(self):
        import threading
        try:
            nv, h = self._nvml_open()
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(nv, h), daemon=True)
            self.thread.start()
            self.source = "nvml, 10 ms"
            return self
        except Exception:
            self.thread = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi, 50 ms"
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.thread is not None:
            nv = self.nvml
            sm = [float(x[0]) for x in self.samples]
            smax = float(self.samples[-1][1]) if self.samples else None
            reasons = set()
            for _, _, bits in self.samples:
                for name, nvname in self.REASONS:
                    bit = getattr(nv, "nvmlClocksEventReason" + nvname, None)
                    if bit is None:
                        bit = getattr(nv, "nvmlClocksThrottleReason" + nvname, 0)
                    if bits & bit:
                        reasons.add(name)
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                    "samples": len(sm), "reasons": sorted(reasons), "source": self.source}
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = [n for n, _ in self.REASONS]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons), "source": self.source}


# ------------------------------------------------------------ CPU oracle

_ORACLE_CODEC = None


def _oracle_codec():
    """The FP64 oracle's hyperprior codec (N=128, M=192), built once: its
    tables are set-up, not part of an encode or decode."""
    global _ORACLE_CODEC
    if _ORACLE_CODEC is None:
        import oracle as O
        from paper_2208_01641_b300 import synth
        _ORACLE_CODEC = O.Codec(1, N_CH, M_CH, synth.make_weights(1, N_CH, M_CH))
    return _ORACLE_CODEC


def oracle_frame(seed_frame=0):
    """Seconds the FP64 oracle takes to encode and decode one whole
    synthetic 1280x720 frame (padded to 1280x768 inside the oracle)."""
    import oracle as O
    from paper_2208_01641_b300 import synth
    oc = _oracle_codec()
    x = synth.make_frames(1, 720, 1280, first=seed_frame)
    t0 = time.perf_counter()
    bs, _ = O.encode(oc, x)
    O.decode(oc, bs)
    return time.perf_counter() - t0


STRIPS = PAD_H // 64   # a padded 720p frame is 12 strips of 1280 x 64


def oracle_strip(k, seed_frame=0):
    """Seconds the FP64 oracle takes to encode and decode strip k (rows
    64k .. 64k+63, full width) of the padded synthetic frame, coded as an
    image of its own; twelve strips make one frame's pixels."""
    import numpy as np
    import oracle as O
    from paper_2208_01641_b300 import synth
    oc = _oracle_codec()
    x = synth.make_frames(1, 720, 1280, first=seed_frame)
    x = np.pad(x, ((0, 0), (0, 0), (0, PAD_H - 720), (0, 0)), mode="edge")
    x = np.ascontiguousarray(x[:, :, 64 * k:64 * k + 64])
    t0 = time.perf_counter()
    bs, _ = O.encode(oc, x)
    O.decode(oc, bs)
    return time.perf_counter() - t0


def cpu_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def job_time_ms(local_ms, dist=None):
    """Time of the whole job: the slowest rank's (MAX over ranks of a NCCL or
    gloo group; the local time without a group)."""
    if dist is None:
        return local_ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(frames_per_rank, ws, job_ms):
    """Whole-job frames/s: every rank's frames over the slowest rank's time."""
    return ws * frames_per_rank / (job_ms / 1000.0)


def reference_arm(args, ws, rank):
    """The oracle, as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    for k in range(args.warmup):
        oracle_strip(k % STRIPS)
    times = [oracle_strip((args.warmup + k) % STRIPS) for k in range(args.steps)]
    total = sum(times)
    fps = (args.steps / STRIPS) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "hyperprior N=128 M=192, 8 x 1280x720 frames padded to 1280x768, enc+dec",
                   "global_batch": args.batch, "parallelism": "replicas"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": "FP64 oracle enc+dec of one full-width 1280x64 strip of the padded synthetic "
                                   "720p frame per step (12 strips = one frame's pixels; strips cycle)"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours

def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return

    import numpy as np
    import torch
    import paper_2208_01641_b300 as lic
    from paper_2208_01641_b300 import synth

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    B, H, W = args.batch, args.height, args.width
    impl = lic.CONV_SIMT if args.conv == "simt" else lic.CONV_AUTO
    Wt = synth.make_weights(lic.HYPERPRIOR, N_CH, M_CH)
    prec = {"fp32": lic.FP32, "bf16": lic.BF16, "fp8": lic.FP8}[args.precision]
    codec = lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, Wt, conv_impl=impl, precision=prec)
    frames_np = synth.make_frames(B, H, W, first=8 * rank)
    frames = torch.from_numpy(frames_np).cuda()
    out = torch.empty_like(frames)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    sid = stream.cuda_stream

    def step():
        bs = codec.encode(frames, stream=sid)
        codec.decode(bs, out, stream=sid)
        return bs

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step()
        codec.sync(sid)

    # the step as two CUDA graphs (encode, decode), captured once the warm-up has sized every
    # buffer; each replay runs the same kernels on the same inputs (None: direct launches)
    graphs = capture_step(codec, frames, out, stream)

    # ---- timed region: device time of K steps, L2 flushed before each ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = codec.launch_count()
    sampler = ClockSampler(local)
    with sampler, torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            if graphs:
                graphs[0].replay()
            else:
                bs = codec.encode(frames, stream=sid)
            ev[k][1].record(stream)
            if graphs:
                graphs[1].replay()
            else:
                codec.decode(bs, out, stream=sid)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    status = codec.sync_status(sid)
    if dist:
        dist.barrier()
    # the library counts the launches it makes; a replay makes the captured ones again
    launches = graphs[3] * args.steps if graphs else codec.launch_count() - launches0
    if graphs:
        bs = graphs[2]
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    enc_ms = [a.elapsed_time(b) for a, b, c in ev]
    dec_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = job_time_ms(sum(step_ms), dist)
    value = job_value(B * args.steps, ws, total_ms)
    frame_bytes = bs.sizes()

    # ---- roofline of the dominant kernel: per-launch CUDA events, live ----
    with torch.cuda.stream(stream):
        codec.profile(True)
        for _ in range(3):
            flush.zero_()
            step()
        codec.sync(sid)
        rep = codec.profile_report()
        codec.profile(False)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    roof = roofline(rep, peaks)
    if roof is not None:
        # the tensor pipe's dense rates measured by this library's own probe (back-to-back MMAs
        # on every SM), as context: the roofline's peaks stay the measured BF16 figure (x the
        # nominal ratio for other types)
        try:
            roof["probe_tflops"] = {k: lic.mma_rate(i) for i, k in enumerate(("tf32", "bf16", "e4m3"))}
        except lic.LicError as e:
            roof["probe_tflops"] = {"error": str(e)}
    # the I/O floor, as context: per frame the frame in and out, the bitstream out (encoder) and
    # in (decoder), and the latents y and z written once and read once, all float32
    Hp, Wp = -(-H // 64) * 64, -(-W // 64) * 64
    lat = M_CH * (Hp // 16) * (Wp // 16) + N_CH * (Hp // 64) * (Wp // 64)
    floor_bytes = sum(2 * 12.0 * H * W + 2.0 * fb + 2 * 4.0 * lat for fb in frame_bytes)
    chain = chain_roofline(rep, peaks, total_ms / args.steps, steps=3, floor_bytes=floor_bytes)

    # ---- the BF16 precision form, same workload ----
    forms = {}
    if want(args, "precision") and args.conv == "auto":
        notes = {"bf16": "g_a/g_s convs bf16 x bf16 -> fp32; GDN norms, h_a, h_s, index fp32",
                 "fp8": "g_a/g_s convs e4m3 x e4m3 -> fp32 (per-output-channel weight scales, activations "
                        "x*16; the 192-channel g_s input bf16); GDN norms, h_a, h_s, index fp32"}
        notes["fp32_1dn"] = ("FP32 chain with 1DN (the paper's variant C, read as GDN without channel mixing) "
                             "in place of GDN/IGDN; its own seeded weights")
        W1 = synth.make_weights(lic.HYPERPRIOR, N_CH, M_CH, norm=synth.NORM_1DN)
        for name, prec, wts, norm in (("bf16", lic.BF16, Wt, lic.NORM_GDN), ("fp8", lic.FP8, Wt, lic.NORM_GDN),
                                      ("fp32_1dn", lic.FP32, W1, lic.NORM_1DN)):
            fcodec = lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, wts, precision=prec, norm=norm)
            fms, fstatus = time_steps(fcodec, frames, out, H, W, args.steps, args.warmup, stream, flush)
            forms[name] = {"value": ws * B * args.steps / (sum(fms) / 1000.0), "unit": "frames/s",
                           "ms_per_step": sum(fms) / args.steps,
                           "p99_ms": sorted(fms)[min(len(fms) - 1, int(0.99 * len(fms)))],
                           "decode_status": fstatus, "note": notes[name]}
            # its rooflines: the dominant launch, the dominant launch of the form's own low-precision
            # type, and the whole step, from a profiled pass of three steps (launches timed one by one)
            frep = profile_steps(fcodec, frames, out, stream, flush, 3)
            forms[name]["roofline"] = roofline(frep, peaks)
            own = [r for r in frep if r["name"].endswith({"bf16": ":bf16", "fp8": ":e4m3"}.get(name, ":tc"))]
            forms[name]["roofline_own_type"] = roofline(own, peaks)
            forms[name]["chain_roofline"] = chain_roofline(frep, peaks, forms[name]["ms_per_step"], steps=3)
            if rank == 0 and not args.no_cpu_baseline:
                forms[name]["psnr_vs_oracle_db"] = psnr_vs_oracle(fcodec, wts, B)
                forms[name]["y_maxabs_vs_oracle"] = sampled_errors(fcodec, wts, frames_np, B)
            fcodec.close()

    # ---- the rate cost of interleaving: y substreams of whole latent planes instead of 16-row bands ----
    if want(args, "substreams"):
        cw = lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, Wt, conv_impl=impl, band_rows=PAD_H // 16)
        wms, wstatus = time_steps(cw, frames, out, H, W, args.steps, args.warmup, stream, flush)
        wbytes = cw.encode(frames).sizes()
        forms["fp32_whole_plane_substreams"] = {
            "value": ws * B * args.steps / (sum(wms) / 1000.0), "unit": "frames/s", "decode_status": wstatus,
            "bits_per_pixel": 8.0 * statistics.mean(wbytes) / (H * W),
            "bits_per_pixel_16_row_bands": 8.0 * statistics.mean(frame_bytes) / (H * W),
            "note": "one y substream (32 interleaved states) per latent plane instead of per 16-row band: a third "
                    "of the states to flush (rate), a third of the decoder's warps (parallelism)"}
        cw.close()

    # ---- substream format 2: escape payloads outside the rANS words (decoder-adaptive coder) ----
    if want(args, "format2"):
        forms["fp32_format2"] = format2_form(args, lic, Wt, impl, frames, out, H, W, stream, flush, ws, B,
                                             frame_bytes, rep)

    # ---- the precision form's own configuration: N=192 M=320, 8 x 1920x1080 ----
    if want(args, "wide") and args.conv == "auto":
        forms["precision_1080p_n192_m320"] = wide_form(args, lic, synth, torch, np, stream, flush, rank)

    # ---- frames pipelined: two codecs on two streams, batches in flight together ----
    if want(args, "two_streams"):
        c2 = [lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, Wt, conv_impl=impl) for _ in range(2)]
        st2 = [torch.cuda.Stream() for _ in range(2)]
        outs = [torch.empty_like(frames) for _ in range(2)]
        for _ in range(max(args.warmup, 3)):
            for c_, s_, o_ in zip(c2, st2, outs):
                with torch.cuda.stream(s_):
                    c_.decode(c_.encode(frames, stream=s_.cuda_stream), o_, stream=s_.cuda_stream)
        torch.cuda.synchronize()
        # each codec's step as CUDA graphs on its own stream (direct launches if a capture fails)
        g2 = [capture_step(c_, frames, o_, s_) for c_, s_, o_ in zip(c2, st2, outs)]
        if not all(g2):
            g2 = [None, None]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(st2[0])
        st2[1].wait_event(e0)
        for _ in range(args.steps):
            for c_, s_, o_, g_ in zip(c2, st2, outs, g2):
                with torch.cuda.stream(s_):
                    if g_:
                        g_[0].replay()
                        g_[1].replay()
                    else:
                        c_.decode(c_.encode(frames, stream=s_.cuda_stream), o_, stream=s_.cuda_stream)
        done = torch.cuda.Event()
        done.record(st2[1])
        st2[0].wait_event(done)
        e1.record(st2[0])
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        forms["fp32_two_streams"] = {
            "value": ws * 2 * B * args.steps / (pms / 1000.0), "unit": "frames/s", "ms_per_step": pms / args.steps,
            "decode_status": max(c_.sync_status() for c_ in c2),
            "launch": "CUDA-graph replays" if g2[0] else "direct launches",
            "note": "two codecs on two CUDA streams, each encoding+decoding its own batch of 8: narrow kernels "
                    "of one batch (hyper transforms, entropy coding) overlap the other's (frames pipelined)"}
        for c_ in c2:
            c_.close()

    # ---- the learned form: distilled student g_s, trained here, decoding in place of g_s ----
    if want(args, "student") and args.student_steps > 0:
        forms["student"] = student_form(args, lic, synth, torch, np, Wt, frames, out, stream, flush, ws, peaks)

    # ---- the serving form: 16 Poisson streams of mixed resolutions through the BF16 codec ----
    if want(args, "serving") and args.serve_seconds > 0:
        forms["serving"] = serving_form(args, lic, synth, torch, np, Wt)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        hin = torch.from_numpy(frames_np).pin_memory()
        hout = torch.empty(hin.shape, dtype=torch.float32).pin_memory()
        nbytes = B * 3 * H * W * 4
        # serial: one codec, one stream -- copies and kernels of a step in sequence
        with torch.cuda.stream(stream):
            for _ in range(2):
                bs2 = codec.encode(hin, stream=sid)
                codec.decode(bs2, hout, stream=sid)
            codec.sync(sid)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                bs2 = codec.encode(hin, stream=sid)
                codec.decode(bs2, hout, stream=sid)
            codec.sync(sid)
            serial_fps = ws * B * args.steps / (time.perf_counter() - t0)
        # pipelined through the serving API: eight lanes (codec + stream, the server's maximum), a
        # batch's host copies and latency-bound stages overlap the other lanes' kernels; at most eight
        # batches in flight, each frame's output its own pinned buffer
        depth = 8
        srv = lic.Server(lic.HYPERPRIOR, N_CH, M_CH, Wt, precision=prec, max_batch=B, lanes=depth,
                         max_pending=(depth + 1) * B, graphs=True, max_wait_ms=1e6)
        srv.prepare(H, W)
        outs = [torch.empty(hin.shape, dtype=torch.float32).pin_memory() for _ in range(depth + 1)]

        def run(nsteps):
            done = 0
            for k in range(nsteps):
                while k - done // B >= depth:
                    done += len(srv.poll((depth + 1) * B, wait_ms=100.0))
                for f in range(B):
                    srv.submit(f, hin[f], outs[k % (depth + 1)][f])
            srv.drain(600000)
            srv.poll((depth + 1) * B * nsteps)

        run(2)
        # at least 60 batches: the pipeline's fill and drain (one batch each) stay a small part
        n_e2e = max(args.steps, 60)
        t0 = time.perf_counter()
        run(n_e2e)
        dt = time.perf_counter() - t0
        est = srv.stats()
        srv.close()
        e2e = {"value": ws * B * n_e2e / dt, "unit": "frames/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "serial_value": serial_fps, "graph_replays": est["graph_replays"],
               "batches": n_e2e,
               "note": f"pinned host frames in, decoded frames out to pinned host memory, through the serving "
                       f"API ({args.precision.upper()} codec, {depth} lanes, batches of {B}, at most {depth} in flight, "
                       f"{n_e2e} batches timed from the first submit to the last result); serial_value: one "
                       f"codec on one stream, copies not overlapped"}

    # ---- reconstruction vs the FP64 oracle on sampled windows ----
    psnr = None
    if rank == 0 and not args.no_cpu_baseline:
        psnr = psnr_vs_oracle(codec, Wt, B)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t = oracle_frame()
        cpu = {"value": 1.0 / t, "unit": "frames/s", "cores": cpu_threads(), "kind": "oracle",
               "seconds": t,
               "sample": "FP64 oracle hyperprior enc+dec of one whole synthetic 1280x720 frame (padded to "
                         "1280x768), N=128 M=192, timed once"}

    if rank == 0:
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[args.precision], "data": "synthetic",
            "config": {"workload": "hyperprior N=128 M=192, 8 x 1280x720 frames padded to 1280x768, enc+dec",
                       "global_batch": B * ws, "seq_len": None, "parallelism": f"replicas{ws}",
                       "conv": args.conv, "precision": args.precision,
                       "l2": "512 MB write before every step, outside the timed events",
                       "launch": ("CUDA-graph replays of the encode and the decode, captured once after the warm-up"
                                  if graphs else "direct launches")},
            "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
            "enc_fps": B * args.steps / (sum(enc_ms) / 1000), "dec_fps": B * args.steps / (sum(dec_ms) / 1000),
            "paper_context": PAPER_CONTEXT,
            "bits_per_pixel": 8.0 * statistics.mean(frame_bytes) / (H * W),
            "psnr_vs_oracle_db": psnr if psnr is None or psnr < 1e9 else "inf", "decode_status": status,
            "roofline": roof, "chain_roofline": chain, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": sampler.summary(), "forms": forms, "kernels": rep,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


STUDENT_C = 64
STUDENT_POOL = 16            # teacher frames the training crops are drawn from
STUDENT_POOL_FIRST = 3000    # their frame seeds
STUDENT_BATCH, STUDENT_CROP = 16, 256
STUDENT_HALO = 0             # latent context around each crop (2 measured: lower training loss, no better PSNR)


def student_form(args, lic, synth, torch, np, Wt, frames, out, stream, flush, ws, peaks):
    """Train the student g_s (192->64->64->64->3 transposed convs, ReLU) on
    (y_hat, x_hat) pairs of the factorized N=128/M=192 codec (16 seeded 720p
    frames), Adam lr 1e-4, batch 16 random 256x256 crops; then decode the
    hyperprior codec's 720p batch (same g_s parameters) with the student:
    per-frame PSNR against the teacher (checked decode, fallback below 35 dB)
    and enc+dec frames/s with the student in place of g_s."""
    H, W = frames.shape[2], frames.shape[3]
    B = frames.shape[0]
    Hy, Wy = PAD_H // 16, PAD_W // 16
    teacher = lic.Codec(lic.FACTORIZED, N_CH, M_CH, synth.make_weights(lic.FACTORIZED, N_CH, M_CH))
    pool_y = torch.empty(STUDENT_POOL, M_CH, Hy, Wy, device="cuda")
    pool_x = torch.empty(STUDENT_POOL, 3, PAD_H, PAD_W, device="cuda")
    for i in range(0, STUDENT_POOL, 8):
        fr = torch.from_numpy(synth.make_frames(8, H, W, first=STUDENT_POOL_FIRST + i)).cuda()
        o = torch.empty_like(fr)
        teacher.decode(teacher.encode(fr), o)
        teacher.read_tensor(lic.T_YHAT, pool_y[i:i + 8])
        teacher.read_tensor(lic.T_XPRE, pool_x[i:i + 8])
    st = lic.Student(synth.make_student_weights(M_CH, STUDENT_C), M_CH, STUDENT_C, max_batch=STUDENT_BATCH,
                     crop=STUDENT_CROP, lr=1e-4, precision=lic.BF16, halo=STUDENT_HALO)
    steps = args.student_steps
    win = STUDENT_CROP // 16 + 2 * STUDENT_HALO
    crops = [synth.draw_crops(k, STUDENT_BATCH, STUDENT_POOL, Hy, Wy, win) for k in range(steps)]
    probe = synth.draw_crops(10 ** 6, STUDENT_BATCH, STUDENT_POOL, Hy, Wy, win)
    sid = stream.cuda_stream
    with torch.cuda.stream(stream):
        loss0 = st.grad(pool_y, pool_x, probe, stream=sid)
        warm = min(5, steps)
        for k in range(warm):
            st.step(pool_y, pool_x, crops[k], stream=sid)
        l0 = st.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(warm, steps):
            st.step(pool_y, pool_x, crops[k], stream=sid)
        e1.record(stream)
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1)
        timed_steps = steps - warm
        launches_per_step = (st.launch_count() - l0) / max(1, timed_steps)
        loss1 = st.grad(pool_y, pool_x, probe, stream=sid)
        st.profile(True)
        st.step(pool_y, pool_x, crops[-1], stream=sid)
        rep = st.profile_report()
        st.profile(False)
    train_flop = sum(r["flop"] for r in rep if r["name"] != "student.adam")
    top = max(rep, key=lambda r: r["ms"])
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    top_ach = top["flop"] / top["launches"] / (top["ms"] / top["launches"] * 1e-3) / 1e12
    if top["name"].endswith(":tc"):
        top_peak, top_bound = peaks.get("bf16_tflops", 1800.0), "tensor"
        top_note = "bf16 tcgen05 kernel against the measured dense BF16 peak"
    else:
        top_peak, top_bound = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12, "alu"
        top_note = "CUDA-core FP32 FMA peak: 148 SMs x 128 lanes x 2 x max SM clock"

    # the codec the pairs came from, checked on the held-out batch (the same frames as below)
    fbs = teacher.encode(frames)
    teacher.set_student(st, min_psnr_db=35.0, checked=True)
    teacher.decode(fbs, out)
    _, ffall, fpsnrs = teacher.student_report()
    teacher.close()
    # the hyperprior codec decoding with the student: checked (per-frame PSNR vs the teacher), then timed
    codec = lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, Wt)
    bs = codec.encode(frames)
    codec.decode(bs, out)
    codec.set_student(st, min_psnr_db=35.0, checked=True)
    codec.decode(bs, out)
    nchk, nfall, psnrs = codec.student_report()
    codec.set_student(st, checked=False)
    fms, fstatus = time_steps(codec, frames, out, H, W, args.steps, args.warmup, stream, flush)
    # decode alone, student vs teacher g_s
    dec = {}
    for name, s_ in (("student", st), ("teacher", None)):
        codec.set_student(s_)
        with torch.cuda.stream(stream):
            for _ in range(3):
                codec.decode(bs, out, stream=sid)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            ev0.record(stream)
            for _ in range(args.steps):
                codec.decode(bs, out, stream=sid)
            ev1.record(stream)
            torch.cuda.synchronize()
        dec[name] = B * args.steps / (ev0.elapsed_time(ev1) / 1000.0)
    codec.close()
    st.close()
    return {
        "value": ws * B * args.steps / (sum(fms) / 1000.0), "unit": "frames/s", "ms_per_step": sum(fms) / args.steps,
        "p99_ms": sorted(fms)[min(len(fms) - 1, int(0.99 * len(fms)))], "decode_status": fstatus,
        "psnr_vs_teacher_db": [round(float(p), 3) for p in psnrs], "frames_checked": nchk,
        "fallbacks_below_35db": nfall,
        "psnr_vs_teacher_factorized_db": [round(float(p), 3) for p in fpsnrs],
        "fallbacks_below_35db_factorized": ffall,
        "decode_fps_student": dec["student"], "decode_fps_teacher": dec["teacher"],
        "train": {"steps": steps, "batch": STUDENT_BATCH, "crop": STUDENT_CROP, "halo_latents": STUDENT_HALO,
                  "lr": 1e-4,
                  "ms_per_step": train_ms / max(1, timed_steps),
                  "crops_per_s": STUDENT_BATCH * timed_steps / (train_ms / 1000.0),
                  "tflops": train_flop / (train_ms / max(1, timed_steps) * 1e-3) / 1e12,
                  "launches_per_step": launches_per_step,
                  "probe_loss_before": loss0, "probe_loss_after": loss1,
                  "pool": f"{STUDENT_POOL} seeded 1280x720 frames through the factorized N=128 M=192 codec"},
        "roofline": {"kernel": top["name"], "bound": top_bound, "achieved": top_ach, "peak": top_peak,
                     "unit": "TFLOP/s", "frac": top_ach / top_peak, "traffic": None, "note": top_note},
        "kernels": rep,
        "note": "student g_s (4 transposed convs 192->64->64->64->3, ReLU, no IGDN), BF16 form: the 64-channel "
                "convs and their input gradients on tcgen05 (bf16 x bf16 -> fp32), weight/bias gradients, the "
                "3-channel layer and Adam in fp32 on CUDA cores; trained on the GPU, decoding the hyperprior "
                "codec in place of g_s",
    }


def serving_form(args, lic, synth, torch, np, Wt):
    """16 streams at 30 frames/s each, Poisson arrivals (seed 7): 6 x 640x480,
    6 x 1280x720, 4 x 1920x1080, submitted in real time to the serving
    runtime (hyperprior N=128 M=192, BF16 form, batches of up to 8 per
    resolution, 2 lanes per resolution, CUDA-graph replays, 40 GB budget);
    frames come from pinned host memory, bitstreams and reconstructions stay
    on the device.  Latency = completion callback - submit, per frame."""
    arrivals = synth.poisson_arrivals(args.serve_seconds)
    shapes = sorted({(a[2], a[3]) for a in arrivals})
    pool = {s: [torch.from_numpy(synth.make_frame(5000 + 10 * k + j, *s)).pin_memory() for j in range(2)]
            for k, s in enumerate(shapes)}
    srv = lic.Server(lic.HYPERPRIOR, N_CH, M_CH, Wt, precision=lic.BF16, max_batch=8, lanes=2, max_pending=1 << 16,
                     graphs=True, max_wait_ms=4.0, hbm_budget=40 << 30)
    for s in shapes:
        srv.prepare(*s)
    # warm every lane once outside the measured workload
    for s in shapes:
        for j in range(16):
            srv.submit(0, pool[s][j % 2])
    srv.drain(120000)
    srv.poll(4096)
    base = srv.stats()
    results, refused = [], 0
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), tag="serving")
    with sampler:
        t0 = time.perf_counter()
        for i, (t, sid, H, W) in enumerate(arrivals):
            d = t0 + t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            try:
                srv.submit(sid, pool[(H, W)][i % 2])
            except lic.LicError:
                refused += 1
            if i % 64 == 0:
                results += srv.poll(4096)
        srv.drain(120000)
        results += srv.poll(1 << 16)
    st = srv.stats()
    # capacity: the same frames submitted all at once (full batches, every lane busy)
    sat = []
    c0 = srv.clock_ms()
    for i, (t, sid, H, W) in enumerate(arrivals):
        srv.submit(sid, pool[(H, W)][i % 2])
    srv.drain(300000)
    sat = srv.poll(1 << 16)
    sat_span_s = (max(r["t_done_ms"] for r in sat) - c0) / 1000.0
    srv.close()
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in results])
    span_s = (max(r["t_done_ms"] for r in results) - min(r["t_submit_ms"] for r in results)) / 1000.0
    per_res = {}
    for s in shapes:
        ls = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in results if (r["H"], r["W"]) == s])
        per_res[f"{s[1]}x{s[0]}"] = {"frames": int(ls.size), "p50_ms": float(np.percentile(ls, 50)),
                                    "p99_ms": float(np.percentile(ls, 99))}
    return {
        "value": len(results) / span_s, "unit": "frames/s", "offered_fps": len(arrivals) / args.serve_seconds,
        "capacity_fps": len(sat) / sat_span_s,
        "capacity_mp_per_s": sum(r["H"] * r["W"] for r in sat) / sat_span_s / 1e6,
        "frames": len(results), "refused": refused, "errors": int(sum(r["status"] != 0 for r in results)),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)), "per_resolution": per_res,
        "batches": st["batches"] - base["batches"], "graph_replays": st["graph_replays"] - base["graph_replays"],
        "mean_batch": len(results) / max(1, st["batches"] - base["batches"]), "device_bytes": st["device_bytes"],
        "clocks": sampler.summary(),
        "note": "hyperprior N=128 M=192 BF16 form; 16 Poisson(30/s) streams for %.0f s, seed 7; frames from pinned "
                "host memory, bitstreams and reconstructions device-resident; latency = submit -> completion"
                % args.serve_seconds,
    }


def wide_form(args, lic, synth, torch, np, stream, flush, rank):
    """Scale hyperprior N=192 M=320 on 8 synthetic 1920x1080 frames (padded to
    1920x1088): FP32 and BF16 enc+dec frames/s; for BF16 the PSNR of x_hat
    against the FP64 oracle's g_s on sampled windows and max |y - y64| on a
    crop interior; for both, encoder and decoder scale indices compared
    element by element; FP8 likewise (e4m3 operands for the 192-channel
    inputs, weights zero-padded per tap to whole 128-channel chunks; the
    320-channel g_s input stays bf16)."""
    N3, M3, H3, W3, B3 = 192, 320, 1080, 1920, 8
    Hp3, Wp3 = 1088, 1920
    Wt3 = synth.make_weights(lic.HYPERPRIOR, N3, M3)
    distinct = synth.make_frames(4, H3, W3, first=200)
    fr_np = np.concatenate([distinct, distinct])
    fr = torch.from_numpy(fr_np).cuda()
    out = torch.empty_like(fr)
    res = {}
    for name, prec in (("fp32", lic.FP32), ("bf16", lic.BF16), ("fp8", lic.FP8)):
        c = lic.Codec(lic.HYPERPRIOR, N3, M3, Wt3, precision=prec)
        fms, status = time_steps(c, fr, out, H3, W3, args.steps, args.warmup, stream, flush)
        bs = c.encode(fr)
        c.sync()
        idx_e = torch.empty(B3, M3, Hp3 // 16, Wp3 // 16, dtype=torch.uint8, device="cuda")
        idx_d = torch.empty_like(idx_e)
        c.read_tensor(lic.T_IDX, idx_e)
        c.decode(bs, out)
        st = c.sync_status()
        c.read_tensor(lic.T_IDX, idx_d)
        r = {"value": B3 * args.steps / (sum(fms) / 1000.0), "unit": "frames/s",
             "ms_per_step": sum(fms) / args.steps, "p99_ms": sorted(fms)[min(len(fms) - 1, int(0.99 * len(fms)))],
             "decode_status": max(status, st), "indices_identical_enc_dec": bool(torch.equal(idx_e, idx_d))}
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        rep3 = profile_steps(c, fr, out, stream, flush, 1)
        r["roofline"] = roofline(rep3, peaks, steps=1)
        own = [q for q in rep3 if q["name"].endswith({"bf16": ":bf16", "fp8": ":e4m3"}.get(name, ":tc"))]
        r["roofline_own_type"] = roofline(own, peaks, steps=1)
        r["chain_roofline"] = chain_roofline(rep3, peaks, r["ms_per_step"], steps=1)
        if prec != lic.FP32 and rank == 0 and not args.no_cpu_baseline:
            r["psnr_vs_oracle_db"] = psnr_vs_oracle(c, Wt3, B3, M3, Hp3, Wp3)
            r["y_maxabs_vs_oracle"] = sampled_errors(c, Wt3, fr_np, B3, M3, Hp3, Wp3)
        c.close()
        res[name] = r
    res["note"] = ("hyperprior N=192 M=320, 8 x 1920x1080 (4 seeded frames twice) padded to 1920x1088; the 320-wide "
                   "layers as tensor-core column slices (192 + 128); BF16 GDN/IGDN unfused at 192 channels")
    return res


def entropy_ms(codec, frames, out, stream):
    """Per-launch device time (ms) of the entropy kernels in one profiled
    encode + decode step: {name: ms per launch}."""
    sid = stream.cuda_stream
    codec.profile(True)
    bs = codec.encode(frames, stream=sid)
    codec.decode(bs, out, stream=sid)
    codec.sync(sid)
    rep = codec.profile_report()
    codec.profile(False)
    return {r["name"]: r["ms"] / r["launches"] for r in rep if r["name"].startswith("rans_")}


def format2_form(args, lic, Wt, impl, frames, out, H, W, stream, flush, ws, B, frame_bytes, rep):
    """Format 2 with whole latent planes as y substreams, no resume records
    (the bench batch has enough planes to fill the GPU), against format 1's
    16-row bands: frames/s, bits per pixel, entropy kernel times; and the
    same with a record every 40 groups (a 16-row band's worth at 720p) for a
    decoder short of planes."""
    out_f = {}
    for name, S in (("whole_planes", 0), ("whole_planes_records40", 40)):
        c = lic.Codec(lic.HYPERPRIOR, N_CH, M_CH, Wt, conv_impl=impl, band_rows=PAD_H // 16, format=lic.FORMAT_2,
                      resume_groups=S)
        ms, status = time_steps(c, frames, out, H, W, args.steps, args.warmup, stream, flush)
        sizes = c.encode(frames).sizes()
        ent = entropy_ms(c, frames, out, stream)
        out_f[name] = {"value": ws * B * args.steps / (sum(ms) / 1000.0), "unit": "frames/s",
                       "ms_per_step": sum(ms) / args.steps, "decode_status": status,
                       "bits_per_pixel": 8.0 * statistics.mean(sizes) / (H * W), "entropy_ms": ent}
        c.close()
    v1 = {r["name"]: r["ms"] / r["launches"] for r in rep if r["name"].startswith("rans_")}
    out_f["format1_16_row_bands"] = {"bits_per_pixel": 8.0 * statistics.mean(frame_bytes) / (H * W),
                                     "entropy_ms": v1}
    out_f["note"] = ("format 2: an escape is the escape symbol alone in the rANS words, its payload and count "
                     "nibbles in sections after them, so a warp decodes every group of 32 symbols in one step; "
                     "whole latent planes as substreams (one 32-state flush per plane); records: resume points "
                     "a decoder may use to split a plane into parallel segments (their bytes counted here)")
    return out_f


def profile_steps(codec, frames, out, stream, flush, n):
    """The library's per-launch report (name, launches, ms, algorithmic flop and
    bytes) over n encode+decode steps, each launch timed with its own events (the
    phases of a transposed conv then run one after another), L2 flushed before
    each step."""
    import torch
    sid = stream.cuda_stream
    with torch.cuda.stream(stream):
        codec.profile(True)
        for _ in range(n):
            flush.zero_()
            bs = codec.encode(frames, stream=sid)
            codec.decode(bs, out, stream=sid)
        codec.sync(sid)
        rep = codec.profile_report()
        codec.profile(False)
    return rep


def capture_step(codec, frames, out, stream):
    """One encode and one decode of the batch captured as two CUDA graphs on
    `stream` (after a warm-up, so the library allocates nothing while capturing):
    (encode graph, decode graph, the captured bitstreams, launches a step), or None
    if the capture fails (the caller then launches directly)."""
    import torch
    sid = stream.cuda_stream
    try:
        ge, gd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        l0 = codec.launch_count()
        with torch.cuda.graph(ge, stream=stream):
            bs = codec.encode(frames, stream=sid)
        with torch.cuda.graph(gd, stream=stream):
            codec.decode(bs, out, stream=sid)
        n = codec.launch_count() - l0
        with torch.cuda.stream(stream):
            ge.replay()
            gd.replay()
        torch.cuda.synchronize()
        return ge, gd, bs, n
    except Exception:
        torch.cuda.synchronize()
        return None


def time_steps(codec, frames, out, H, W, steps, warmup, stream, flush):
    """Device time (ms) of `steps` encode+decode steps after `warmup`, L2
    flushed before each step outside the events; the step replayed as CUDA
    graphs where it can be captured."""
    import torch
    sid = stream.cuda_stream
    with torch.cuda.stream(stream):
        for _ in range(max(warmup, 3)):
            bs = codec.encode(frames, stream=sid)
            codec.decode(bs, out, stream=sid)
        codec.sync(sid)
    graphs = capture_step(codec, frames, out, stream)
    with torch.cuda.stream(stream):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            if graphs:
                graphs[0].replay()
                graphs[1].replay()
            else:
                bs = codec.encode(frames, stream=sid)
                codec.decode(bs, out, stream=sid)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], codec.sync_status(sid)


def sampled_errors(codec, Wt, frames_np, B, M=M_CH, Hp=PAD_H, Wp=PAD_W):
    """Errors of a form against the FP64 oracle on sampled crops of the last
    encode/decode: max |y - y64| on the interior of a 192x192 crop (g_a's
    receptive field inside the crop) and PSNR of x_hat against the oracle's
    g_s on two 12x12-latent windows of the decoded symbols."""
    import numpy as np
    import oracle as O
    import paper_2208_01641_b300 as lic
    xp = np.pad(frames_np, ((0, 0), (0, 0), (0, Hp - frames_np.shape[2]), (0, Wp - frames_np.shape[3])),
                mode="edge")
    y = np.zeros((B, M, Hp // 16, Wp // 16), np.float32)
    bs = codec.encode(__import__("torch").from_numpy(frames_np).cuda())
    codec.sync()
    codec.read_tensor(lic.T_Y, y)
    crop = xp[0:1, :, 256:448, 512:704]
    ry = O.g_a(Wt, crop)[0]
    yerr = float(np.abs(y[0, :, 16:28, 32:44][:, 4:8, 4:8] - ry[:, 4:8, 4:8]).max())
    return yerr


def roofline(rep, peaks, steps=3):
    """Dominant launch name by total time; achieved = algorithmic work per
    launch / mean launch time; peak from MEASURED_PEAKS.json (rep covers
    `steps` steps)."""
    if not rep:
        return None
    top = max(rep, key=lambda r: r["ms"])
    per_ms = top["ms"] / top["launches"]
    hbm = peaks.get("hbm_gbs", 6400.0)
    bf16 = peaks.get("bf16_tflops", 1800.0)
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    name = top["name"]
    extra = {}
    if name.endswith(":tc"):
        # TF32 tensor peak = measured BF16 dense x nominal TF32/BF16 ratio (1.1/2.25)
        peak = bf16 * 1.1 / 2.25
        ach = top["flop"] / top["launches"] / (per_ms * 1e-3) / 1e12
        bound, unit = "tensor", "TFLOP/s"
        note = ("FP32-accurate 3xTF32 on tcgen05: algorithmic FP32 flops over the TF32 peak (measured BF16 "
                "x 1.1/2.25); three TF32 MMAs per product bound the algorithmic rate at a third of it")
        extra = {"ceiling_3xtf32": peak / 3, "frac_of_3xtf32_ceiling": ach / (peak / 3)}
    elif name.endswith((":bf16", ":e4m3")):
        # BF16: the measured dense BF16 peak; e4m3: that x the nominal FP8/BF16 ratio (4.5/2.25)
        peak = bf16 * (2.0 if name.endswith(":e4m3") else 1.0)
        ach = top["flop"] / top["launches"] / (per_ms * 1e-3) / 1e12
        bound, unit = "tensor", "TFLOP/s"
        note = "low-precision tcgen05 MMA with FP32 accumulation; algorithmic flops over the dense peak of its type"
    elif top["flop"] > 0:
        # FP32 FMA: 148 SMs x 128 lanes x 2 flop x max SM clock
        peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = top["flop"] / top["launches"] / (per_ms * 1e-3) / 1e12
        bound, unit = "alu", "TFLOP/s"
        note = "CUDA-core FP32 FMA peak: 148 SMs x 128 lanes x 2 x max SM clock"
    else:
        peak = hbm
        ach = top["bytes"] / top["launches"] / (per_ms * 1e-3) / 1e9
        bound, unit = "hbm", "GB/s"
        note = "measured HBM copy bandwidth"
    out = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
           "traffic": TRAFFIC.get(name), "launch_ms": per_ms, "launches_per_step": top["launches"] / steps,
           "note": note, "peak_source": "MEASURED_PEAKS.json" if peaks else "fallback"}
    out.update(extra)
    return out


def chain_roofline(rep, peaks, measured_ms, steps, floor_bytes=None):
    """The whole step against its roofline: T_roof = sum over launches of
    max(algorithmic FLOP / the launch's peak, algorithmic bytes / HBM), per
    step (rep covers `steps` steps, timed launch by launch); frac = T_roof /
    the measured step time.  Peaks: FP32-accurate 3xTF32 = a third of the TF32
    peak (measured BF16 x 1.1/2.25), BF16 measured, e4m3 2x BF16, CUDA-core
    FP32 = 148 x 128 x 2 x max SM clock, HBM measured."""
    if not rep:
        return None
    hbm = peaks.get("hbm_gbs", 6400.0) * 1e9
    bf16 = peaks.get("bf16_tflops", 1800.0) * 1e12
    fma = 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6
    t_roof = t_flop = t_mem = 0.0
    for r in rep:
        n = r["name"]
        peak = (bf16 * 1.1 / 2.25 / 3 if n.endswith(":tc") else bf16 if n.endswith(":bf16")
                else 2 * bf16 if n.endswith(":e4m3") else fma)
        tf = r["flop"] / peak
        tm = r["bytes"] / hbm
        t_roof += max(tf, tm)
        t_flop += tf
        t_mem += tm
    t_roof_ms = t_roof * 1e3 / steps
    return {"t_roof_ms": t_roof_ms, "t_measured_ms": measured_ms, "frac": t_roof_ms / measured_ms,
            "t_compute_ms": t_flop * 1e3 / steps, "t_hbm_ms": t_mem * 1e3 / steps,
            "t_io_floor_ms": None if floor_bytes is None else floor_bytes / hbm * 1e3,
            "note": "sum over the step's launches of max(FLOP / peak of the launch's arithmetic, bytes / "
                    "measured HBM); algorithmic FLOP and bytes as the library counts them; FP32 convs "
                    "against the 3xTF32 ceiling (a third of the TF32 peak)",
            "peak_source": "MEASURED_PEAKS.json" if peaks else "fallback"}


# The paper's own figures for this codec and frame size (Table 4: scale hyperprior, N=128 M=192,
# 1280x720, FP16, encoder and decoder timed separately, per-frame latency), with the hardware it
# names; context only (another machine, another precision, no combined enc+dec figure)
PAPER_CONTEXT = {
    "source": "Table 4 (scale hyperprior, 1280x720)",
    "hardware": "Dell T630: 2x Xeon E5-2680 v4 + RTX 2080 Ti; TensorRT FP16 transforms, CPU entropy coding",
    "pipelined_gdn": {"enc_fps": 279, "dec_fps": 157, "enc_latency_ms": 36, "dec_latency_ms": 33},
    "pipelined_1dn": {"enc_fps": 281, "dec_fps": 161, "enc_latency_ms": 36, "dec_latency_ms": 37},
    "baseline_pytorch_fp16": {"enc_fps": 11, "dec_fps": 16, "enc_latency_ms": 86, "dec_latency_ms": 61},
}


# DRAM bytes (read + write) per launch of the dominant kernels, from the ncu
# captures summarised in profiles/ (None until a capture of the current build)
TRAFFIC = {
    # conv_tcx_kernel, ncu on one batch-1 launch: 130.9 MB read + 13.5 MB written,
    # x8 for the batch-8 launch (traffic grows with the tiles)
    "g_a.conv1+gdn1:tc": 8 * 144.396800e6,
}


def psnr_vs_oracle(codec, Wt, B, M=M_CH, Hp=PAD_H, Wp=PAD_W):
    """Decoder output vs the oracle's g_s on two 12x12-latent windows of the
    decoded symbols of the last batch (64x64 interior pixels each)."""
    import numpy as np
    import oracle as O
    import paper_2208_01641_b300 as lic
    sy = np.zeros((B, M, Hp // 16, Wp // 16), np.int32)
    xpre = np.zeros((B, 3, Hp, Wp), np.float32)
    codec.read_tensor(lic.T_SY, sy)
    codec.read_tensor(lic.T_XPRE, xpre)
    se, n = 0.0, 0
    for (b, iy, ix) in [(0, 20, 30), (B - 1, 30, 60)]:
        win = sy[b:b + 1, :, iy:iy + 12, ix:ix + 12].astype(np.float32)
        rx = np.clip(O.g_s(Wt, win)[0][:, 64:128, 64:128], 0, 1)
        gx = np.clip(xpre[b, :, 16 * iy + 64:16 * iy + 128, 16 * ix + 64:16 * ix + 128], 0, 1)
        se += float(((gx - rx) ** 2).sum())
        n += gx.size
    mse = se / n
    return 1e10 if mse == 0 else float(10 * np.log10(1.0 / mse))


if __name__ == "__main__":
    main()
