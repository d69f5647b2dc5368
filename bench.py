"""Benchmark: 1080p CVC encode + decode throughput on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: seeded synthetic 1920x1080 RGB video (12 textured moving objects on
a smooth background, Gaussian noise sigma 3), YCoCg-R + 4:2:0, contourlet
transform with 5 LP levels (CDF 9/7) and 32/16/16/8/8 directions, step 8
(QPH 8, QPL 1), key frame every 10 frames, RLE bitstream.  One step encodes
and decodes one frame of every stream this rank serves.  The headline value
is the batched form (--batch concurrent 1080p streams coded by one
cvc_batch_step, i.e. one CUDA-graph launch per step); the plain per-frame
path (one cvc_encode_frame + one cvc_decode_frame per frame) is reported
beside it under "plain".

N > 1 (torchrun): every rank serves its own independent streams (the codec
shards by stream; there is no exchange step), so scaling is weak.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a horizontal band of the same frames and decomposition).
"""
import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_, H_, LEVELS, DIRS, QPH, QPL, KINT = 1920, 1080, 5, [5, 4, 4, 3, 3], 8, 1, 10
METRIC = "1080p encode+decode frames/s"
UNIT = "frames/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
CSRC = os.path.join(ROOT, "paper_1510_00561_b300", "csrc")
# Counters of one ncu capture of a batched 1080p step (4 streams), per frame:
# the DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of each
# stage's launches and the warp instructions (smsp__inst_executed.sum)
# of the whole step.  They hold only for the kernel sources they were taken on:
# `sources_sha256` is kernel_sources_sha() of that build, and the bench reports
# them (roofline.traffic, roofline.alu) only while the sources still match.
CAPTURE = {"sources_sha256": "8651f8cdacce8d26db0683ad0cff24b3f0409375de767000e01eb64c5f1c21ef",
           "dram_per_frame": {"colour_fwd": 6475392,
                              "lp_analysis": 20901440,
                              "dfb_analysis": 81866880,
                              "quantise_kp": 33368576,
                              "rle_stream": 17114624,
                              "parse_unrle": 3723200,
                              "unquantise_kp": 28115776,
                              "dfb_synthesis": 82856192,
                              "lp_synthesis": 29105856,
                              "colour_inv": 12526336,
                              "step": 316057600},
           "warp_inst_per_frame": 162596834,
           "profile": "profiles/launches_1080p_batched.md (ncu, 4 streams, one batched step)"}
# issue rate of one SM sub-partition: one warp instruction per cycle
SMSP_PER_SM, N_SM = 4, 148


def kernel_sources_sha():
    """SHA-256 over the library's CUDA sources (file names and contents, sorted)."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            with open(os.path.join(CSRC, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def host_info():
    """nproc and the CPU model of this host"""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _gen_frames(seed, n, start=0):
    from paper_1510_00561_b300 import synthetic as S
    v = S.SyntheticVideo(S.spec_for(W_, H_, seed=seed))
    return [v.frame(start + t) for t in range(n)]


def _gen_one(args):
    seed, t = args
    from paper_1510_00561_b300 import synthetic as S
    return S.SyntheticVideo(S.spec_for(W_, H_, seed=seed)).frame(t)


def make_frames(seed, n):
    """Frames of one stream, drawn in a spawn pool (safe before or after CUDA init)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = max(1, min(n, (os.cpu_count() or 2) - 1, 16))
    if workers == 1:
        return _gen_frames(seed, n)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_one, [(seed, t) for t in range(n)]))


def _gen_sized(args):
    w, h, seed, t = args
    from paper_1510_00561_b300 import synthetic as S
    return S.SyntheticVideo(S.spec_for(w, h, seed=seed)).frame(t)


def make_frames_sized(jobs):
    """frames for a list of (width, height, seed, index), drawn in a spawn pool"""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = max(1, min(len(jobs), (os.cpu_count() or 2) - 1, 16))
    if workers == 1:
        return [_gen_sized(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_sized, jobs))


def combine_ranks(local_ms, local_units, dist=None, device=None):
    """Whole-job throughput of independent replicas: units summed over ranks,
    divided by the slowest rank's time (max over ranks).  Returns
    (value per second, max ms, total units).  No data moves between ranks
    besides these two numbers."""
    import torch
    ms = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    units = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        dist.all_reduce(units, op=dist.ReduceOp.SUM)
    max_ms, total = float(ms.item()), float(units.item())
    return total / (max_ms / 1e3), max_ms, total


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), source="measured")
    except Exception:
        return dict(hbm_gbs=6400.0, source="fallback")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons around the timed region.
    Started before the warm-up steps (nvidia-smi takes a few hundred ms to its first
    sample); every sample carries its timestamp, and the report keeps those taken
    between begin() and end(), or, for a region shorter than the sampling period,
    the samples adjacent to it ("window": "adjacent")."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    def _rows(self):
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                continue
            rows.append((ts, parts[1:]))
        return rows

    def stop(self):
        if self.proc is None:
            return None
        # wait (at most 2 s) for a sample after the region, so that a short region has a neighbour
        deadline = time.time() + 2.0
        while self.t1 is not None and time.time() < deadline and not any(ts >= self.t1 for ts, _ in self._rows()):
            time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = self._rows()
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for ts, r in rows if self.t0 is not None and self.t0 <= ts <= self.t1]
        window = "timed region"
        if not inside:
            before = [r for ts, r in rows if self.t0 is not None and ts < self.t0][-1:]
            after = [r for ts, r in rows if self.t1 is not None and ts > self.t1][:1]
            inside = before + after or [rows[-1][1]]
            window = "adjacent"
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "window": window}


def stage_bytes(info, tokens):
    """Algorithmic HBM bytes per frame of each stage: every input read once and
    every output written once at its storage width (RGB bytes, float planes
    and coefficients, int16 codes, state and tokens)."""
    N = W_ * H_
    Hp, Wp = info.padded_height, info.padded_width
    Hcp, Wcp = info.padded_chroma_height, info.padded_chroma_width
    P = [(Hp, Wp), (Hcp, Wcp), (Hcp, Wcp)]
    C = info.coeffs
    lp = 0
    dfb = 0
    for (h, w) in P:
        for j in range(1, LEVELS + 1):
            pj = (h >> (j - 1)) * (w >> (j - 1))
            k = DIRS[j - 1]
            lp += 4 * (pj + pj // 4 + pj)               # read level input, write lowpass + detail
            # DFB launches touching level j: one for stages 1-2 (fused), one per stage >= 3;
            # each reads and writes every sample of the level once
            launches = 0 if k == 0 else 1 + max(0, k - 2)
            dfb += launches * 8 * pj
    nplane = Hp * Wp + 2 * Hcp * Wcp
    return {
        "colour_fwd": 3 * N + 4 * nplane,
        "lp_analysis": lp,
        "dfb_analysis": dfb,
        "quantise_kp": 4 * C + 2 * C + 2 * C + 2 * C,
        "rle_stream": 2 * C + 2 * C + 2 * tokens,
        "parse_unrle": 2 * tokens + 2 * C,
        "unquantise_kp": 2 * C + 2 * C + 2 * C + 4 * C,
        "dfb_synthesis": dfb,
        "lp_synthesis": lp,
        "colour_inv": 4 * N + 2 * 4 * N // 4 + 3 * N,
    }


def _luma(x):
    x = x.float()
    return (x[..., 0] + 2 * x[..., 1] + x[..., 2]) / 4


def sequence_run(dev, flush, w, h, L, k, qph, qpl, kint, n, seed, frames=None):
    """The plain per-frame pipeline on one stream: n frames encoded one call each, then
    decoded one call each, through the synchronous API (every call waits for its result),
    each call bracketed by CUDA events with L2 flushed before it; then the same calls
    through the asynchronous API, queued back to back (n encodes, then n decodes reading
    their lengths from device memory), one synchronisation per direction, L2 flushed once
    before each queue.  Also the mean stream size and the luma PSNR of the decoded frames."""
    import numpy as np
    import torch
    from paper_1510_00561_b300 import Codec
    from paper_1510_00561_b300 import synthetic as S
    if frames is None:
        frames = S.SyntheticVideo(S.spec_for(w, h, seed=seed)).frames(n)
    frames = [torch.from_numpy(f).to(dev) for f in frames]
    kw = dict(width=w, height=h, levels=L, dirs_log2=k, qph=qph, qpl=qpl, key_interval=kint)
    enc, dec = Codec(**kw), Codec(**kw)
    outs = [torch.empty(enc.max_stream, dtype=torch.uint8, device=dev) for _ in range(n)]
    rgbs = [torch.empty((h, w, 3), dtype=torch.uint8, device=dev) for _ in range(n)]
    st = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for t in range(min(n, 3)):                               # warm-up of both APIs, then fresh coder state
        s_, _ = enc.encode(frames[t], out=outs[t])
        dec.decode(s_, out=rgbs[t])
    enc.reset()
    dec.reset()
    w_len = torch.zeros(1, dtype=torch.int64, device=dev)
    for t in range(min(n, 3)):
        enc.encode_async(frames[t], outs[t], out_len=w_len)
        dec.decode_async(outs[t], rgbs[t], in_len=w_len)
    torch.cuda.synchronize()
    assert enc.get_error() == 0 and dec.get_error() == 0
    enc.reset()
    dec.reset()
    lens = [0] * n

    def per_call(fn):
        tot = 0.0
        for t in range(n):
            flush.zero_()
            e0, e1 = ev(), ev()
            e0.record(st)
            fn(t)
            e1.record(st)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    def enc_call(t):
        s_, _ = enc.encode(frames[t], out=outs[t])
        lens[t] = s_.numel()

    enc_ms = per_call(enc_call)
    dec_ms = per_call(lambda t: dec.decode(outs[t][:lens[t]], out=rgbs[t]))
    mse = [float(((_luma(rgbs[t]) - _luma(frames[t])) ** 2).mean()) for t in range(n)]
    enc.reset()
    dec.reset()
    d_len = torch.zeros(n, dtype=torch.int64, device=dev)

    def queued(fn):
        flush.zero_()
        e0, e1 = ev(), ev()
        e0.record(st)
        for t in range(n):
            fn(t)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    aenc_ms = queued(lambda t: enc.encode_async(frames[t], outs[t], out_len=d_len[t:t + 1]))
    adec_ms = queued(lambda t: dec.decode_async(outs[t], rgbs[t], in_len=d_len[t:t + 1]))
    assert d_len.cpu().tolist() == lens and enc.get_error() == 0 and dec.get_error() == 0
    return {"frames": n, "qph": qph, "qpl": qpl,
            "encode_frames_per_s": n * 1e3 / enc_ms, "decode_frames_per_s": n * 1e3 / dec_ms,
            "encode_decode_frames_per_s": n * 1e3 / (enc_ms + dec_ms),
            "async_encode_frames_per_s": n * 1e3 / aenc_ms, "async_decode_frames_per_s": n * 1e3 / adec_ms,
            "async_encode_decode_frames_per_s": n * 1e3 / (aenc_ms + adec_ms),
            "mean_stream_bytes": sum(lens) / n,
            "y_psnr_db": float(np.mean([10 * np.log10(255.0 ** 2 / max(m, 1e-12)) for m in mse]))}


def differentiable_run(dev, flush, steps=10, warm=3):
    """The differentiable transform: batch 8 of 1088 x 1920 float luma planes (the 1080p
    decomposition, 5 levels, 32/16/16/8/8), loss mean((S soft_T(A x) - x)^2) with one learnable
    threshold per directional subband, forward and backward (hand-written adjoints) per step.
    Algorithmic bytes of a step, each FP32 array read or written once per use: forward A (x in,
    c out), soft threshold (c in, y out), inverse S (y in, x' out), the loss (x', x in) and its
    gradient (out), S^T (in, out), the threshold backward (c and the gradient in, dL/dc out) and
    A^T (in, out): 28 P + 36 C bytes per plane (P pixels, C coefficients)."""
    import torch
    from paper_1510_00561_b300 import synthetic as S
    from paper_1510_00561_b300.autograd import ThresholdedReconstruction
    H, W, B = 1088, 1920, 8
    x = torch.from_numpy(S.luma_planes(B, W, H, seed=3)).to(dev)
    m = ThresholdedReconstruction(H, W, LEVELS, DIRS, B, t_init=4.0, device=dev)
    st = torch.cuda.current_stream()

    def step():
        m.T.grad = None
        loss = ((m(x) - x) ** 2).mean()
        loss.backward()
        return loss

    for _ in range(warm):
        step()
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        loss = step()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / steps
    P, C = H * W, m.plan.total
    nbytes = B * (28 * P + 36 * C)
    pk = peaks()
    return {"workload": "differentiable CT, batch 8 of 1088x1920 float32 luma planes, 5 levels, 32/16/16/8/8, "
                        "forward + adjoint backward with 80 learnable thresholds",
            "ms_per_step": ms, "planes_per_s": B * 1e3 / ms, "steps": steps, "loss": float(loss),
            "algorithmic_bytes_per_step": nbytes, "achieved_gbs": nbytes / (ms / 1e3) / 1e9,
            "frac": nbytes / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "l2": "flushed before every step"}


MIXED_CLASSES = [(176, 144, 3, [3, 2, 2]), (352, 288, 3, [3, 2, 2]), (640, 480, 4, [4, 3, 3, 2]),
                 (1280, 720, 5, [5, 4, 4, 3, 3])]


def mixed_batch_run(dev, flush, T=30, warm=3, per_class=16, distinct=30):
    """Batched multi-stream coding: 64 streams (16 each of QCIF, CIF, VGA, 720p, pyramid depth
    3/3/4/5), step 8, K every 10, one encode+decode per stream per step, each step one CUDA-graph
    launch; stream j of a class shows its class's sequence shifted by 2j frames.  T timed steps,
    L2 flushed before each."""
    import torch
    from paper_1510_00561_b300 import Batch
    jobs = [(w, h, 70 + ci, t) for ci, (w, h, _, _) in enumerate(MIXED_CLASSES) for t in range(distinct)]
    flat = make_frames_sized(jobs)
    seqs = [[torch.from_numpy(f).to(dev) for f in flat[ci * distinct:(ci + 1) * distinct]]
            for ci in range(len(MIXED_CLASSES))]
    streams = [dict(width=w, height=h, levels=L, dirs_log2=k, qph=QPH, qpl=QPL, key_interval=KINT)
               for (w, h, L, k) in MIXED_CLASSES for _ in range(per_class)]
    b = Batch(streams)
    outs = [torch.empty((s["height"], s["width"], 3), dtype=torch.uint8, device=dev) for s in streams]

    def frames_at(t):
        return [seqs[ci][(t + 2 * j) % distinct] for ci in range(len(MIXED_CLASSES)) for j in range(per_class)]

    shape = b.autotune(3, rgb=frames_at(0), rgb_out=outs, reps=3)
    for t in range(warm):
        b.step(3, rgb=frames_at(t), rgb_out=outs)
    b.reset()
    st = torch.cuda.current_stream()
    tot, nbytes = 0.0, 0
    for t in range(T):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        res = b.step(3, rgb=frames_at(t), rgb_out=outs)
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        nbytes += sum(r["out_len"] for r in res)
    n = len(streams)
    return {"workload": "64 streams (16 each QCIF, CIF, VGA, 720p; 3/3/4/5 levels), encode+decode, one "
                        "graph launch per step, %d steps" % T,
            "frames_per_s": n * T * 1e3 / tot, "ms_per_step": tot / T, "steps": T,
            "launch_shape": list(shape),
            "mean_stream_bytes": nbytes / (n * T), "l2": "flushed before every step"}


def plain_e2e_async(kw, h_frames, dev, steps, ring=4):
    """The plain per-frame path end to end through host buffers, with the asynchronous API: per
    frame the pinned RGB frame goes up, is encoded, its bitstream comes down to pinned memory and
    goes back up (a sender's and a receiver's copies), is decoded, and the decoded frame comes
    down.  Coding runs on the compute stream, copies on a copy stream; the host reads each
    frame's length (8 bytes copied after its encode) while the next frame's encode is already
    queued, so the device never waits for the host.  Uploads and downloads go on copy streams
    of their own (the two copy engines work at once).  Returns (frames/s, H2D bytes/frame,
    D2H bytes/frame)."""
    import torch
    from paper_1510_00561_b300 import Codec
    enc, dec = Codec(**kw), Codec(**kw)
    H, W = kw["height"], kw["width"]
    cs, cp, cd = torch.cuda.current_stream(), torch.cuda.Stream(dev), torch.cuda.Stream(dev)   # compute, up, down
    R = ring
    d_in = [torch.empty((H, W, 3), dtype=torch.uint8, device=dev) for _ in range(R)]
    d_out = [torch.empty(enc.max_stream, dtype=torch.uint8, device=dev) for _ in range(R)]
    d_sin = [torch.empty(enc.max_stream, dtype=torch.uint8, device=dev) for _ in range(R)]
    d_rgb = [torch.empty((H, W, 3), dtype=torch.uint8, device=dev) for _ in range(R)]
    h_str = [torch.empty(enc.max_stream, dtype=torch.uint8).pin_memory() for _ in range(R)]
    h_rgb = [torch.empty((H, W, 3), dtype=torch.uint8).pin_memory() for _ in range(R)]
    d_len = torch.zeros(R, dtype=torch.int64, device=dev)
    h_len = torch.zeros(R, dtype=torch.int64).pin_memory()
    ev = {name: [torch.cuda.Event() for _ in range(R)] for name in ("in", "enc", "sdown", "sin", "dec", "done")}
    io = [0, 0]

    def upload_encode(t):
        k = t % R
        if t >= R:
            ev["done"][k].synchronize()          # frame t - R has left slot k
        with torch.cuda.stream(cp):
            d_in[k].copy_(h_frames[t % len(h_frames)], non_blocking=True)
            ev["in"][k].record(cp)
        cs.wait_event(ev["in"][k])
        enc.encode_async(d_in[k], d_out[k], out_len=d_len[k:k + 1], stream=cs)
        h_len[k:k + 1].copy_(d_len[k:k + 1], non_blocking=True)
        ev["enc"][k].record(cs)
        io[0] += d_in[k].numel()

    def round_trip_decode(t):
        k = t % R
        ev["enc"][k].synchronize()
        n = int(h_len[k])
        with torch.cuda.stream(cd):
            cd.wait_event(ev["enc"][k])
            h_str[k][:n].copy_(d_out[k][:n], non_blocking=True)
            ev["sdown"][k].record(cd)
        with torch.cuda.stream(cp):
            cp.wait_event(ev["sdown"][k])
            d_sin[k][:n].copy_(h_str[k][:n], non_blocking=True)
            ev["sin"][k].record(cp)
        cs.wait_event(ev["sin"][k])
        dec.decode_async(d_sin[k][:n], d_rgb[k], stream=cs)
        ev["dec"][k].record(cs)
        with torch.cuda.stream(cd):
            cd.wait_event(ev["dec"][k])
            h_rgb[k].copy_(d_rgb[k], non_blocking=True)
            ev["done"][k].record(cd)
        io[0] += n
        io[1] += n + d_rgb[k].numel() + 8

    def run(nsteps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cs)
        cp.wait_event(e0)
        cd.wait_event(e0)
        upload_encode(0)
        for t in range(1, nsteps):
            upload_encode(t)
            round_trip_decode(t - 1)
        round_trip_decode(nsteps - 1)
        cs.wait_stream(cp)
        cs.wait_stream(cd)
        e1.record(cs)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    run(min(steps, 4))
    enc.reset()
    dec.reset()
    io[0] = io[1] = 0
    ms = run(steps)
    assert enc.get_error() == 0 and dec.get_error() == 0
    return steps * 1e3 / ms, io[0] // steps, io[1] // steps


def cpu_oracle_rate(frames, band_rows=None, seconds_cap=30.0):
    """Oracle encode+decode frames/s on host cores (single thread), on a bounded
    sample: whole frames, or horizontal bands of band_rows rows of them."""
    import numpy as np
    import oracle as O
    rows = band_rows or H_
    cod = O.Codec(W_, rows, LEVELS, DIRS, QPH, QPL, 0.0, KINT)
    done = 0
    t0 = time.perf_counter()
    for f in frames:
        s, _ = cod.encode(np.ascontiguousarray(f[:rows]))
        cod.decode(s)
        done += 1
        if time.perf_counter() - t0 > seconds_cap:
            break
    dt = time.perf_counter() - t0
    return done * rows / H_ / dt, done, dt


def _oracle_stream(args):
    """One worker process: the oracle encodes and decodes `n` frames of its own 1080p stream
    (single-threaded); returns (frames, wall-clock start, wall-clock end) of the coding alone."""
    seed, n = args
    import numpy as np
    import oracle as O
    frames = _gen_frames(seed, n)
    cod = O.Codec(W_, H_, LEVELS, DIRS, QPH, QPL, 0.0, KINT)
    t0 = time.time()
    for f in frames:
        s, _ = cod.encode(np.ascontiguousarray(f))
        cod.decode(s)
    return n, t0, time.time()


def cpu_oracle_parallel(workers, frames_each=2):
    """Oracle encode+decode frames/s with `workers` processes on the host cores, each coding
    its own stream (streams are independent, so this is how the oracle uses many cores
    without any change to it).  Rate = all frames / (last end - first start)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_stream, [(100 + i, frames_each) for i in range(workers)]))
    n = sum(r[0] for r in res)
    dt = max(r[2] for r in res) - min(r[1] for r in res)
    return n / dt, n, dt


SERVE_CLASSES = [  # (width, height, levels, dirs_log2, weight)
    (176, 144, 3, [3, 2, 2], 0.20), (352, 288, 3, [3, 2, 2], 0.30), (640, 480, 4, [4, 3, 3, 2], 0.30),
    (1280, 720, 5, [5, 4, 4, 3, 3], 0.15), (1920, 1080, 5, [5, 4, 4, 3, 3], 0.05)]


def served_run(d_frames, dev, n_streams=256, fps=30.0, load=1.0, seconds=3.0, budget=120 << 30, slots=16,
               ring=4, seed=0, depth=1):
    """Continuous-batching run: n_streams sessions with resolutions drawn by
    the class weights, Poisson frame arrivals at fps * load per session, each
    arrival an encode + decode request.  Frames are crops of the 1080p
    sequence.  A session holds `ring` request buffers; an arrival that finds
    them all in flight waits on the host (its latency counts from arrival)."""
    import collections
    import numpy as np
    import torch
    from paper_1510_00561_b300 import Codec, Server
    from paper_1510_00561_b300 import _lib as cvclib
    rng = np.random.default_rng(seed)
    cls = rng.choice(len(SERVE_CLASSES), n_streams, p=[c[4] for c in SERVE_CLASSES])
    srv = Server(budget, slots_per_shard=slots, steps_in_flight=depth)
    sess = []
    max_stream = {}
    for i in range(n_streams):
        w, h, L, k, _ = SERVE_CLASSES[cls[i]]
        cfg = dict(width=w, height=h, levels=L, dirs_log2=k, qph=QPH, qpl=QPL, key_interval=KINT)
        if (w, h) not in max_stream:
            max_stream[(w, h)] = Codec(**cfg).max_stream
        bufs = [(torch.empty(max_stream[(w, h)], dtype=torch.uint8, device=dev),
                 torch.empty((h, w, 3), dtype=torch.uint8, device=dev)) for _ in range(ring)]
        # one prepared request record per ring buffer; a request only sets its frame
        ios = []
        for out, rgb_out in bufs:
            io = cvclib.BatchIo()
            io.pitch_bytes = d_frames[0].stride(0)
            io.d_out, io.out_cap = out.data_ptr(), out.numel()
            io.d_rgb_out, io.pitch_out = rgb_out.data_ptr(), rgb_out.stride(0)
            ios.append(io)
        sess.append(dict(id=srv.open(**cfg), w=w, h=h, bufs=bufs, ios=ios, free=list(range(ring)),
                         arrivals=collections.deque(), t=0))
    # frames are top-left crops of the 1080p frames: the same base pointers and row pitch
    frame_ptr = [f.data_ptr() for f in d_frames]
    setup = srv.stats()
    # arrival times (seconds from start) of every session
    events = []
    for i in range(n_streams):
        t = rng.exponential(1.0 / (fps * load))
        while t < seconds:
            events.append((t, i))
            t += rng.exponential(1.0 / (fps * load))
    events.sort()
    lat, inflight = [], {}
    tag = 0
    t0 = Server.now_ns()
    ev_i = 0
    done = 0
    deadline = t0 + int(seconds * 4e9)
    pending = set()        # sessions with arrivals not yet submitted

    F = len(d_frames)
    ev_t = [t0 + int(t * 1e9) for t, _ in events]

    def pump():
        nonlocal tag
        for i in list(pending):
            S = sess[i]
            while S["arrivals"] and S["free"]:
                arr = S["arrivals"].popleft()
                b = S["free"].pop()
                io = S["ios"][b]
                io.d_rgb = frame_ptr[S["t"] % F]
                S["t"] += 1
                srv.submit_io(S["id"], 3, io, tag)
                inflight[tag] = (i, b, arr)
                tag += 1
            if not S["arrivals"]:
                pending.discard(i)

    while True:
        now = Server.now_ns()
        while ev_i < len(events) and ev_t[ev_i] <= now:
            i = events[ev_i][1]
            sess[i]["arrivals"].append(ev_t[ev_i])
            pending.add(i)
            ev_i += 1
        pump()
        for tg, es, ds, t_done in srv.poll_raw(wait_us=200):
            i, b, arr = inflight.pop(tg)
            sess[i]["free"].append(b)
            if es == 0 and ds == 0:
                lat.append((t_done - arr) / 1e6)
                done += 1
            if sess[i]["arrivals"]:
                pending.add(i)
        if ev_i == len(events) and not inflight and not pending:
            break
        if now > deadline:
            break
    t_end = Server.now_ns()
    st = srv.stats()
    wall = (t_end - t0) / 1e9
    lat_sorted = sorted(lat)
    q = lambda p: lat_sorted[min(len(lat_sorted) - 1, int(p * len(lat_sorted)))] if lat_sorted else None
    return {"streams": n_streams, "load": load, "slots_per_shard": slots, "steps_in_flight": depth,
            "offered_fps": len(events) / seconds,
            "completed": done, "requests": len(events), "frames_per_s": done / wall, "wall_s": wall,
            "p50_ms": q(0.50), "p99_ms": q(0.99), "max_ms": lat_sorted[-1] if lat_sorted else None,
            "shards": setup["shards"], "admitted": setup["active_sessions"], "waiting": setup["waiting_sessions"],
            "peak_bytes": st["peak_used_bytes"], "budget_bytes": budget, "steps": st["steps"],
            "requests_per_step": st["requests_done"] / max(1, st["steps"])}


def deflate_run(kstreams, dev, reps=3):
    """§3.9 DEFLATE of one K-frame period of the batch's encoded 1080p frames, in both modes
    (scalable: a stream per component; CVC-NTS: a stream per frame): the B frames of each
    step deflated, then inflated, in one call each (cvc_deflate_frames, cvc_inflate_frames;
    CUDA events around the calls, which synchronise), their sizes, and zlib's Huffman-only
    and default sizes of the same token bytes for reference."""
    import zlib
    import numpy as np
    import torch
    from paper_1510_00561_b300 import Deflater
    B = len(kstreams[0])
    pouts = [[torch.empty(f.numel() + (1 << 16), dtype=torch.uint8, device=dev) for f in ks] for ks in kstreams]
    outs = [[torch.empty(f.numel() + 16, dtype=torch.uint8, device=dev) for f in ks] for ks in kstreams]
    st = torch.cuda.current_stream()

    def mode(nts):
        dfl = Deflater(max_frames=B, nts=nts, width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH,
                       qpl=QPL, key_interval=KINT)
        packed = []
        for ks, po in zip(kstreams, pouts):                  # warm-up, and the outputs
            p, sts = dfl.deflate_many(ks, po)
            assert all(v == 0 for v in sts)
            packed.append([x.clone() for x in p])
        for pk, o, ks in zip(packed, outs, kstreams):
            back, sts = dfl.inflate_many(pk, o)
            assert all(v == 0 for v in sts) and all(torch.equal(b, k) for b, k in zip(back, ks))
        times = {}
        for name, fn in (("deflate", lambda t: dfl.deflate_many(kstreams[t], pouts[t])),
                         ("inflate", lambda t: dfl.inflate_many(packed[t], outs[t]))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(reps):
                for t in range(len(kstreams)):
                    fn(t)
            e1.record(st)
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) / (reps * len(kstreams))
        return times, sum(x.numel() for pk in packed for x in pk)

    times, out = mode(False)
    times_nts, out_nts = mode(True)
    frames = [f for ks in kstreams for f in ks]
    raw = sum(f.numel() for f in frames)
    tok = zh = zd = 0
    for f in frames[:KINT]:                                  # zlib on stream 0's period (host time)
        b = bytes(f.cpu().numpy())
        ncomp = int(np.frombuffer(b[28:32], "<u4")[0])
        counts = np.frombuffer(b[32:32 + 4 * ncomp], "<u4")
        tok += 2 * int(counts.sum())
        pos = 32 + 4 * ncomp
        for n in counts:
            t = b[pos:pos + 2 * int(n)]
            pos += 2 * int(n)
            for strat, acc in ((zlib.Z_HUFFMAN_ONLY, "h"), (zlib.Z_DEFAULT_STRATEGY, "d")):
                z = zlib.compressobj(6, zlib.DEFLATED, -15, 8, strat)
                k = len(z.compress(t) + z.flush())
                if acc == "h":
                    zh += k
                else:
                    zd += k
    return {"workload": "DEFLATE (scalable mode: per-component Huffman-only streams; nts: one per frame) of "
                        "%d encoded 1080p frames (%d streams x one K-frame period), %d frames per call"
                        % (len(frames), B, B),
            "deflate_ms_per_call": times["deflate"], "inflate_ms_per_call": times["inflate"],
            "deflate_frames_per_s": B * 1e3 / times["deflate"], "inflate_frames_per_s": B * 1e3 / times["inflate"],
            "mean_frame_bytes": raw / len(frames), "mean_deflated_bytes": out / len(frames),
            "ratio": out / raw, "token_bytes_ratio_zlib_huffman_only": zh / tok,
            "token_bytes_ratio_zlib_default": zd / tok,
            "nts": {"deflate_ms_per_call": times_nts["deflate"], "inflate_ms_per_call": times_nts["inflate"],
                    "deflate_frames_per_s": B * 1e3 / times_nts["deflate"],
                    "inflate_frames_per_s": B * 1e3 / times_nts["inflate"],
                    "mean_deflated_bytes": out_nts / len(frames), "ratio": out_nts / raw}}


def rd_run(dev, n_frames=30):
    """Rate-distortion analogues of the paper's QCIF experiments (§4.1, Figs 3, 4, 6-8) on the
    synthetic QCIF sequence: mean Y-PSNR of the decoded frames, and mean deflated bits per frame
    (DEFLATE stage, scalable and CVC-NTS).  rd: the whole QPH range with QPL = max(1, QPH // 14), motion
    search +-8, K every 10; rd8: the same with the paper's 8-bit storage; qph: QPH with QPL = 1 (Fig. 3);
    qpl: QPL with QPH = 1 (Fig. 4).  k_subband_nonzero: the share of non-zero subband codes of the K-frames.
    fig5: deflated bytes of the K-frames' lowpass bands with and without the column filter (Fig. 5)."""
    import numpy as np
    import torch
    from paper_1510_00561_b300 import Codec, Deflater
    from paper_1510_00561_b300 import synthetic as S
    w, h, L, k = 176, 144, 3, [3, 2, 2]
    src = S.SyntheticVideo(S.spec_for(w, h, seed=0)).frames(n_frames)
    d_src = [torch.from_numpy(f).to(dev) for f in src]

    def luma(x):
        x = x.float()
        return (x[..., 0] + 2 * x[..., 1] + x[..., 2]) / 4

    y_src = [luma(f) for f in d_src]

    nsub = 1 + sum(1 << d for d in k)                        # components of one plane

    def subband_codes(s, ncomp):
        """(non-zero, all) subband codes of a K-frame, from its tokens"""
        b = s.cpu().numpy()
        counts = np.frombuffer(b[32:32 + 4 * ncomp].tobytes(), "<u4")
        toks = np.frombuffer(b[32 + 4 * ncomp:32 + 4 * ncomp + 2 * int(counts.sum())].tobytes(), "<i2")
        nz = tot = pos = 0
        for j, n in enumerate(counts):
            t = toks[pos:pos + int(n)]
            pos += int(n)
            if j % nsub:
                runs = t == 0
                run_len = np.roll(runs, 1)                   # the count after each run marker
                run_len[0] = False
                nz += int((~runs & ~run_len).sum())
                tot += int((~runs & ~run_len).sum()) + int(t[np.flatnonzero(runs) + 1].sum())
        return nz, tot

    def point(qph, qpl, motion, storage8=False):
        kw = dict(width=w, height=h, levels=L, dirs_log2=k, qph=qph, qpl=qpl, key_interval=10, motion_range=motion,
                  storage8=storage8)
        enc, dec, dfl, nts = Codec(**kw), Codec(**kw), Deflater(**kw), Deflater(nts=True, **kw)
        mse, bits, bits_nts, nz, tot = 0.0, 0, 0, 0, 0
        for f, ys in zip(d_src, y_src):
            s, ft = enc.encode(f)
            bits += 8 * dfl.deflate(s).numel()
            bits_nts += 8 * nts.deflate(s).numel()
            mse += float(((luma(dec.decode(s.clone())) - ys) ** 2).mean())
            if ft == 0:
                a, b = subband_codes(s, enc.ncomp)
                nz, tot = nz + a, tot + b
        mse /= len(d_src)
        return {"qph": qph, "qpl": qpl, "y_psnr_db": 10 * np.log10(255.0 ** 2 / max(mse, 1e-12)),
                "kbit_per_frame": bits / len(d_src) / 1e3, "kbit_per_frame_nts": bits_nts / len(d_src) / 1e3,
                "k_subband_nonzero": nz / max(tot, 1)}

    def fig5(qpl):
        """§3.7 / Fig. 5: deflated bytes of the K-frames' lowpass bands with the column
        filter (as coded) and without it (the running sums of the coded differences)"""
        kw = dict(width=w, height=h, levels=L, dirs_log2=k, qph=8, qpl=qpl, key_interval=10)
        enc, dfl = Codec(**kw), Deflater(**kw)
        shapes = [(enc.Hp >> L, enc.Wp >> L)] + [(enc.Hcp >> L, enc.Wcp >> L)] * 2
        filt = raw = 0
        for t, f in enumerate(d_src):
            s, ft = enc.encode(f)
            if ft != 0:
                continue
            b = s.cpu().numpy().copy()
            nc = enc.ncomp
            counts = np.frombuffer(b[32:32 + 4 * nc].tobytes(), "<u4").astype(np.int64)
            starts = 32 + 4 * nc + 2 * np.concatenate([[0], np.cumsum(counts)[:-1]])
            for p_, j in enumerate(range(0, nc, nsub)):
                hh, ww = shapes[p_]
                assert counts[j] == hh * ww
                d = np.frombuffer(b[starts[j]:starts[j] + 2 * hh * ww].tobytes(), "<i2").reshape(hh, ww)
                codes = np.cumsum(d.astype(np.int64), axis=0).astype(np.int16)   # undo the filter
                b[starts[j]:starts[j] + 2 * hh * ww] = np.frombuffer(codes.tobytes(), np.uint8)
            lens = []
            for frame in (s, torch.from_numpy(b).to(dev)):
                pk = dfl.deflate(frame).cpu().numpy()
                sl = np.frombuffer(pk[32 + 4 * nc:32 + 8 * nc].tobytes(), "<u4")
                lens.append(int(sl[::nsub].sum()))
            filt, raw = filt + lens[0], raw + lens[1]
        return {"qpl": qpl, "lowpass_bytes_filtered": filt, "lowpass_bytes_unfiltered": raw,
                "gain": raw / max(filt, 1)}

    qphs = [1, 2, 4, 8, 16, 32, 64, 128, 181]
    return {"workload": "synthetic QCIF, %d frames, 3 levels 8/4/4 directions, 4:2:0" % n_frames,
            "fig5": [fig5(q) for q in (1, 4, 12)],
            "rd": [point(q, max(1, q // 14), 8) for q in qphs],
            "rd8": [point(q, max(1, q // 14), 8, storage8=True) for q in qphs],
            "qph": [point(q, 1, 0) for q in qphs],
            "qpl": [point(1, q, 0) for q in [1, 2, 4, 8, 16, 32, 48, 71]]}


def run_reference(args, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    # size the band so that the whole run takes about two minutes (one 1080p frame ~ 6 s)
    per_step = min(6.5, 120.0 / max(1, steps + warm))
    band = max(64, min(H_, int(per_step / 6.5 * H_) // 64 * 64))   # rows of the frame actually coded
    frames = _gen_frames(0, min(steps + warm, 12))
    import numpy as np
    import oracle as O
    cod = O.Codec(W_, band, LEVELS, DIRS, QPH, QPL, 0.0, KINT)
    for i in range(warm):
        s, _ = cod.encode(np.ascontiguousarray(frames[i % len(frames)][:band]))
        cod.decode(s)
    t0 = time.perf_counter()
    for i in range(steps):
        s, _ = cod.encode(np.ascontiguousarray(frames[(warm + i) % len(frames)][:band]))
        cod.decode(s)
    dt = time.perf_counter() - t0
    value = steps * band / H_ / dt
    sample = "oracle encode+decode of a 1920x%d band of each 1080p frame per step (%.3f frame)" % (band, band / H_)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3 / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1080p CVC encode+decode, 5-level CT 32/16/16/8/8, step 8, K every 10",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=30, help="distinct frames per stream (cycled)")
    ap.add_argument("--e2e-steps", type=int, default=30, help="steps of the host-buffer end-to-end pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--batch", type=int, default=16, help="concurrent 1080p streams per GPU in the batched form")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="length of the served run (0: skip)")
    ap.add_argument("--serve-sweep", default="", help="comma-separated load multipliers for extra served runs")
    ap.add_argument("--serve-slots", type=int, default=8, help="slots per shard of the served loop")
    ap.add_argument("--serve-depth", type=int, default=2, help="steps in flight per shard of the served loop")
    ap.add_argument("--no-scalable", action="store_true", help="skip the per-scale decode pass")
    ap.add_argument("--motion-range", type=int, default=8, help="search range of the motion pass (0: skip)")
    ap.add_argument("--no-rd", action="store_true", help="skip the QCIF rate-distortion sweeps")
    ap.add_argument("--no-taps", action="store_true", help="skip the 6- and 8-tap DFB prototype pass")
    ap.add_argument("--no-suite", action="store_true",
                    help="skip the QCIF / VGA sequences, the differentiable transform and the mixed batch")
    ap.add_argument("--profile", action="store_true",
                    help="for ncu: --warmup batched steps, then one step inside the NVTX range 'profile_step'; "
                         "no timing, no JSON line")
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="processes of the many-core oracle baseline (0: min(nproc, 16))")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    # the served loop runs one CUDA stream per shard: give the device as many hardware
    # queues as it allows, so that shards do not share queues (read at context creation)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    frames = make_frames(seed=rank, n=args.frames)
    vga_frames = None
    if not args.no_suite:
        vga_frames = make_frames_sized([(640, 480, 0, t) for t in range(60)])
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1510_00561_b300 import Batch, Codec, kernel_launches

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.profile:
        d_frames = [torch.from_numpy(f).to(dev) for f in frames]
        B = args.batch
        pb = Batch([dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL,
                         key_interval=KINT)] * B)
        p_outs = [torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)]
        for i in range(args.warmup + 1):
            if i == args.warmup:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("profile_step")
            pb.step(3, rgb=[d_frames[(i + 3 * j) % len(d_frames)] for j in range(B)], rgb_out=p_outs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("profiled one batched step of %d streams (P-frame %d)" % (B, args.warmup), flush=True)
        return

    codec = Codec(W_, H_, LEVELS, DIRS, QPH, QPL, 0.0, KINT)
    d_frames = [torch.from_numpy(f).to(dev) for f in frames]
    out = torch.empty(codec.max_stream, dtype=torch.uint8, device=dev)
    rgb = torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()
    F = len(d_frames)

    def timed(step, steps, flush_between=True):
        """CUDA-event time (ms, this rank) of `steps` steps, L2 flushed before each."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            if flush_between and not args.no_flush:
                flush.zero_()
            starts[i].record(stream)
            step(i)
            ends[i].record(stream)
        torch.cuda.synchronize()
        barrier()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends))

    # ---------------------------------------------------------------- plain
    plain_bytes = [0]

    def plain_step(i):
        s, _ = codec.encode(d_frames[i % F], out=out)
        codec.decode(s, out=rgb)
        plain_bytes[0] += s.numel()

    for i in range(args.warmup):
        plain_step(i)
    plain_value, plain_ms, _ = combine_ranks(timed(lambda i: plain_step(args.warmup + i), args.steps), args.steps,
                                             dist, dev)

    # plain end to end through the C ABI with host buffers (pinned), per step:
    # H2D frame, encode, D2H bitstream, H2D bitstream, decode, D2H frame
    h_frames = [torch.from_numpy(f).pin_memory() for f in frames[:min(F, 8)]]
    h_stream = torch.empty(codec.max_stream, dtype=torch.uint8).pin_memory()
    h_rgb = torch.empty((H_, W_, 3), dtype=torch.uint8).pin_memory()
    d_in = torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev)
    d_sin = torch.empty(codec.max_stream, dtype=torch.uint8, device=dev)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    io_bytes = [0, 0]

    def plain_e2e_step(i):
        d_in.copy_(h_frames[i % len(h_frames)], non_blocking=True)
        s, _ = codec.encode(d_in, out=out)
        n = s.numel()
        h_stream[:n].copy_(s, non_blocking=True)
        d_sin[:n].copy_(h_stream[:n], non_blocking=True)
        codec.decode(d_sin[:n], out=rgb)
        h_rgb.copy_(rgb, non_blocking=True)
        io_bytes[0] += d_in.numel() + n
        io_bytes[1] += n + rgb.numel()

    plain_e2e_value = combine_ranks(timed(plain_e2e_step, e2e_steps, flush_between=False), e2e_steps, dist, dev)[0]
    del codec
    kw1080 = dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL, key_interval=KINT)
    a_rate, a_h2d, a_d2h = plain_e2e_async(kw1080, h_frames, dev, e2e_steps)
    a_value = combine_ranks(e2e_steps * 1e3 / a_rate, e2e_steps, dist, dev)[0]
    plain = {"value": plain_value, "ms_per_step": plain_ms / args.steps, "streams_per_gpu": 1,
             "e2e": {"value": plain_e2e_value, "unit": UNIT, "api": "synchronous calls",
                     "h2d_bytes_per_step": io_bytes[0] // e2e_steps, "d2h_bytes_per_step": io_bytes[1] // e2e_steps},
             "e2e_async": {"value": a_value, "unit": UNIT, "api": "asynchronous calls, copies on a copy stream",
                           "h2d_bytes_per_step": a_h2d, "d2h_bytes_per_step": a_d2h}}

    # -------------------------------------------------------------- batched
    # B concurrent 1080p streams; stream j shows the rank's sequence shifted by 3j frames
    B = args.batch
    batch = Batch([dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL,
                        key_interval=KINT)] * B)
    outs_rgb = [torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)]

    def frames_at(i):
        return [d_frames[(i + 3 * j) % F] for j in range(B)]

    shape = (8, 148 * 8, 0, 0) if args.no_autotune else batch.autotune(3, rgb=frames_at(0), rgb_out=outs_rgb, reps=3)
    info0 = batch.info[0]
    batch_bytes = [0]

    def batch_step(i):
        res = batch.step(3, rgb=frames_at(i), rgb_out=outs_rgb)
        batch_bytes[0] += sum(r["out_len"] for r in res)

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    for i in range(args.warmup):
        batch_step(i)
    launches0 = kernel_launches()
    if clocks:
        clocks.begin()
    t_wall = time.perf_counter()
    value, tot_ms, _ = combine_ranks(timed(lambda i: batch_step(args.warmup + i), args.steps), args.steps * B,
                                     dist, dev)
    t_wall = time.perf_counter() - t_wall
    if clocks:
        clocks.end()
    launches = kernel_launches() - launches0
    clk = clocks.stop() if clocks else None

    # stage breakdown of the same steps as direct launches bracketed by CUDA events
    batch.set_timing(True)
    stage_steps = min(args.steps, 20)
    timed(lambda i: batch_step(args.warmup + i), stage_steps)
    stage = batch.timing()
    batch.set_timing(False)

    # batched end to end through the public API: every step uploads its B frames
    # from pinned memory and downloads its B bitstreams and B reconstructed
    # frames.  Double-buffered and asynchronous (cvc_batch_step_async): step t+1
    # is queued before the host reads step t's lengths and queues its downloads,
    # so the device never waits for the host; uploads and downloads run on copy
    # streams of their own (the host-to-device and device-to-host copy engines
    # work at once) while the steps compute.
    copy_st = torch.cuda.Stream(dev)     # uploads
    down_st = torch.cuda.Stream(dev)     # downloads
    d_ins = [[torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)] for _ in range(2)]
    d_outs = [[torch.empty(batch.info[j].max_stream_bytes, dtype=torch.uint8, device=dev) for j in range(B)]
              for _ in range(2)]
    d_rgbs = [[torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)] for _ in range(2)]
    h_outs = [[torch.empty(batch.info[j].max_stream_bytes, dtype=torch.uint8).pin_memory() for j in range(B)]
              for _ in range(2)]
    h_rgbs = [[torch.empty((H_, W_, 3), dtype=torch.uint8).pin_memory() for _ in range(B)] for _ in range(2)]
    d_res = [batch.results_buffer(dev) for _ in range(2)]
    h_res = [torch.empty(d_res[0].numel(), dtype=torch.uint8).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_res = [torch.cuda.Event() for _ in range(2)]
    io_bytes = [0, 0]

    def upload(t, k):
        with torch.cuda.stream(copy_st):
            for j in range(B):
                d_ins[k][j].copy_(h_frames[(t + j) % len(h_frames)], non_blocking=True)
                io_bytes[0] += d_ins[k][j].numel()
            ev_in[k].record(copy_st)

    def download(k):
        # the step in slot k has finished: its per-stream results are on the host
        ev_res[k].synchronize()
        res = batch.results_of(h_res[k])
        with torch.cuda.stream(down_st):
            down_st.wait_event(ev_res[k])
            for j in range(B):
                if res[j]["enc_status"] != 0 or res[j]["dec_status"] != 0:
                    raise RuntimeError("end-to-end step failed on stream %d: %s" % (j, res[j]))
                n = res[j]["out_len"]
                h_outs[k][j][:n].copy_(d_outs[k][j][:n], non_blocking=True)
                h_rgbs[k][j].copy_(d_rgbs[k][j], non_blocking=True)
                io_bytes[1] += n + d_rgbs[k][j].numel()
            ev_out[k].record(down_st)

    def e2e_run(nsteps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        for k in range(2):
            ev_out[k].record(stream)
            ev_res[k].record(stream)
        e0.record(stream)
        copy_st.wait_event(e0)
        down_st.wait_event(e0)
        upload(0, 0)
        for t in range(nsteps):
            k = t % 2
            if t + 1 < nsteps:
                copy_st.wait_event(ev_res[1 - k])   # step t-1 has read its inputs (slot 1-k)
                upload(t + 1, 1 - k)
            stream.wait_event(ev_in[k])
            stream.wait_event(ev_out[k])        # slot k's outputs downloaded two steps ago
            batch.step_async(3, rgb=d_ins[k], rgb_out=d_rgbs[k], outs=d_outs[k], results=d_res[k], stream=stream)
            h_res[k].copy_(d_res[k], non_blocking=True)
            ev_res[k].record(stream)
            if t > 0:
                download(1 - k)
        download((nsteps - 1) % 2)
        stream.wait_stream(copy_st)
        stream.wait_stream(down_st)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    e2e_run(2)                                   # warm-up of the copy path
    io_bytes[0] = io_bytes[1] = 0
    e2e_value = combine_ranks(e2e_run(e2e_steps), e2e_steps * B, dist, dev)[0]
    del d_ins, d_outs, d_rgbs

    # scalable decoding (§3.3): the same B streams decoded alone at every pyramid
    # scale; one K-frame period of bitstreams is encoded once and decoded in order
    scalable = deflate = None
    if not args.no_scalable:
        batch.reset()
        kstreams = []
        for t in range(KINT):
            res = batch.step(1, rgb=frames_at(t))
            kstreams.append([r["bytes"].clone() for r in res])
        del batch, outs_rgb
        dbatch = Batch([dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL,
                             key_interval=KINT)] * B)
        dbatch.set_shape(*shape[:2])
        dbatch.set_fusion(shape[2])
        dbatch.set_dfb_threads(shape[3])
        sc_steps = max(KINT, min(args.steps, 2 * KINT))
        scales = []
        for sc in range(LEVELS + 1):
            hs, ws = dbatch.scaled_size(0, sc)
            souts = [torch.empty((hs, ws, 3), dtype=torch.uint8, device=dev) for _ in range(B)]

            def dec_step(i, sc=sc, souts=souts):
                dbatch.step(2, streams_in=kstreams[i % KINT], rgb_out=souts, scale=sc)

            dbatch.reset()
            for i in range(KINT):                # warm-up: one whole K-frame period
                dec_step(i)
            v, ms, _ = combine_ranks(timed(dec_step, sc_steps), sc_steps * B, dist, dev)
            scales.append({"scale": sc, "size": [hs, ws], "value": v, "ms_per_step": ms / sc_steps})
        scalable = {"workload": "decode only of %d 1080p streams, each at pyramid scale s (ceil(1080/2^s) x "
                                "ceil(1920/2^s) output), K-frame period decoded in order" % B,
                    "unit": UNIT, "steps": sc_steps, "scales": scales}
        deflate = deflate_run(kstreams, dev)
        del dbatch, kstreams
    else:
        del batch, outs_rgb

    # motion-compensated P-frames (§3.2, §3.7): the same batched encode+decode with a
    # full search of +-8 pixels, against the zero-motion rate and stream size above
    motion = None
    if args.motion_range > 0:
        mb = Batch([dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL,
                         key_interval=KINT, motion_range=args.motion_range)] * B)
        mb.set_shape(*shape[:2])
        mb.set_fusion(shape[2])
        mb.set_dfb_threads(shape[3])
        m_outs = [torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)]
        m_bytes = [0, 0]

        def motion_step(i):
            res = mb.step(3, rgb=frames_at(i), rgb_out=m_outs)
            m_bytes[0] += sum(r["out_len"] for r in res)
            m_bytes[1] += B

        for i in range(args.warmup):
            motion_step(i)
        m_bytes[0] = m_bytes[1] = 0
        m_steps = max(KINT, min(args.steps, 2 * KINT))
        mv_value, m_ms, _ = combine_ranks(timed(lambda i: motion_step(args.warmup + i), m_steps), m_steps * B,
                                          dist, dev)
        mb.set_timing(True)
        timed(lambda i: motion_step(args.warmup + m_steps + i), KINT)
        m_stage = mb.timing()
        mb.set_timing(False)
        motion = {"workload": "%d 1080p streams batched, encode+decode, full search +-%d pixels on 16x16 luma "
                              "blocks, motion-compensated P-frames" % (B, args.motion_range),
                  "value": mv_value, "unit": UNIT, "ms_per_step": m_ms / m_steps, "steps": m_steps,
                  "mean_stream_bytes": m_bytes[0] / max(1, m_bytes[1]),
                  "stages_ms_per_frame": {k: v[0] / (KINT * B) for k, v in m_stage.items()}}
        del mb, m_outs

    # longer DFB prototypes (6 and 8 taps, the plain per-sample DFB path): the same batched
    # encode+decode, and its per-stage times
    taps = None
    if not args.no_taps:
        taps = []
        for nt in (6, 8):
            tb = Batch([dict(width=W_, height=H_, levels=LEVELS, dirs_log2=DIRS, qph=QPH, qpl=QPL,
                             key_interval=KINT, dfb_taps=nt)] * B)
            tb.set_shape(*shape[:2])
            tb.set_fusion(shape[2])
            tb.set_dfb_threads(shape[3])
            t_outs = [torch.empty((H_, W_, 3), dtype=torch.uint8, device=dev) for _ in range(B)]

            def taps_step(i, tb=tb, t_outs=t_outs):
                tb.step(3, rgb=frames_at(i), rgb_out=t_outs)

            for i in range(args.warmup):
                taps_step(i)
            t_steps = max(4, min(args.steps, KINT))
            t_value, t_ms, _ = combine_ranks(timed(lambda i: taps_step(args.warmup + i), t_steps), t_steps * B,
                                             dist, dev)
            tb.set_timing(True)
            timed(lambda i: taps_step(args.warmup + t_steps + i), KINT)
            t_stage = tb.timing()
            tb.set_timing(False)
            taps.append({"dfb_taps": nt, "value": t_value, "unit": UNIT, "ms_per_step": t_ms / t_steps,
                         "steps": t_steps,
                         "stages_ms_per_frame": {k: v[0] / (KINT * B) for k, v in t_stage.items()}})
            del tb, t_outs

    rd = rd_run(dev) if (not args.no_rd and rank == 0) else None

    # the other workloads: QCIF and VGA plain sequences, the differentiable transform, the mixed batch
    suite = None
    if not args.no_suite:
        suite = {"qcif_plain": sequence_run(dev, flush, 176, 144, 3, [3, 2, 2], 8, 1, 8, 16, seed=0),
                 "vga": [sequence_run(dev, flush, 640, 480, 4, [4, 3, 3, 2], q, 1, 10, 60, seed=0,
                                      frames=vga_frames) for q in (4, 8, 16)],
                 "differentiable": differentiable_run(dev, flush),
                 "mixed_batch": mixed_batch_run(dev, flush)}

    # served form: continuous batching of concurrent streams under a memory budget
    served = None
    if args.serve_seconds > 0:
        torch.cuda.synchronize()
        served = served_run(d_frames, dev, seconds=args.serve_seconds, seed=rank, slots=args.serve_slots,
                            depth=args.serve_depth)
        if args.serve_sweep:
            served["sweep"] = [served_run(d_frames, dev, seconds=args.serve_seconds, load=float(m), seed=rank,
                                          slots=args.serve_slots, depth=args.serve_depth)
                               for m in args.serve_sweep.split(",")]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- rooflines (per-stage CUDA events of batched steps; ncu counters where they match the sources)
    pk = peaks()
    frames_staged = stage_steps * B
    mean_bytes = batch_bytes[0] / ((args.warmup + args.steps + stage_steps) * B)
    info = info0
    tokens = (mean_bytes - 32 - 4 * info.components) / 2
    sb = stage_bytes(info, tokens)
    dom = max(stage, key=lambda k: stage[k][0])
    ms_dom, n_dom = stage[dom]
    per_launch_ms = ms_dom / max(1, n_dom)
    bytes_per_launch = sb[dom] * frames_staged / max(1, n_dom)
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    sources_ok = CAPTURE["sources_sha256"] is not None and CAPTURE["sources_sha256"] == kernel_sources_sha()
    dram = CAPTURE["dram_per_frame"] if sources_ok else {}
    # the whole path, as the survey defines its algorithmic traffic: per frame the encoder reads
    # the RGB frame (3N) and the coder state (2C), writes the state (2C) and the stream (S); the
    # decoder reads the stream (S) and its state (2C), writes the state (2C) and the frame (3N)
    N, C = W_ * H_, info.coeffs
    path_bytes = 6 * N + 8 * C + 2 * mean_bytes
    path_gbs = path_bytes * value / 1e9
    bw_roof = pk["hbm_gbs"] * 1e9 / path_bytes
    # issue-slot roof: the step's warp instructions per frame (ncu) against 148 SMs x 4
    # sub-partitions x one warp instruction per cycle at the SM clock sampled in the timed region
    alu = None
    if sources_ok and CAPTURE["warp_inst_per_frame"]:
        mhz = (clk or {}).get("sm_mhz") or 2032.0
        slots = N_SM * SMSP_PER_SM * mhz * 1e6
        alu = {"warp_inst_per_frame": CAPTURE["warp_inst_per_frame"], "issue_slots_per_s": slots,
               "sm_mhz": mhz, "roof_frames_per_s": slots / CAPTURE["warp_inst_per_frame"],
               "frac": value / (slots / CAPTURE["warp_inst_per_frame"])}
    roofs = {"hbm": bw_roof}
    if alu:
        roofs["alu"] = alu["roof_frames_per_s"]
    binding = min(roofs, key=roofs.get)
    roof = {"bound": "hbm", "achieved": path_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": path_gbs / pk["hbm_gbs"], "path_frac": path_gbs / pk["hbm_gbs"],
            "traffic": dram.get("step") * 1.0 if dram.get("step") else None,
            "definition": "whole encode+decode path per 1080p frame: algorithmic bytes 6N + 8C + 2S "
                          "(N pixels, C coefficients, S mean stream bytes) x frames/s, against the measured "
                          "copy bandwidth; traffic = DRAM bytes of one step's launches per frame (ncu)",
            "bytes_per_frame": path_bytes, "roof_frames_per_s": bw_roof, "peak_source": pk["source"],
            "alu": alu, "binding_roof": binding, "frac_of_binding_roof": value / roofs[binding],
            "counters": CAPTURE["profile"] if sources_ok else "no ncu capture of the current kernel sources",
            "dominant_stage": {"stage": dom, "achieved": achieved, "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                               "launches": n_dom, "bytes_per_launch": bytes_per_launch,
                               "traffic": dram[dom] * frames_staged / max(1, n_dom) if dom in dram else None,
                               "definition": "the stage's algorithmic bytes (each launch reads and writes "
                                             "what it touches once) over the stage's CUDA-event time"},
            "stages_ms_per_frame": {k: v[0] / frames_staged for k, v in stage.items()}}

    cpu = None
    if not args.no_cpu_baseline:
        rate, done, dt = cpu_oracle_rate(frames[:2], seconds_cap=25.0)
        hi = host_info()
        workers = args.cpu_workers or max(1, min(hi["nproc"] or 1, 16))
        prate, pdone, pdt = cpu_oracle_parallel(workers)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", **hi,
               "sample": "%d full 1080p frames (K then P) encoded+decoded by the FP64 oracle in %.1f s" % (done, dt),
               "all_cores": {"value": prate, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": "%d processes, each coding 2 frames (K then P) of its own 1080p stream: "
                                       "%d frames in %.1f s" % (workers, pdone, pdt)}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1080p CVC encode+decode, %d concurrent streams per GPU in one batch "
                                   "(one CUDA-graph launch per step), 1920x1080 RGB, 5-level CDF 9/7 LP + "
                                   "32/16/16/8/8 ladder DFB, QPH 8 / QPL 1, K every 10" % B,
                       "streams_per_gpu": B, "frames_cycled": F, "launch_shape": list(shape),
                       "l2": "flushed (256 MB write) before every step" if not args.no_flush else "not flushed",
                       "parallelism": "replicas (stream sharding)" if world > 1 else "single GPU",
                       "mean_stream_bytes": mean_bytes},
            "plain": plain, "served": served, "scalable": scalable, "motion": motion, "taps": taps, "deflate": deflate,
            "rd": rd, "suite": suite,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes[0] // e2e_steps,
                    "d2h_bytes_per_step": io_bytes[1] // e2e_steps},
            "gpu_launches": int(launches), "clocks": clk, "wall_s": t_wall}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
