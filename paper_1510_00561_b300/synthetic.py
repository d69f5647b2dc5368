"""Seeded synthetic inputs shaped like the paper's conferencing workloads.

This module holds no step of the codec: it only draws pixels.  Both the
CUDA path and the oracle are fed from here, so that they see identical
frames.  The paper measures on the Akiyo, Claire and Hall-monitor QCIF
sequences (§4.1), which are not available; these generators stand in for
them with the same structure: a static smooth background, a few moving
textured objects and sensor noise.

Random numbers come from a counter-based generator (SplitMix64 finaliser of
seed/stream/counter, published by Steele, Lea and Flood, 2014), so any frame
of any stream can be drawn independently and reproducibly; Gaussian noise
uses the Box-Muller transform.
"""
from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, stream, counters):
    """Uniform doubles in (0, 1) for the given counters (53-bit resolution)."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(0xD1B54A32D192ED03)
               + np.uint64(stream) * np.uint64(0x8CB92BA72F3D8DD7))
        z = _splitmix64(np.asarray(counters, dtype=np.uint64) + key)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed, stream, counters):
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        u1 = uniform(seed, stream, c * np.uint64(2))
        u2 = uniform(seed, stream, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class VideoSpec:
    width: int
    height: int
    n_objects: int
    noise_sigma: float
    seed: int = 0


QCIF = (176, 144)
CIF = (352, 288)
VGA = (640, 480)
HD720 = (1280, 720)
HD1080 = (1920, 1080)


def spec_for(width, height, seed=0):
    """Object count and noise level by resolution: 4 objects / sigma 2 at
    QCIF and CIF, 12 objects / sigma 3 from VGA up."""
    small = width * height <= 352 * 288
    return VideoSpec(width, height, 4 if small else 12, 2.0 if small else 3.0, seed)


class SyntheticVideo:
    """Frame t of a seeded conferencing-like sequence, RGB uint8 (H, W, 3)."""

    def __init__(self, spec: VideoSpec):
        self.spec = spec
        s, W, H = spec.seed, spec.width, spec.height
        u = uniform(s, 1, np.arange(64))
        # background: per channel a + b x/W + c y/H + 20 sin(low frequency)
        self.bg = []
        for ch in range(3):
            a = 60 + 100 * u[4 * ch]
            b = 60 * (u[4 * ch + 1] - 0.5)
            c = 60 * (u[4 * ch + 2] - 0.5)
            ph = 2 * np.pi * u[4 * ch + 3]
            self.bg.append((a, b, c, ph))
        fx, fy = 0.5 + 2.0 * u[20], 0.5 + 2.0 * u[21]
        self.bg_freq = (fx, fy)
        # objects: rectangles with sinusoid or checker texture and integer velocity
        self.objects = []
        for i in range(spec.n_objects):
            v = uniform(s, 100 + i, np.arange(16))
            ow = max(2, int((0.1 + 0.2 * v[0]) * W))
            oh = max(2, int((0.1 + 0.2 * v[1]) * H))
            x0 = int(v[2] * (W - ow))
            y0 = int(v[3] * (H - oh))
            vx = int(1 + 3 * v[4]) * (1 if v[5] < 0.5 else -1)
            vy = int(1 + 3 * v[6]) * (1 if v[7] < 0.5 else -1)
            vx = max(-3, min(3, vx)) or 1
            vy = max(-3, min(3, vy)) or 1
            period = 4 + 12 * v[8]
            theta = np.pi * v[9]
            checker = v[10] < 0.5
            colour = 40 + 180 * v[11:14]
            self.objects.append(dict(w=ow, h=oh, x0=x0, y0=y0, vx=vx, vy=vy, period=period,
                                     theta=theta, checker=checker, colour=colour))
        yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
        base = np.empty((H, W, 3))
        for ch, (a, b, c, ph) in enumerate(self.bg):
            base[..., ch] = (a + b * xx / W + c * yy / H
                             + 20.0 * np.sin(2 * np.pi * (fx * xx / W + fy * yy / H) + ph))
        self.background = base

    @staticmethod
    def _bounce(p0, v, t, span):
        if span <= 0:
            return 0
        period = 2 * span
        q = (p0 + v * t) % period
        return int(q if q <= span else period - q)

    def frame(self, t):
        sp = self.spec
        W, H = sp.width, sp.height
        img = self.background.copy()
        for o in self.objects:
            x = self._bounce(o["x0"], o["vx"], t, W - o["w"])
            y = self._bounce(o["y0"], o["vy"], t, H - o["h"])
            yy, xx = np.mgrid[0:o["h"], 0:o["w"]].astype(np.float64)
            ct, st = np.cos(o["theta"]), np.sin(o["theta"])
            ph = (xx * ct + yy * st) * (2 * np.pi / o["period"])
            if o["checker"]:
                tex = np.where(np.sin(ph) * np.sin((yy * ct - xx * st) * (2 * np.pi / o["period"])) >= 0, 1.0, -1.0)
            else:
                tex = np.sin(ph)
            for ch in range(3):
                img[y:y + o["h"], x:x + o["w"], ch] = o["colour"][ch] + 35.0 * tex
        n = H * W * 3
        noise = normal(sp.seed, 7, np.arange(n, dtype=np.uint64) + np.uint64(t) * np.uint64(n))
        img += sp.noise_sigma * noise.reshape(H, W, 3)
        return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)

    def frames(self, n, start=0):
        return [self.frame(start + t) for t in range(n)]


def luma_planes(batch, width, height, seed=0):
    """Float32 planes for the differentiable transform workload:
    0.25 * U[0,255] + 0.75 * (sum of 8 seeded low-frequency cosines scaled to [0,255])."""
    out = np.empty((batch, height, width), np.float32)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    for b in range(batch):
        u = uniform(seed, 1000 + b, np.arange(32))
        f = np.zeros((height, width))
        for i in range(8):
            fx, fy = 0.5 + 3.5 * u[4 * i], 0.5 + 3.5 * u[4 * i + 1]
            ph = 2 * np.pi * u[4 * i + 2]
            amp = 0.5 + u[4 * i + 3]
            f += amp * np.cos(2 * np.pi * (fx * xx / width + fy * yy / height) + ph)
        f = (f - f.min()) / max(1e-12, f.max() - f.min()) * 255.0
        noise = uniform(seed, 2000 + b, np.arange(height * width)).reshape(height, width) * 255.0
        out[b] = (0.25 * noise + 0.75 * f).astype(np.float32)
    return out
