"""Seeded synthetic inputs for the dataflow graph (shared by tests and bench).

This module holds no arithmetic of the method itself: it only draws the input
stream, the FIR taps, the matrix H, the per-frame burst pattern and the
per-instance thresholds of the workloads, deterministically from a seed.

Generator: a counter-based hash, the SplitMix64 finaliser (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied
to ``key + (counter + 1) * 0x9E3779B97F4A7C15``, turned into a uniform double
in (0, 1) from its top 53 bits, and into Gaussians by the Box-Muller
transform in FP64, rounded to FP32 at the end.  Any frame of any instance can
be regenerated on its own, on the CPU or on a CUDA device, from
(seed, tag, instance, frame).

Distribution conventions: CN(0, s2) has real and imaginary parts each
N(0, s2 / 2); a "burst" block is the same draw with its amplitude scaled by 4
(energy x16); a frame with burst fraction p has exactly round(p * F) burst
blocks chosen without replacement (the blocks with the smallest per-block hash
draws).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB

TAG_X, TAG_TAPS, TAG_H, TAG_BURST, TAG_FRAC, TAG_TAU, TAG_SHAPE, TAG_ARRIVAL, TAG_MASK = 1, 2, 3, 4, 5, 6, 7, 8, 9


def mix64(z: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _C1) & MASK64
    z = ((z ^ (z >> 27)) * _C2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *ids: int) -> int:
    """A 64-bit key for one named stream (tag, instance, frame ...)."""
    k = mix64(seed + GOLDEN)
    for i in ids:
        k = mix64(k ^ mix64((i + 1) * GOLDEN))
    return k


def _s64(v: int) -> int:
    """Reinterpret an unsigned 64-bit value as signed (torch int64)."""
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _shr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64_t(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _shr(z, 30)) * _s64(_C1)
    z = (z ^ _shr(z, 27)) * _s64(_C2)
    return z ^ _shr(z, 31)


def uniform(key: int, start: int, n: int, device="cpu") -> torch.Tensor:
    """Doubles in (0, 1): counters start .. start+n-1 of stream ``key``."""
    ctr = torch.arange(start + 1, start + 1 + n, dtype=torch.int64, device=device)
    z = _mix64_t(ctr * _s64(GOLDEN) + _s64(key))
    top = _shr(z, 11).to(torch.float64)
    return (top + 0.5) * (2.0 ** -53)


def cnormal(key: int, n: int, var: float = 1.0, device="cpu", start: int = 0) -> torch.Tensor:
    """n samples of CN(0, var) as complex128 (counters 2i, 2i+1 per sample)."""
    u = uniform(key, 2 * start, 2 * n, device).view(n, 2)
    r = torch.sqrt(-2.0 * torch.log(u[:, 0]))
    th = (2.0 * math.pi) * u[:, 1]
    s = math.sqrt(var / 2.0)
    return torch.complex(s * r * torch.cos(th), s * r * torch.sin(th))


def taps(seed: int, T: int, instance: int = 0, device="cpu") -> torch.Tensor:
    """FIR taps h[0..T) ~ CN(0, 1/T), complex64."""
    return cnormal(stream_key(seed, TAG_TAPS, instance), T, 1.0 / T, device).to(torch.complex64)


def hmat(seed: int, N: int, instance: int = 0, device="cpu") -> torch.Tensor:
    """H ~ CN(0, 1/N) entries, [N, N] row-major complex64."""
    return cnormal(stream_key(seed, TAG_H, instance), N * N, 1.0 / N, device).to(torch.complex64).view(N, N)


def burst_mask(seed: int, F: int, p: float, instance: int, frame: int, device="cpu") -> torch.Tensor:
    """Bool [F]: exactly round(p * F) burst blocks, chosen without replacement."""
    nb = int(math.floor(p * F + 0.5))
    u = uniform(stream_key(seed, TAG_BURST, instance, frame), 0, F, device)
    order = torch.argsort(u, stable=True)
    m = torch.zeros(F, dtype=torch.bool, device=device)
    m[order[:nb]] = True
    return m


def frame(seed: int, F: int, B: int, p: float, instance: int, k: int, device="cpu") -> torch.Tensor:
    """Frame k of one instance: [F, B] complex64, CN(0, 1) with the burst
    blocks scaled by 4 in amplitude."""
    x = cnormal(stream_key(seed, TAG_X, instance, k), F * B, 1.0, device).view(F, B)
    m = burst_mask(seed, F, p, instance, k, device)
    x = torch.where(m[:, None], 4.0 * x, x)
    return x.to(torch.complex64)


def frame_uniform(seed: int, tag: int, instance: int, k: int) -> float:
    """One seeded U(0, 1) draw per (tag, instance, frame)."""
    return float(uniform(stream_key(seed, tag, instance, k), 0, 1)[0])


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class PlainWorkload:
    """One graph instance: F blocks of B complex samples per frame, T taps,
    N x N matrix H, DET threshold tau, and a burst fraction per frame that is
    either fixed (``p``) or drawn U(p_lo, p_hi) per frame."""
    name: str
    F: int
    B: int
    T: int
    N: int
    frames: int
    tau: float
    seed: int
    p: float | None = 0.25
    p_lo: float = 0.1
    p_hi: float = 0.9
    C: int = 3

    def burst_fraction(self, k: int, instance: int = 0) -> float:
        if self.p is not None:
            return self.p
        u = frame_uniform(self.seed, TAG_FRAC, instance, k)
        return self.p_lo + (self.p_hi - self.p_lo) * u

    def frame(self, k: int, device="cpu", instance: int = 0) -> torch.Tensor:
        return frame(self.seed, self.F, self.B, self.burst_fraction(k, instance), instance, k, device)

    def frames_tensor(self, k0: int, n: int, device="cpu", instance: int = 0) -> torch.Tensor:
        return torch.stack([self.frame(k, device, instance) for k in range(k0, k0 + n)])

    def taps(self, device="cpu", instance: int = 0):
        return taps(self.seed, self.T, instance, device)

    def H(self, device="cpu", instance: int = 0):
        return hmat(self.seed, self.N, instance, device)

    @property
    def samples_per_frame(self) -> int:
        return self.F * self.B


# Plain graph, 100 frames of 64 blocks x 256 samples, 25% burst blocks,
# 16 taps, H 16x16, tau = 4B.
PLAIN_SMALL = PlainWorkload("plain_F64_B256_T16_N16_100fr", F=64, B=256, T=16, N=16, frames=100,
                            tau=4.0 * 256, seed=1, p=0.25)
# Plain graph, 1000 frames of 4096 blocks x 1024 samples, burst fraction
# U(0.1, 0.9) per frame, 64 taps, H 32x32, tau = 4B.
PLAIN_LARGE = PlainWorkload("plain_F4096_B1024_T64_N32_1000fr", F=4096, B=1024, T=64, N=32,
                            frames=1000, tau=4.0 * 1024, seed=2, p=None, p_lo=0.1, p_hi=0.9)

# Differentiation: the 100-frame plain shapes with 64 taps and H 32x32; the
# L2 loss is taken against the sink output of a target graph with the same
# frames and the parameters of seed 5 (DIFF_TARGET).
DIFF = PlainWorkload("diff_F64_B256_T64_N32_100fr", F=64, B=256, T=64, N=32, frames=100,
                     tau=4.0 * 256, seed=4, p=0.25)
DIFF_TARGET_SEED = 5


@dataclass
class BatchedWorkload:
    """Many independent graph instances with uneven shapes: F log-uniform in
    [F_lo, F_hi], T drawn from ``T_choices``, per-instance burst fraction
    U(p_lo, p_hi) and tau = kappa * B with kappa ~ U(kappa_lo, kappa_hi)."""
    name: str
    instances: int
    B: int
    N: int
    seed: int
    F_lo: int = 16
    F_hi: int = 4096
    T_choices: tuple = (8, 32, 128)
    p_lo: float = 0.05
    p_hi: float = 0.95
    kappa_lo: float = 2.0
    kappa_hi: float = 8.0
    frames: int = 1
    shapes: list = field(default_factory=list)

    def __post_init__(self):
        self.shapes = []
        for i in range(self.instances):
            u = uniform(stream_key(self.seed, TAG_SHAPE, i), 0, 4)
            F = int(math.floor(math.exp(math.log(self.F_lo) + float(u[0]) * (math.log(self.F_hi) - math.log(self.F_lo)))))
            F = max(self.F_lo, min(self.F_hi, F))
            T = self.T_choices[min(int(float(u[1]) * len(self.T_choices)), len(self.T_choices) - 1)]
            p = self.p_lo + (self.p_hi - self.p_lo) * float(u[2])
            kappa = self.kappa_lo + (self.kappa_hi - self.kappa_lo) * float(u[3])
            self.shapes.append({"F": F, "T": T, "p": p, "tau": float(kappa * self.B)})

    def instance(self, i: int) -> PlainWorkload:
        s = self.shapes[i]
        return PlainWorkload(f"{self.name}[{i}]", F=s["F"], B=self.B, T=s["T"], N=self.N,
                             frames=self.frames, tau=s["tau"], seed=self.seed * 100003 + i, p=s["p"])


# 512 instances, F log-uniform in [16, 4096], B = 256, T in {8, 32, 128},
# H 64x64 per instance.
BATCHED = BatchedWorkload("batched_512x_B256_N64", instances=512, B=256, N=64, seed=3)


@dataclass
class ServingWorkload:
    """Streams of frames arriving as a Poisson process of rate ``lam`` per
    second (exponential inter-arrival times): frames per stream a log-uniform
    integer in [fr_lo, fr_hi], F a uniform integer in [F_lo, F_hi], common B,
    T and N, tau = kappa * B with kappa ~ U(kappa_lo, kappa_hi), taps and H per
    stream.  The frames are read from a device-resident pool of ``pool``
    frames of F_hi * B samples (pool frame k has burst fraction U(p_lo, p_hi)):
    stream i reads F*B-sample frames cyclically, period up to 8, from its own
    offset into the flat pool."""
    name: str
    streams: int
    lam: float
    B: int
    T: int
    N: int
    seed: int
    fr_lo: int = 10
    fr_hi: int = 10000
    F_lo: int = 64
    F_hi: int = 2048
    p_lo: float = 0.05
    p_hi: float = 0.95
    kappa_lo: float = 2.0
    kappa_hi: float = 8.0
    pool: int = 16

    def stream(self, i: int) -> dict:
        u = uniform(stream_key(self.seed, TAG_SHAPE, i), 0, 3)
        lf = math.log(self.fr_lo) + float(u[0]) * (math.log(self.fr_hi + 1) - math.log(self.fr_lo))
        frames = max(self.fr_lo, min(self.fr_hi, int(math.floor(math.exp(lf)))))
        F = self.F_lo + min(int(float(u[1]) * (self.F_hi - self.F_lo + 1)), self.F_hi - self.F_lo)
        kappa = self.kappa_lo + (self.kappa_hi - self.kappa_lo) * float(u[2])
        L, plen = F * self.B, self.pool * self.F_hi * self.B
        off = ((i * 7919) % self.pool) * self.F_hi * self.B
        period = max(1, min(8, (plen - off) // L))
        return {"F": F, "frames": frames, "tau": float(kappa * self.B), "offset": off, "period": period}

    def arrivals(self) -> list:
        """Arrival times in seconds from 0 (cumulative exponential draws)."""
        u = uniform(stream_key(self.seed, TAG_ARRIVAL), 0, self.streams)
        return torch.cumsum(-torch.log(u) / self.lam, 0).tolist()

    def taps(self, i: int, device="cpu"):
        return taps(self.seed, self.T, i, device)

    def H(self, i: int, device="cpu"):
        return hmat(self.seed, self.N, i, device)

    def pool_tensor(self, device="cpu") -> torch.Tensor:
        """The frame pool, flat complex64 [pool * F_hi * B]."""
        out = []
        for k in range(self.pool):
            p = self.p_lo + (self.p_hi - self.p_lo) * frame_uniform(self.seed, TAG_FRAC, -1, k)
            out.append(frame(self.seed, self.F_hi, self.B, p, -1, k, device).reshape(-1))
        return torch.cat(out)


# Streams arriving at 2000/s, 10..10^4 frames each, F in [64, 2048],
# B = 512, T = 32, H 64x64 per stream.
SERVING = ServingWorkload("serving_poisson2000_B512_T32_N64", streams=256, lam=2000.0, B=512, T=32, N=64, seed=5)


@dataclass
class DpdWorkload:
    """The Dynamic Predistortion stream: P periods of `period` samples of
    CN(0, var) input, K branches of T taps ~ CN(0, 1/(K T)) each, and per
    period an active set of a ~ U{a_lo..a_hi} branches drawn without
    replacement (the external configuration input)."""
    name: str
    periods: int
    period: int
    K: int
    T: int
    seed: int
    var: float = 0.25
    a_lo: int = 2
    a_hi: int = 10

    def x(self, p0: int = 0, n: int | None = None, device="cpu") -> torch.Tensor:
        n = self.periods - p0 if n is None else n
        return cnormal(stream_key(self.seed, TAG_X), n * self.period, self.var, device,
                       start=p0 * self.period).to(torch.complex64)

    def taps(self, device="cpu") -> torch.Tensor:
        return cnormal(stream_key(self.seed, TAG_TAPS), self.K * self.T, 1.0 / (self.K * self.T),
                       device).to(torch.complex64).view(self.K, self.T)

    def masks(self) -> torch.Tensor:
        out = []
        for p in range(self.periods):
            u = uniform(stream_key(self.seed, TAG_MASK, p), 0, 1 + self.K)
            a = self.a_lo + min(int(float(u[0]) * (self.a_hi - self.a_lo + 1)), self.a_hi - self.a_lo)
            order = torch.argsort(u[1:], stable=True)[:a]
            out.append(int(sum(1 << int(k) for k in order)))
        return torch.tensor(out, dtype=torch.int32)


# 67 M samples (1024 periods of 65536) as in the paper's DPD stream, 10
# branches of 10 taps, 2..10 branches active per period.
DPD = DpdWorkload("dpd_1024x65536_K10_T10", periods=1024, period=65536, K=10, T=10, seed=6)
