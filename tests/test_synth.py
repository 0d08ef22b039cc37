"""The seeded generator: SplitMix64 published outputs, distributions, burst
counts and determinism (the generator feeds both sides)."""
import math

import torch

from paper_1802_06625_b300 import synth


def test_splitmix64_published_sequence():
    # SplitMix64 with state 0: the first three outputs.
    assert synth.mix64(1 * synth.GOLDEN) == 0xE220A8397B1DCDAF
    assert synth.mix64(2 * synth.GOLDEN) == 0x6E789E6AA1B965F4
    assert synth.mix64(3 * synth.GOLDEN) == 0x06C45D188009454F
    # the tensor version agrees with the int version
    key = synth.stream_key(7, 1, 2)
    u = synth.uniform(key, 0, 5)
    for i in range(5):
        z = synth.mix64(key + (i + 1) * synth.GOLDEN)
        assert u[i].item() == ((z >> 11) + 0.5) * 2.0 ** -53


def test_cnormal_moments():
    z = synth.cnormal(synth.stream_key(1, 99), 200000, var=2.0)
    assert abs(z.real.mean().item()) < 0.02 and abs(z.imag.mean().item()) < 0.02
    assert abs(z.real.var().item() - 1.0) < 0.02 and abs(z.imag.var().item() - 1.0) < 0.02
    assert abs((z.real * z.imag).mean().item()) < 0.02


def test_burst_count_is_exact_and_frames_are_independent():
    w = synth.PLAIN_SMALL
    for k in range(5):
        m = synth.burst_mask(w.seed, w.F, 0.25, 0, k)
        assert int(m.sum()) == 16
    f3a = w.frame(3)
    f3b = w.frames_tensor(0, 4)[3]
    assert torch.equal(f3a, f3b)
    assert not torch.equal(w.frame(3), w.frame(4))
    e = (f3a.abs() ** 2).sum(dim=1)
    m = synth.burst_mask(w.seed, w.F, 0.25, 0, 3)
    assert e[m].min() > e[~m].max()        # x4 amplitude blocks stand out


def test_taps_and_H_variance():
    t = synth.taps(5, 4096)
    assert abs((t.abs() ** 2).mean().item() * 4096 - 1.0) < 0.1
    H = synth.hmat(5, 64)
    assert H.shape == (64, 64) and abs((H.abs() ** 2).mean().item() * 64 - 1.0) < 0.1


def test_per_frame_fraction_range():
    w = synth.PLAIN_LARGE
    ps = [w.burst_fraction(k) for k in range(50)]
    assert all(0.1 <= p <= 0.9 for p in ps) and max(ps) - min(ps) > 0.3


def test_batched_shapes():
    b = synth.BATCHED
    Fs = [s["F"] for s in b.shapes]
    assert len(Fs) == 512 and min(Fs) >= 16 and max(Fs) <= 4096
    assert {s["T"] for s in b.shapes} == {8, 32, 128}
    med = sorted(Fs)[256]
    assert 128 <= med <= 512          # log-uniform median ~ sqrt(16 * 4096) = 256
