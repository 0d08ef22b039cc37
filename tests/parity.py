"""Comparison helpers shared by the GPU parity tests (test code only)."""
import numpy as np

# Floating-point bar: max |y_gpu - y_oracle| <= TOL_REL * RMS(y_oracle).
TOL_REL = 1e-4
# Decisions E_b > tau are compared bit-exactly outside a guard band of
# GUARD_REL * |tau| around tau: the FP32 energy of the kernel differs from the
# FP64 energy of the oracle by at most about (2T + B) * 2^-24 relative
# (worst-case FP32 rounding of T products and B squares), below 1.6e-4 for
# every supported T <= 256, B <= 2048; the band is 6x that.
GUARD_REL = 1e-3


def in_band(energy, tau):
    return np.abs(energy - tau) <= GUARD_REL * max(abs(tau), 1e-30)


def compare_frame(c_g, idx_g, y_g, oracle_c, oracle_idx, oracle_y, oracle_energy, tau, B):
    """Compare one frame record.  Returns (max abs error, rms of oracle y,
    number of in-band blocks)."""
    band = in_band(oracle_energy, tau)
    idx_g = np.asarray(idx_g)[:c_g]
    sel_g = np.zeros(len(oracle_energy), bool)
    sel_g[idx_g] = True
    sel_o = np.zeros(len(oracle_energy), bool)
    sel_o[np.asarray(oracle_idx)] = True
    assert np.all(np.diff(idx_g) > 0), "idx must be strictly ascending"
    assert np.array_equal(sel_g[~band], sel_o[~band]), "decisions differ outside the guard band"
    if not band.any():
        assert c_g == oracle_c and np.array_equal(idx_g, oracle_idx)
    # y on the blocks both selected
    common = sel_g & sel_o
    pos_g = {b: j for j, b in enumerate(idx_g)}
    pos_o = {b: j for j, b in enumerate(np.asarray(oracle_idx))}
    err, ss, cnt = 0.0, 0.0, 0
    for b in np.nonzero(common)[0]:
        yo = oracle_y[pos_o[b]]
        yg = np.asarray(y_g[pos_g[b]], np.complex128)
        err = max(err, float(np.max(np.abs(yg - yo))))
        ss += float(np.sum(np.abs(yo) ** 2))
        cnt += yo.size
    rms = (ss / cnt) ** 0.5 if cnt else 0.0
    return err, rms, int(band.sum())
