"""The low-precision operand formats of the mixed solvers, restated from
their definitions on the CPU and pinned against independent conversions:

* BF16 (8 significant bits, round to nearest even) against torch's bfloat16
  cast; the split form x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
  keeps 16 significant bits, and the three products hi.hi + hi.lo + lo.hi
  miss a product by at most |lo_x lo_y| (about 2^-16 relative);
* FP8 e4m3 (bias 7, 3 fraction bits, subnormals, largest finite 448)
  against torch's float8_e4m3fn cast, and the per-tile scale s = amax / 448
  that keeps every code finite, with the quantisation error within half a
  unit in the last place (2^-4 relative, or half the subnormal step)."""
import math

import numpy as np
import pytest
import torch


def bf16_rne(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def e4m3_rne(v):
    """Nearest e4m3 value (ties to even significand), saturated at +-448."""
    out = np.empty_like(v)
    for i, x in enumerate(v):
        a = abs(x)
        if a == 0:
            out[i] = 0.0
            continue
        e = max(math.floor(math.log2(a)), -6)          # subnormals share 2^-6 scaling
        q = 2.0 ** (e - 3)                             # spacing of representable values
        m = a / q
        fl = math.floor(m)
        frac = m - fl
        n = fl + (1 if frac > 0.5 or (frac == 0.5 and fl % 2 == 1) else 0)
        val = min(n * q, 448.0)
        out[i] = math.copysign(val, x)
    return out


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-30, 30, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(bf16_rne(x), ref)


def test_split_bf16_keeps_16_bits_and_three_products():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(5000).astype(np.float32)
    y = rng.standard_normal(5000).astype(np.float32)
    hx = bf16_rne(x); lx = bf16_rne(x - hx)
    hy = bf16_rne(y); ly = bf16_rne(y - hy)
    assert np.all(np.abs((hx.astype(np.float64) + lx) - x) <= 2.0 ** -16 * np.abs(x))
    three = hx.astype(np.float64) * hy + hx.astype(np.float64) * ly + lx.astype(np.float64) * hy
    full = (hx.astype(np.float64) + lx) * (hy.astype(np.float64) + ly)
    assert np.all(np.abs(full - three) == np.abs(lx.astype(np.float64) * ly))
    assert np.all(np.abs(three - x.astype(np.float64) * y) <= 2.0 ** -14 * np.abs(x.astype(np.float64) * y))


def test_e4m3_rounding_matches_torch():
    rng = np.random.default_rng(2)
    v = (rng.uniform(-1, 1, 4000) * np.exp2(rng.integers(-12, 9, 4000))).astype(np.float32)
    v = np.clip(v, -448, 448)
    mine = e4m3_rne(v.astype(np.float64)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(mine, ref)


@pytest.mark.parametrize("amax", [1e-3, 1.0, 37.5, 1e6])
def test_tile_scale_keeps_codes_finite_and_accurate(amax):
    rng = np.random.default_rng(3)
    tile = rng.uniform(-1, 1, (128, 128)) * amax
    tile.flat[0] = amax
    s = np.abs(tile).max() / 448.0
    q = e4m3_rne((tile / s).ravel()).reshape(tile.shape)
    assert np.abs(q).max() <= 448.0
    back = q * s
    err = np.abs(back - tile)
    bound = np.maximum(2.0 ** -4 * np.abs(tile), 2.0 ** -10 * s)   # half ulp, or half the subnormal step
    assert np.all(err <= bound * (1 + 1e-12))
