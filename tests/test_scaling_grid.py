"""The tensor-core operands of BF16 and TF32 are scaled by 2^-e' with e' the block's frexp
exponent e rounded up to a multiple of 32; FP16 ones by 2^-e.  For formats with FP32's exponent
range the two scalings give the same roundings: round(x 2^-e) 2^e = round(x 2^-e') 2^e' for
every entry down to 2^-94 of the block's maximum (both scaled values are normal numbers, and
round-to-nearest-even commutes with power-of-two scaling there), and so do the split residuals
round((x 2^-e - hi) 2^s) down to 2^-80 (a residual of one unit in the last place of the scaled
entry, times 2^s, is still a normal number).  Checked here with the oracle's FP32 rounding routines on blocks of
wide dynamic range; the oracle's emulation (exact e) therefore stands for the GPU's images."""
import numpy as np
import pytest

from oracle import precision as OP


def _coarse(e: int) -> int:
    return ((e + 31) >> 5) << 5


def _scaled(x32, e):
    return np.ldexp(x32, np.int32(-e)).astype(np.float32)    # exact: a power-of-two scaling


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
@pytest.mark.parametrize("e_max", [-140, -100, -33, -1, 0, 1, 31, 32, 33, 64, 100, 127])
def test_coarse_grid_rounds_like_exact(fmt, e_max):
    g = np.random.Generator(np.random.PCG64(e_max + 1000))
    mag = np.exp2(g.uniform(-94.0, 0.0, size=4096) + (e_max - 1))
    x = (mag * g.choice([-1.0, 1.0], size=mag.shape)).astype(np.float32)
    x[0] = np.float32(np.ldexp(0.75, e_max))            # the block maximum: frexp exponent e_max
    e = OP.block_exponent(x)
    assert e == e_max
    ec = _coarse(e)
    assert -32 < e - ec <= 0
    keep = np.abs(x.astype(np.float64)) >= np.ldexp(0.75, e_max - 94)
    keep_lo = np.abs(x.astype(np.float64)) >= np.ldexp(1.0, e_max - 80)
    s = OP.lo_shift(fmt)
    out = []
    for ee in (e, ec):
        sc = _scaled(x, ee)
        hi = OP.round_to(fmt, sc)
        lo = OP.round_to(fmt, np.ldexp((sc - hi).astype(np.float32), np.int32(s)).astype(np.float32))
        out.append((np.ldexp(hi.astype(np.float64), ee), np.ldexp(lo.astype(np.float64), ee - s)))
    assert np.array_equal(out[0][0][keep], out[1][0][keep])
    assert np.array_equal(out[0][1][keep_lo], out[1][1][keep_lo])


def test_coarse_grid_values():
    assert [_coarse(e) for e in (-148, -97, -96, -95, -1, 0, 1, 32, 33, 128)] == \
        [-128, -96, -96, -64, 0, 0, 32, 32, 64, 128]
