"""The memory-level int8 F, G and G_0R of the decoder compute their bytes as f16
pairs (``op_i8x4`` / ``h4_op`` in ``polar_ops.cuh``). This checks, on the host
and for every pair of int8 LLRs in [-127, 127], the arithmetic that makes those
results the byte results bit for bit:

* a byte x enters as the f16 whose high byte is 0x64 and whose low byte is
  x ^ 0x80, i.e. 1024 + x + 128; adding -1152 (bit pattern 0xE480) leaves x;
* Eq. 1 (min of the magnitudes with the XOR of the signs), Eq. 2 (one add with
  the sign of alpha_v[i] flipped by beta_l) and G_0R are exact in f16 on these
  integers; the int8 clamp to [-127, 127] (the saturating byte add followed by
  max(-127) of Listing 4) uses the f16 constants 0xD7F0 = -127, 0x57F0 = 127;
* a result y leaves as the low byte of the f16 1280 + y (0x6500 = 1280), which is
  y's two's-complement byte, -0 included.

The GPU parity tests compare the decoders themselves with the oracle; this pins
the constants and the exactness argument the kernel code states."""
import numpy as np

F16 = np.float16


def f16(bits):
    return np.array(bits, dtype=np.uint16).view(F16)


def enter(x):
    """int8 values -> f16 the way the kernel forms them (byte permute, then +0xE480)."""
    u = (x.astype(np.int16) & 0xFF) ^ 0x80
    return (((0x64 << 8) | u).astype(np.uint16).view(F16) + f16(0xE480)).astype(F16)


def leave(h):
    """f16 results -> int8 bytes: low byte of the mantissa of 1280 + y."""
    bits = (h.astype(F16) + f16(0x6500)).astype(F16).view(np.uint16)
    return (bits & 0xFF).astype(np.uint8).view(np.int8)


def sat(v):
    return np.clip(v, -127, 127)


def pairs():
    v = np.arange(-127, 128, dtype=np.int32)
    a, b = np.meshgrid(v, v, indexing="ij")
    return a.ravel(), b.ravel()


def test_constants():
    assert f16(0xE480) == F16(-1152) and f16(0x6500) == F16(1280)
    assert f16(0xD7F0) == F16(-127) and f16(0x57F0) == F16(127)
    assert f16(0x6400) == F16(1024)


def test_enter_is_exact_and_leave_inverts_it():
    x = np.arange(-127, 128, dtype=np.int32)
    h = enter(x)
    assert np.array_equal(h.astype(np.int32), x)
    assert np.array_equal(leave(h).astype(np.int32), x)
    # every integer an unclamped sum can reach survives the way out, and -0 leaves as 0
    y = np.arange(-254, 255, dtype=np.int32)
    assert np.array_equal(leave(y.astype(F16)).astype(np.int32), ((y + 128) % 256) - 128)
    assert leave(np.array([-0.0], F16))[0] == 0


def test_f_is_eq1_exactly():
    a, b = pairs()
    ha, hb = enter(a), enter(b)
    mag = np.minimum(np.abs(ha), np.abs(hb))
    neg = np.signbit(ha) ^ np.signbit(hb)
    r = leave(np.where(neg, -mag, mag).astype(F16)).astype(np.int32)
    want = np.sign(a) * np.sign(b) * np.minimum(np.abs(a), np.abs(b))
    assert np.array_equal(r, want)


def test_g_and_g0r_are_eq2_with_int8_saturation():
    a, b = pairs()
    ha, hb = enter(a), enter(b)
    lo, hi = f16(0xD7F0), f16(0x57F0)
    for beta in (0, 1):
        flipped = (-ha if beta else ha).astype(F16)  # the sign-bit XOR of Listing 3
        s = (hb + flipped).astype(F16)
        assert np.array_equal(s.astype(np.int32), b - a if beta else b + a)  # exact
        r = leave(np.minimum(np.maximum(s, lo), hi)).astype(np.int32)
        assert np.array_equal(r, sat(b - a if beta else b + a))
    # G_0R: G with beta_l = 0
    r = leave(np.minimum(np.maximum((hb + ha).astype(F16), lo), hi)).astype(np.int32)
    assert np.array_equal(r, sat(a + b))
