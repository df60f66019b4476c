"""Integer CDF quantizer and 32-bit range coder (oracle side).

The paper codes each byte with arithmetic coding driven by Pr(i)
(Sec. 2.1, "Data Encoding"; Algorithm 1, encode and decode steps). It does
not fix the coder's precision, the CDF quantization or the flush. The
reading used here:

Quantizer. The coder's input is an FP32 probability vector p (256 entries).
  f_j = 1 + floor(fl32(p_j * 65280)), computed as one FP32 product; so every
  f_j >= 1 and the rounding decision is taken in FP32.
  The remainder T - sum(f), T = 2**16, is added to the symbol with the
  largest f (the lowest index on ties).
  cum is the exclusive prefix sum of f, with cum[256] = T.

Range coder (32-bit, carry-propagating, bytewise renormalisation).
  Encoder state: low (33 bits), range R (32 bits), one cached byte and a
  count of pending 0xFF bytes.
  Encode (cum, f): r = R >> 16; low += r*cum;
    R = R - r*cum if cum + f == T (the last symbol takes the leftover),
    else R = r*f.
  While R < 2**24: R <<= 8 and shift one byte out of low. A carry out of bit
  32 is added to the cached byte and turns pending 0xFF bytes into 0x00.
  There is no leading byte: the first cached byte is the first one written.
  Flush: the value V = low rounded up to a multiple of 2**24 lies in
  [low, low + R); its top byte is shifted out, the cache is emitted, and
  trailing zero bytes are dropped. The decoder reads missing bytes as zero.
  Decoder: code = the first 4 bytes, big-endian; r = R >> 16;
  target = min(code // r, T - 1); the symbol s has cum[s] <= target < cum[s+1];
  then code -= r*cum[s] and R is updated as in the encoder, and one byte is
  read per renormalisation shift.

Parity: pinned by an unbounded-integer restatement of the same interval
arithmetic (no carry logic), by the rational width of the exact coding
interval, by exhaustive round trips over all 2-byte inputs, and by the
closed-form quantizer cases of uniform and one-hot p
(tests/test_oracle_coder.py).
"""
from __future__ import annotations

import math

import numpy as np

T_BITS = 16
T = 1 << T_BITS
TOP = 1 << 24
MASK32 = 0xFFFFFFFF


def quantize_cdf(p32):
    """Integer frequencies and CDF from FP32 probabilities.

    ``p32``: (..., 256). Returns (f, cum): int64 arrays of shape (..., 256)
    and (..., 257).
    """
    p32 = np.asarray(p32, dtype=np.float32)
    scaled = p32 * np.float32(T - 256)          # one FP32 product per symbol
    f = np.floor(scaled).astype(np.int64) + 1
    rem = T - f.sum(axis=-1)
    am = np.argmax(f, axis=-1)                  # first maximum on ties
    np.put_along_axis(f, am[..., None], np.take_along_axis(f, am[..., None], -1) + rem[..., None], -1)
    cum = np.zeros(f.shape[:-1] + (257,), dtype=np.int64)
    np.cumsum(f, axis=-1, out=cum[..., 1:])
    return f, cum


class RangeEncoder:
    def __init__(self):
        self.low = 0
        self.range = MASK32
        self.cache = 0
        self.pending = 0
        self.started = False
        self.out = bytearray()
        self.ideal_bits = 0.0   # sum of -log2(f/T)
        self.trunc_bits = 0.0   # sum of -log2(r*T/R), the loss from R >> 16

    def _shift_low(self):
        if self.low < 0xFF000000 or self.low >= (1 << 32):
            carry = self.low >> 32
            if self.started:
                self.out.append((self.cache + carry) & 0xFF)
            for _ in range(self.pending):
                self.out.append((0xFF + carry) & 0xFF)
            self.pending = 0
            self.cache = (self.low >> 24) & 0xFF
            self.started = True
        else:
            self.pending += 1
        self.low = (self.low & 0x00FFFFFF) << 8

    def encode(self, cum: int, f: int) -> None:
        cum, f = int(cum), int(f)
        R = self.range
        r = R >> T_BITS
        self.ideal_bits += T_BITS - math.log2(f)
        self.trunc_bits += -math.log2(r * T / R)
        self.low += r * cum
        if cum + f == T:
            self.range = R - r * cum
        else:
            self.range = r * f
        while self.range < TOP:
            self.range = (self.range << 8) & MASK32
            self._shift_low()

    def finish(self) -> bytes:
        self.low = (self.low + (TOP - 1)) & ~(TOP - 1)
        self._shift_low()
        self._shift_low()
        out = bytes(self.out)
        return out.rstrip(b"\x00")


class RangeDecoder:
    def __init__(self, data: bytes):
        self.data = bytes(data)
        self.pos = 0
        self.range = MASK32
        self.code = 0
        for _ in range(4):
            self.code = (self.code << 8) | self._next()

    def _next(self) -> int:
        b = self.data[self.pos] if self.pos < len(self.data) else 0
        self.pos += 1
        return b

    def _update(self, r: int, c: int, f: int) -> None:
        self.code -= r * c
        self.range = self.range - r * c if c + f == T else r * f
        while self.range < TOP:
            self.code = ((self.code << 8) | self._next()) & MASK32
            self.range = (self.range << 8) & MASK32

    def decode(self, cum: np.ndarray) -> int:
        """Symbol for the CDF ``cum`` (257 entries, cum[256] = T)."""
        r = self.range >> T_BITS
        target = min(self.code // r, T - 1)
        s = int(np.searchsorted(cum, target, side="right")) - 1
        c = int(cum[s])
        self._update(r, c, int(cum[s + 1]) - c)
        return s

    def decode_uniform(self) -> int:
        """Symbol coded with f = 256 for every byte (the uniform prefix)."""
        r = self.range >> T_BITS
        target = min(self.code // r, T - 1)
        s = target >> 8
        self._update(r, s << 8, 256)
        return s
