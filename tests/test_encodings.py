"""The integer encodings the kernels rely on, checked exhaustively against their
definitions (no GPU; restated from the formulas, not imported from the kernels):

- the compact entry word of a group of four conditions: byte c = R | W << 2;
  with x = s XOR R, d = x - 2 [x = 3] equals |s - R|, and a DP4A of d against
  the word masked to 0x0c0c0c0c sums 4 W |s - R| (quarter units);
- the biased image byte a = 127 + K: bit 7 of a plus bit 7 of a - 1 is
  clamp(K, 0, 2) (Sections 2.1-2.2), and the accumulator stays inside its byte
  for in-degree <= 31 (edge terms 4 + (s // t) w p in [0, 8]);
- the byte-SIMD update state: drive counters below 128 and priorities
  u (tau - last) below 2^15 for T <= 128 (Section 2.2)."""
import itertools

import pytest


def _dp4a(a, b, acc):
    # signed 8-bit lanes of a times unsigned 8-bit lanes of b, summed into acc
    total = acc
    for k in range(4):
        x = (a >> (8 * k)) & 0xFF
        x = x - 256 if x >= 128 else x
        total += x * ((b >> (8 * k)) & 0xFF)
    return total


def test_entry_error_identity():
    for s, R in itertools.product(range(3), repeat=2):
        x = s ^ R
        assert x - 2 * (x == 3) == abs(s - R)
    # four conditions at once: every combination of (s, R, W) per byte
    cases = list(itertools.product(range(3), range(3), range(4)))
    for quad in itertools.product(cases, repeat=2):
        quad = quad + quad[:2]                       # 4 bytes from 2 drawn cases, repeated
        word = sum((R | W << 2) << (8 * c) for c, (_, R, W) in enumerate(quad))
        dword = 0
        for c, (s, R, _) in enumerate(quad):
            x = s ^ (((word >> (8 * c)) & 0xFF) & 3)
            dword |= ((x - 2 * (x == 3)) & 0xFF) << (8 * c)
        quarter = _dp4a(dword, word & 0x0C0C0C0C, 0)
        assert quarter == 4 * sum(W * abs(s - R) for s, R, W in quad)
        assert quarter >> 2 == sum(W * abs(s - R) for s, R, W in quad)


def _target4(a):
    # bit 7 of the byte a, plus bit 7 of a - 1 computed within the byte
    return ((a >> 7) & 1) + ((((a - 1) & 0xFF) >> 7) & 1)


@pytest.mark.parametrize("K", range(-124, 125))
def test_image_byte_target(K):
    # |K| <= 4 * 31 = 124 for in-degree <= 31, so a = 127 + K lies in [3, 251]
    assert _target4(127 + K) == min(max(K, 0), 2)


def test_image_byte_target_fails_where_the_byte_wraps():
    # a = 0 (K = -127) would wrap a - 1 to 255: the reason for the in-degree cap
    assert _target4(0) == 1 != 0


def test_image_accumulator_stays_in_its_byte():
    # an edge adds 4 + (s // t) w p, in [0, 8]; the accumulator of a node of
    # in-degree D starts at 127 - 4 D, so after D edges it is 127 + K, K in [-4D, 4D]
    terms = {4 + (s // t) * w * p for s in range(3) for t in (1, 2) for w in range(3)
             for p in (-1, 0, 1)}
    assert min(terms) == 0 and max(terms) == 8
    for D in range(0, 32):
        lo, hi = 127 - 4 * D, 127 - 4 * D + 8 * D
        assert 0 <= lo and hi <= 255                  # no carry into the next byte
        assert lo == 127 - 4 * D and hi == 127 + 4 * D
    assert 127 - 4 * 32 < 0                           # in-degree 32 could leave the byte (K = -128)


def test_update_state_widths():
    T_max, u_max = 128, 12
    assert (T_max - 1) < 128                          # a drive counter fits a byte, below its top bit
    assert u_max * (T_max - 1) < 2 ** 15              # priority in a 16-bit lane, below its top bit
