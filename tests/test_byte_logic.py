"""CPU checks of the byte-level tricks in pass 1's chunk tests.

Pass 1 classifies 16-pixel chunks (48 interleaved RGB bytes, twelve 32-bit
words) with byte permutes and 16-bit SIMD minima instead of per-pixel code:

* the per-channel minima of a chunk (the corner at which the density bound is
  taken), from 16-bit minima of the words and of their byte-swapped forms;
* each pixel's smallest channel, from three regrouped words per pixel pair,
  and the count of white pixels (every channel above the threshold T) from a
  carry test on four bytes at a time.

These tests restate those steps with an emulation of the two instructions
(the byte permute in its default mode, and the lane-wise unsigned 16-bit
minimum) and compare them with brute force on random chunks, for every
threshold 0..255.  The selector constants are the ones chunk_channel_min,
white_bytes and chunk_nonwhite use; a change there should be mirrored here.
"""
import numpy as np
import pytest

M32 = np.uint64(0xFFFFFFFF)


def u32(x):
    return np.asarray(x, dtype=np.uint64) & M32


def byte_perm(x, y, s):
    """Result byte i = byte (s >> 4i) & 7 of the 64-bit value y:x."""
    v = (u32(y) << np.uint64(32)) | u32(x)
    r = np.zeros_like(v)
    for i in range(4):
        sel = (s >> (4 * i)) & 7
        r |= ((v >> np.uint64(8 * sel)) & np.uint64(0xFF)) << np.uint64(8 * i)
    return r


def min_u16x2(a, b):
    a, b = u32(a), u32(b)
    lo = np.minimum(a & np.uint64(0xFFFF), b & np.uint64(0xFFFF))
    hi = np.minimum(a >> np.uint64(16), b >> np.uint64(16))
    return (hi << np.uint64(16)) | lo


def byte(x, k):
    return (x >> np.uint64(8 * k)) & np.uint64(0xFF)


def white_bytes(T):
    """(k, m) of the test: bit 7 of (b & (t | m)) | (t & m), t = (b & 0x7F) + k,
    is set exactly when b > T."""
    if T >= 127:
        return np.uint64((255 - T) * 0x01010101), np.uint64(0)
    return np.uint64((127 - T) * 0x01010101), np.uint64(0xFFFFFFFF)


def white_flags(z, T):
    k, m = white_bytes(T)
    s = u32((z & np.uint64(0x7F7F7F7F)) + k)
    return u32((z & (s | m)) | (s & m))


def chunk_channel_min(w):
    A, B = [], []
    for k in range(3):
        A.append(min_u16x2(min_u16x2(w[:, k], w[:, k + 3]), min_u16x2(w[:, k + 6], w[:, k + 9])))
        sw = [byte_perm(w[:, k + 3 * i], 0, 0x2301) for i in range(4)]
        B.append(min_u16x2(min_u16x2(sw[0], sw[1]), min_u16x2(sw[2], sw[3])))
    x1 = byte_perm(B[0], A[0], 0x5010)
    x2 = byte_perm(A[0], B[1], 0x5030)
    x3 = byte_perm(B[1], A[1], 0x7030)
    x4 = byte_perm(A[2], B[2], 0x7010)
    rg = min_u16x2(min_u16x2(x1, x2), min_u16x2(x3, x4))
    y = min_u16x2(byte_perm(B[0], A[1], 0x5030), byte_perm(A[2], B[2], 0x5030))
    bb = min_u16x2(y, y >> np.uint64(16))
    return rg, bb


def chunk_nonwhite(w, T):
    f = []
    for j in range(4):
        a, b, c = w[:, 3 * j], w[:, 3 * j + 1], w[:, 3 * j + 2]
        m01 = min_u16x2(min_u16x2(a, byte_perm(a, b, 0x4400)), byte_perm(a, b, 0x5520))
        m23 = min_u16x2(min_u16x2(u32(c << np.uint64(8)), byte_perm(b, c, 0x5520)),
                        byte_perm(b, c, 0x7330))
        f.append(white_flags(byte_perm(m01, m23, 0x7531), T))
    x = (f[0] & np.uint64(0x80808080)) | ((f[1] >> np.uint64(1)) & np.uint64(0x7F7F7F7F))
    x = (x & np.uint64(0xC0C0C0C0)) | ((f[2] >> np.uint64(2)) & np.uint64(0x3F3F3F3F))
    x = (x & np.uint64(0xE0E0E0E0)) | ((f[3] >> np.uint64(3)) & np.uint64(0x1F1F1F1F))
    x &= np.uint64(0xF0F0F0F0)
    white = np.array([bin(int(v)).count("1") for v in x])
    return 16 - white


def random_chunks(rng, n, T):
    """n chunks: uniform bytes, bytes within 3 of T, or white-ish mixes."""
    mode = rng.integers(0, 3, size=(n, 1))
    uni = rng.integers(0, 256, size=(n, 48))
    near = np.clip(T + rng.integers(-3, 4, size=(n, 48)), 0, 255)
    mix = np.where(rng.random((n, 48)) < 0.8, rng.integers(T, 256, size=(n, 48)),
                   rng.integers(0, 256, size=(n, 48)))
    by = np.where(mode == 0, uni, np.where(mode == 1, near, mix)).astype(np.uint64)
    w = np.zeros((n, 12), dtype=np.uint64)
    for i in range(48):
        w[:, i >> 2] |= by[:, i] << np.uint64(8 * (i & 3))
    return by, w


def test_byte_test_is_exactly_above_threshold():
    b = np.arange(256, dtype=np.uint64)
    z = b | (b << np.uint64(8)) | (b << np.uint64(16)) | (b << np.uint64(24))
    for T in range(256):
        f = white_flags(z, T)
        got = (f & np.uint64(0x80)) != 0
        assert np.array_equal(got, np.arange(256) > T), T


def test_channel_minima_of_a_chunk():
    rng = np.random.default_rng(11)
    by, w = random_chunks(rng, 20000, 128)
    rg, bb = chunk_channel_min(w)
    mins = by.reshape(-1, 16, 3).min(axis=1)
    assert np.array_equal(byte(rg, 1), mins[:, 0])
    assert np.array_equal(byte(rg, 3), mins[:, 1])
    assert np.array_equal(byte(bb, 1), mins[:, 2])


@pytest.mark.parametrize("T", list(range(0, 256, 5)) + [126, 127, 128, 219, 220, 221, 254, 255])
def test_nonwhite_count_of_a_chunk(T):
    rng = np.random.default_rng(1000 + T)
    by, w = random_chunks(rng, 600, T)
    ref = (by.reshape(-1, 16, 3).min(axis=2) <= T).sum(axis=1)
    assert np.array_equal(chunk_nonwhite(w, T), ref)
