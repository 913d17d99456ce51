// Device code shared by the single-image pixel passes and the batched
// persistent kernel: chunk traversal, the pass-1 window test, the exact
// radix select, and the pass-2 reconstruction of a chunk.  Every kernel that
// includes this header runs the same per-pixel arithmetic, so all of them
// produce the same densities, keys and output bytes for the same pixel.
#pragma once

#include <string.h>

#include "spcn_internal.cuh"

namespace spcn {

// ------------------------------------------------------------ traversal
struct ChunkPos {
  u64 px;           // raster index of the chunk's first pixel
  int64_t src_off;  // byte offset in the source
  int64_t dst_off;  // byte offset in the destination
  int n;            // valid pixels (16 except at row ends)
};

// One long row, 16-byte aligned, with fewer than 2^31 full chunks: the
// traversal may use 32-bit chunk indices and plain vector loads.
__device__ __forceinline__ bool flat_fast(const Geometry& g) {
  return g.flat && g.vec_src && (u64)g.npx / kChunk < (1ull << 31);
}

__device__ __forceinline__ ChunkPos chunk_pos(const Geometry& g, u64 q) {
  ChunkPos p;
  if (g.flat) {
    p.px = q * kChunk;
    const u64 left = (u64)g.npx - p.px;
    p.n = left < (u64)kChunk ? (int)left : kChunk;
    p.src_off = (int64_t)(p.px * 3);
    p.dst_off = p.src_off;
  } else {
    const u64 y = div_chunks(q, g.cpr, g.magic);
    const u64 x0 = (q - y * g.cpr) * kChunk;
    const u64 left = (u64)g.width - x0;
    p.n = left < (u64)kChunk ? (int)left : kChunk;
    p.px = y * (u64)g.width + x0;
    p.src_off = (int64_t)y * g.src_pitch + (int64_t)(x0 * 3);
    p.dst_off = (int64_t)y * g.dst_pitch + (int64_t)(x0 * 3);
  }
  return p;
}

// Geometry of an image whose rows are contiguous in both source and
// destination (one long row): the traversal needs only the two base
// pointers and the pixel count, which keeps loops over tiles whose geometry
// comes from memory (not from kernel parameters) within the register budget.
struct FlatGeometry {
  const uint8_t* src;
  uint8_t* dst;
  u64 npx;
  int vec_src, vec_dst;
#ifdef SPCN_CHECKED
  int64_t src_bytes, dst_bytes;
  int* err;
#endif
};

__device__ __forceinline__ ChunkPos chunk_pos(const FlatGeometry& g, u64 q) {
  ChunkPos p;
  p.px = q * kChunk;
  const u64 left = g.npx - p.px;
  p.n = left < (u64)kChunk ? (int)left : kChunk;
  p.src_off = (int64_t)(p.px * 3);
  p.dst_off = p.src_off;
  return p;
}

__device__ __forceinline__ unsigned byte_at(const unsigned (&w)[12], int i) {
  return (w[i >> 2] >> ((i & 3) * 8)) & 0xFFu;
}

// Load a chunk into 12 little-endian words; STREAM selects the evict-first
// policy for data read for the last time.  Pixels past the end of a row read
// as 0xFF bytes, so every chunk takes the same unrolled path: their outputs
// are never stored, and pass 1 counts a row's partial chunk pixel by pixel
// (at white threshold 255 the padding would not read as white).
template <bool STREAM, class G>
__device__ __forceinline__ void load_chunk(const G& g, const ChunkPos& p,
                                           unsigned (&w)[12]) {
  if (!SPCN_CHECK(p.src_off >= 0 && p.n >= 0 && p.n <= kChunk &&
                  p.src_off + 3 * (int64_t)p.n <= g.src_bytes, g.err)) {
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = 0xFFFFFFFFu;
    return;
  }
  const uint8_t* s = g.src + p.src_off;
  if (p.n == kChunk && g.vec_src) {
    const uint4* v = reinterpret_cast<const uint4*>(s);
    uint4 a, b, c;
    if (STREAM) {
      a = __ldcs(v); b = __ldcs(v + 1); c = __ldcs(v + 2);
    } else {
      a = __ldg(v); b = __ldg(v + 1); c = __ldg(v + 2);
    }
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = 0xFFFFFFFFu;
    const int nb = 3 * p.n;
#pragma unroll
    for (int i = 0; i < 48; ++i)
      if (i < nb) w[i >> 2] = (w[i >> 2] & ~(0xFFu << ((i & 3) * 8))) |
                              ((unsigned)__ldg(s + i) << ((i & 3) * 8));
  }
}

template <class G>
__device__ __forceinline__ void store_chunk(const G& g, const ChunkPos& p,
                                            const unsigned (&o)[12]) {
  if (!SPCN_CHECK(p.dst_off >= 0 && p.n >= 0 && p.n <= kChunk &&
                  p.dst_off + 3 * (int64_t)p.n <= g.dst_bytes, g.err))
    return;
  uint8_t* d = g.dst + p.dst_off;
  if (p.n == kChunk && g.vec_dst) {
    uint4* v = reinterpret_cast<uint4*>(d);
    __stcs(v, make_uint4(o[0], o[1], o[2], o[3]));
    __stcs(v + 1, make_uint4(o[4], o[5], o[6], o[7]));
    __stcs(v + 2, make_uint4(o[8], o[9], o[10], o[11]));
  } else {
    const int nb = 3 * p.n;
#pragma unroll
    for (int i = 0; i < 48; ++i)
      if (i < nb) d[i] = (uint8_t)byte_at(o, i);
  }
}

// Table offsets of the three channels of pixel k of a chunk.
__device__ __forceinline__ void pixel_addr(const unsigned (&w)[12], int k, unsigned lr,
                                           unsigned& aR, unsigned& aG, unsigned& aB) {
  const int o = 3 * k;
  aR = lut_addr(w[o >> 2], lr, o & 3);
  aG = lut_addr(w[(o + 1) >> 2], lr, (o + 1) & 3);
  aB = lut_addr(w[(o + 2) >> 2], lr, (o + 2) & 3);
}

// Strided loop over chunks q = q0, q0 + stride, ... < n; body(w, pos) is
// called for every chunk.  With PREFETCH the next chunk's loads are issued
// before the current chunk is processed (two register buffers, so no
// copies); the issue-bound pass 1 runs faster without it, the
// bandwidth-bound pass 2 with it.
template <bool STREAM, bool PREFETCH, class G, class Body>
__device__ __forceinline__ void for_chunks(const G& g, u64 q, u64 n, u64 stride,
                                           Body&& body) {
  if (!PREFETCH) {
    for (; q < n; q += stride) {
      const ChunkPos p = chunk_pos(g, q);
      unsigned w[12];
      load_chunk<STREAM>(g, p, w);
      body(w, p);
    }
    return;
  }
  unsigned wa[12], wb[12];
  ChunkPos pa, pb;
  if (q < n) { pa = chunk_pos(g, q); load_chunk<STREAM>(g, pa, wa); }
  while (q < n) {
    u64 qn = q + stride;
    if (qn < n) { pb = chunk_pos(g, qn); load_chunk<STREAM>(g, pb, wb); }
    body(wa, pa);
    q = qn;
    if (q >= n) break;
    qn = q + stride;
    if (qn < n) { pa = chunk_pos(g, qn); load_chunk<STREAM>(g, pa, wa); }
    body(wb, pb);
    q = qn;
  }
}

// Persistent grid-stride loop over all chunks of an image.
template <bool STREAM, bool PREFETCH, class Body>
__device__ __forceinline__ void for_each_chunk(const Geometry& g, Body&& body) {
  for_chunks<STREAM, PREFETCH>(g, (u64)blockIdx.x * blockDim.x + threadIdx.x, g.nchunks,
                               (u64)gridDim.x * blockDim.x, body);
}

// ------------------------------------------------------------ pass 1
// Per-launch constants of pass 1, held in registers by the pixel loop.
struct WindowConst {
  u64* fine;
  unsigned wthr, lo0, lo1, nb0, nb1;
  float nk0, lk0, nk1, lk1;   // sat(h~ nk + lk) = [h~ < lo]   (exact, see window_of)
  float nh0, hk0, nh1, hk1;   // sat(h~ nh + hk) = [h~ < lo + nb]
};

// Fire-and-forget increments (no return value, no compiler-side aggregation).
__device__ __forceinline__ void red_add_global(u64* p, u64 v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(unsigned* p, unsigned v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void window_hit(const WindowConst& C, unsigned* s_coarse, unsigned r1,
                                           unsigned r2) {
  if (r1 < C.nb0) {
    red_add_global(C.fine + r1, 1ull);
    red_add_shared(s_coarse + (r1 >> kWinGroupBits), 1u);
  }
  if (r2 < C.nb1) {
    red_add_global(C.fine + kWinBins + r2, 1ull);
    red_add_shared(s_coarse + kWinGroups + (r2 >> kWinGroupBits), 1u);
  }
}

// Pass 1 on one chunk.  Per pixel, all on the FMA pipe: the non-white flag
// (as 0/1), [h~ < lo] and [h~ < hi] per stain by saturated FMAs, accumulated
// with packed FMAs.  The number of windows a pixel falls in (0, 1 or 2) is
// packed base 4 into `mask` (pixel pair p at digit 7-p, even pixels in the
// low lane, odd pixels in the high lane): exact small integers in FP32.
// WHITES_BELOW: every white pixel is known to lie below both window starts
// (see whites_below), so the pixels are not masked by their non-white flag:
// a white pixel adds 1 to each below count, which the caller has subtracted
// (with the chunk's non-white count added) when it classified the chunk, and
// is never in a window.
template <bool PINV = false, bool WHITES_BELOW = false>
__device__ __forceinline__ void window_chunk(const unsigned (&w)[12], const char* lut,
                                             unsigned lr, f2 NR1, f2 NR2, float kappa,
                                             const WindowConst& a, f2& c_nw, f2& c_b0, f2& c_b1,
                                             f2& mask) {
  const f2 M1 = pk(-1.f, -1.f), FOUR = pk(4.f, 4.f);
  mask = pk(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < kChunk / 2; ++p) {
    const int kA = 2 * p, kB = 2 * p + 1;
    unsigned aRA, aGA, aBA, aRB, aGB, aBB;
    pixel_addr(w, kA, lr, aRA, aGA, aBA);
    pixel_addr(w, kB, lr, aRB, aGB, aBB);
    f2 H1, H2;
    solve_pair<PINV>(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, kappa, H1, H2);
    const float h1A = lo_of(H1), h1B = hi_of(H1), h2A = lo_of(H2), h2B = hi_of(H2);
    const f2 B0 = pk(fma_sat(h1A, a.nk0, a.lk0), fma_sat(h1B, a.nk0, a.lk0));
    const f2 B1 = pk(fma_sat(h2A, a.nk1, a.lk1), fma_sat(h2B, a.nk1, a.lk1));
    const f2 T0 = pk(fma_sat(h1A, a.nh0, a.hk0), fma_sat(h1B, a.nh0, a.hk0));
    const f2 T1 = pk(fma_sat(h2A, a.nh1, a.hk1), fma_sat(h2B, a.nh1, a.hk1));
    // T - B is 1 exactly for an in-window density
    const f2 X = add2(fma2(B0, M1, T0), fma2(B1, M1, T1));
    if (WHITES_BELOW) {
      c_b0 = add2(c_b0, B0);
      c_b1 = add2(c_b1, B1);
      mask = fma2(mask, FOUR, X);
    } else {
      const bool nwA = min(min(aRA, aGA), aBA) < a.wthr;
      const bool nwB = min(min(aRB, aGB), aBB) < a.wthr;
      const f2 NW = pk(nwA ? 1.f : 0.f, nwB ? 1.f : 0.f);
      c_nw = add2(c_nw, NW);
      c_b0 = fma2(B0, NW, c_b0);
      c_b1 = fma2(B1, NW, c_b1);
      mask = fma2(mask, FOUR, mul2(X, NW));
    }
  }
}

// Per-warp stack of full tissue chunks (data and chunk index).
__device__ __forceinline__ void stack_put(uint4* stk, unsigned* stq, int slot,
                                          const unsigned (&w)[12], unsigned qi) {
  uint4* d = stk + 3 * slot;
  d[0] = make_uint4(w[0], w[1], w[2], w[3]);
  d[1] = make_uint4(w[4], w[5], w[6], w[7]);
  d[2] = make_uint4(w[8], w[9], w[10], w[11]);
  stq[slot] = qi;
}
__device__ __forceinline__ void stack_get(const uint4* stk, const unsigned* stq, int slot,
                                          unsigned (&w)[12], unsigned& qi) {
  const uint4* d = stk + 3 * slot;
  const uint4 a = d[0], b = d[1], c = d[2];
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
  w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
  qi = stq[slot];
}

// Conservative all-white test of a full chunk: every byte has the top bits
// of wm set, which puts it above the white threshold (no padding in a full
// chunk).  Such chunks add nothing to any count of pass 1.
__device__ __forceinline__ bool chunk_white(const unsigned (&w)[12], unsigned wm, unsigned we) {
  unsigned acc = w[0];
#pragma unroll
  for (int i = 1; i < 12; ++i) acc &= w[i];
  return (acc & wm) == we;
}

// Lane-wise minimum of two 16-bit pairs (native on this GPU).  The high
// byte of a 16-bit minimum is the minimum of the high bytes whatever the low
// bytes hold, which the per-channel minima below rely on.
__device__ __forceinline__ unsigned min_u16x2(unsigned a, unsigned b) {
  unsigned r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// Per-channel minima of a full chunk (16 interleaved RGB pixels in 12
// words): words 3i, 3i+1, 3i+2 carry the byte patterns [R G B R],
// [G B R G], [B R G B].  16-bit minima of the words give the minima of their
// bytes 1 and 3, of the byte-swapped words those of bytes 0 and 2; the
// twelve candidates are then regathered into high bytes and reduced.  Returns
// (min R, min G) in bytes 1 and 3 of *rg and min B in byte 1 of *bb.
__device__ __forceinline__ void chunk_channel_min(const unsigned (&w)[12], unsigned* rg,
                                                  unsigned* bb) {
  unsigned A[3], B[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A[k] = min_u16x2(min_u16x2(w[k], w[k + 3]), min_u16x2(w[k + 6], w[k + 9]));
    B[k] = min_u16x2(min_u16x2(__byte_perm(w[k], 0u, 0x2301u), __byte_perm(w[k + 3], 0u, 0x2301u)),
                     min_u16x2(__byte_perm(w[k + 6], 0u, 0x2301u), __byte_perm(w[k + 9], 0u, 0x2301u)));
  }
  const unsigned x1 = __byte_perm(B[0], A[0], 0x5010u);   // R: B0.b1   G: A0.b1
  const unsigned x2 = __byte_perm(A[0], B[1], 0x5030u);   // R: A0.b3   G: B1.b1
  const unsigned x3 = __byte_perm(B[1], A[1], 0x7030u);   // R: B1.b3   G: A1.b3
  const unsigned x4 = __byte_perm(A[2], B[2], 0x7010u);   // R: A2.b1   G: B2.b3
  *rg = min_u16x2(min_u16x2(x1, x2), min_u16x2(x3, x4));
  const unsigned y = min_u16x2(__byte_perm(B[0], A[1], 0x5030u),    // B0.b3, A1.b1
                               __byte_perm(A[2], B[2], 0x5030u));   // A2.b3, B2.b1
  *bb = min_u16x2(y, y >> 16);
}

// True when every pixel of a full chunk is below both window starts: the
// densities' bound D~ at the per-channel minima rg (R in byte 1, G in byte 3)
// and bb (B in byte 1), with the same table sums and saturation as
// solve_one, passes the window's exact test.  Every
// table entry is non-increasing in the intensity (W >= 0), FP32 addition and
// the saturation are monotone, and h~ = min(D~, t) <= D~, so each pixel's
// test gives the same 1.  (Not for the pseudo-inverse, whose rows may be
// negative.)
__device__ __forceinline__ bool below_bound(unsigned rg, unsigned bb, const char* lut,
                                            unsigned lr, const WindowConst& C) {
  // table offsets: the intensity in byte 1, the lane's copy in byte 0
  const float2 eR = lut_ld(lut, __byte_perm(rg, lr, 0x5514u));
  const float2 eG = lut_ld(lut, __byte_perm(rg, lr, 0x5534u) + kLutOffG);
  const float2 eB = lut_ld(lut, __byte_perm(bb, lr, 0x5514u) + kLutOffB);
  const float D1 = add_sat(eR.x + eG.x, eB.x);
  const float D2 = add_sat(eR.y + eG.y, eB.y);
  return fma_sat(D1, C.nk0, C.lk0) == 1.f && fma_sat(D2, C.nk1, C.lk1) == 1.f;
}
__device__ __forceinline__ bool chunk_below_window(const unsigned (&w)[12], const char* lut,
                                                   unsigned lr, const WindowConst& C) {
  unsigned rg, bb;
  chunk_channel_min(w, &rg, &bb);
  return below_bound(rg, bb, lut, lr, C);
}

// The bound itself: D~ of both stains at the chunk's per-channel minima, as
// FP32 bit patterns (keys), at or above the key of every pixel's density.
__device__ __forceinline__ void chunk_bound_keys(const unsigned (&w)[12], const char* lut,
                                                 unsigned lr, unsigned* k1, unsigned* k2) {
  unsigned rg, bb;
  chunk_channel_min(w, &rg, &bb);
  const float2 eR = lut_ld(lut, __byte_perm(rg, lr, 0x5514u));
  const float2 eG = lut_ld(lut, __byte_perm(rg, lr, 0x5534u) + kLutOffG);
  const float2 eB = lut_ld(lut, __byte_perm(bb, lr, 0x5514u) + kLutOffB);
  *k1 = __float_as_uint(add_sat(eR.x + eG.x, eB.x));
  *k2 = __float_as_uint(add_sat(eR.y + eG.y, eB.y));
}

// True when every white pixel (all channels above the threshold T) lies
// below both window starts: the same bound at the intensities (T+1, T+1,
// T+1), which every white pixel's channels reach or exceed.  At T = 255 no
// pixel is white.  The same value on every thread.
__device__ __forceinline__ bool whites_below(unsigned T, const char* lut, unsigned lr,
                                             const WindowConst& C) {
  if (T >= 255u) return true;
  const unsigned t1 = T + 1u;
  return below_bound((t1 << 8) | (t1 << 24), t1 << 8, lut, lr, C);
}

// Constants of the byte test "above the white threshold T" used by
// chunk_nonwhite: with t = (b & 0x7F) + k, bit 7 of (b & (t | m)) | (t & m)
// is set exactly when b > T (k = 255 - T, m = 0 for T >= 127: b needs its top
// bit and the low bits must carry; k = 127 - T, m = ~0 below: either does).
struct WhiteBytes {
  unsigned k, m;
};
__device__ __forceinline__ WhiteBytes white_bytes(unsigned T) {
  return T >= 127u ? WhiteBytes{(255u - T) * 0x01010101u, 0u}
                   : WhiteBytes{(127u - T) * 0x01010101u, 0xFFFFFFFFu};
}

// Non-white pixels of a full chunk (some channel at or below the threshold).
// Four pixels are three words a = [R0 G0 B0 R1], b = [G1 B1 R2 G2],
// c = [B2 R3 G3 B3].  Three words per pixel pair carry the pair's channels in
// the high bytes of their 16-bit lanes (a itself, two byte permutes of a and
// b for pixels 0-1; c << 8 and two permutes of b and c for pixels 2-3), so two
// 16-bit minima give each pixel's smallest channel; the four minima are
// gathered into one word and tested once (white: minimum above T).  The four
// groups' flags are merged into bits 7..4 of each byte for one bit count.
__device__ __forceinline__ float chunk_nonwhite(const unsigned (&w)[12], const WhiteBytes& t) {
  unsigned f[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned a = w[3 * j], b = w[3 * j + 1], c = w[3 * j + 2];
    const unsigned m01 = min_u16x2(min_u16x2(a, __byte_perm(a, b, 0x4400u)),   // G0 R1, R0 G1
                                   __byte_perm(a, b, 0x5520u));                 // B0 B1
    const unsigned m23 = min_u16x2(min_u16x2(c << 8, __byte_perm(b, c, 0x5520u)),   // B2 G3, R2 R3
                                   __byte_perm(b, c, 0x7330u));                      // G2 B3
    const unsigned z = __byte_perm(m01, m23, 0x7531u);   // the four pixels' minima
    const unsigned s = (z & 0x7F7F7F7Fu) + t.k;
    f[j] = (z & (s | t.m)) | (s & t.m);   // bit 7 of each byte: the pixel is white
  }
  unsigned x = (f[0] & 0x80808080u) | ((f[1] >> 1) & 0x7F7F7F7Fu);
  x = (x & 0xC0C0C0C0u) | ((f[2] >> 2) & 0x3F3F3F3Fu);
  x = (x & 0xE0E0E0E0u) | ((f[3] >> 3) & 0x1F1F1F1Fu);
  return (float)(kChunk - __popc(x & 0xF0F0F0F0u));
}

// chunk_nonwhite and, from the same regrouped words, the chunk's
// per-channel minima in the layout of chunk_channel_min (R in byte 1 and G in
// byte 3 of *rg, B in byte 1 of *bb).  Per group of four pixels the six
// words a, P, Q (pixels 0-1) and C8, Q2, P2 (pixels 2-3) carry, in the high
// bytes of their 16-bit lanes, the channels (G0, R1), (R0, G1), (B0, B1),
// (B2, G3), (R2, R3) and (G2, B3); 16-bit minima over the groups keep those
// high bytes' minima per word type, and six lane swaps and minima gather
// them by channel.
__device__ __forceinline__ float chunk_nonwhite_min(const unsigned (&w)[12], const WhiteBytes& t,
                                                    unsigned* rg, unsigned* bb) {
  unsigned f[4];
  unsigned ka = 0u, kp = 0u, kq = 0u, kc = 0u, kq2 = 0u, kp2 = 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned a = w[3 * j], b = w[3 * j + 1], c = w[3 * j + 2];
    const unsigned P = __byte_perm(a, b, 0x4400u), Q = __byte_perm(a, b, 0x5520u);
    const unsigned C8 = c << 8, Q2 = __byte_perm(b, c, 0x5520u), P2 = __byte_perm(b, c, 0x7330u);
    const unsigned m01 = min_u16x2(min_u16x2(a, P), Q);
    const unsigned m23 = min_u16x2(min_u16x2(C8, Q2), P2);
    const unsigned z = __byte_perm(m01, m23, 0x7531u);   // the four pixels' minima
    const unsigned s = (z & 0x7F7F7F7Fu) + t.k;
    f[j] = (z & (s | t.m)) | (s & t.m);   // bit 7 of each byte: the pixel is white
    if (j == 0) {
      ka = a; kp = P; kq = Q; kc = C8; kq2 = Q2; kp2 = P2;
    } else {
      ka = min_u16x2(ka, a); kp = min_u16x2(kp, P); kq = min_u16x2(kq, Q);
      kc = min_u16x2(kc, C8); kq2 = min_u16x2(kq2, Q2); kp2 = min_u16x2(kp2, P2);
    }
  }
  const unsigned x1 = min_u16x2(__byte_perm(ka, 0u, 0x1032u), kp);    // (R, G)
  const unsigned y = min_u16x2(kc, __byte_perm(kp2, 0u, 0x1032u));    // (B, G)
  const unsigned r2 = min_u16x2(kq2, __byte_perm(kq2, 0u, 0x1032u));  // (R, R)
  const unsigned b2 = min_u16x2(kq, __byte_perm(kq, 0u, 0x1032u));    // (B, B)
  *rg = min_u16x2(x1, __byte_perm(r2, y, 0x7610u));                   // (R, G)
  *bb = min_u16x2(y, b2);                                              // (B, -)
  unsigned x = (f[0] & 0x80808080u) | ((f[1] >> 1) & 0x7F7F7F7Fu);
  x = (x & 0xC0C0C0C0u) | ((f[2] >> 2) & 0x3F3F3F3Fu);
  x = (x & 0xE0E0E0E0u) | ((f[3] >> 3) & 0x1F1F1F1Fu);
  return (float)(kChunk - __popc(x & 0xF0F0F0F0u));
}

constexpr int kWarpQueue = 64;    // queue entries per warp; drained as soon as 32 are waiting, so
                                  // the re-read pixels are recent enough to still be in L2

// ------------------------------------------------------------ radix fallback
struct ImageSource {
  Geometry g;
  unsigned thr;
  template <class F>
  __device__ __forceinline__ void for_each(F&& f) const {
    const unsigned lr = lane_reg();
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < g.nchunks; q += stride) {
      const ChunkPos p = chunk_pos(g, q);
      unsigned w[12];
      load_chunk<false>(g, p, w);
      for (int k = 0; k < p.n; ++k) {
        const unsigned r = byte_at(w, 3 * k), gg = byte_at(w, 3 * k + 1), b = byte_at(w, 3 * k + 2);
        unsigned aR, aG, aB;
        pixel_addr(w, k, lr, aR, aG, aB);
        f(aR, aG, aB, min(r, min(gg, b)) <= thr);
      }
    }
  }
};

struct ListSource {
  const uint32_t* items;   // packed R | G<<8 | B<<16, all non-white; 16-byte aligned
  u64 n;
  unsigned sub;            // 1: every item; s > 1: the groups of four items 0, s, 2s, ... only
  // Items visited (the population the select ranks).
  __host__ __device__ static u64 visited(u64 n, unsigned sub) {
    return sub > 1 ? 4 * (((n >> 2) + sub - 1) / sub) : n;
  }
  template <class F>
  __device__ __forceinline__ void for_each(F&& f) const {
    const unsigned lr = lane_reg();
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    // four items per 16-byte load, then the tail
    const uint4* v4 = reinterpret_cast<const uint4*>(items);
    const u64 n4 = n >> 2;
    for (u64 i = t * sub; i < n4; i += stride * sub) {
      const uint4 v = __ldg(v4 + i);
      f(lut_addr(v.x, lr, 0), lut_addr(v.x, lr, 1), lut_addr(v.x, lr, 2), true);
      f(lut_addr(v.y, lr, 0), lut_addr(v.y, lr, 1), lut_addr(v.y, lr, 2), true);
      f(lut_addr(v.z, lr, 0), lut_addr(v.z, lr, 1), lut_addr(v.z, lr, 2), true);
      f(lut_addr(v.w, lr, 0), lut_addr(v.w, lr, 1), lut_addr(v.w, lr, 2), true);
    }
    if (sub > 1) return;
    for (u64 i = (n4 << 2) + t; i < n; i += stride) {
      const uint32_t v = __ldg(items + i);
      f(lut_addr(v, lr, 0), lut_addr(v, lr, 1), lut_addr(v, lr, 2), true);
    }
  }
};

// Exact radix select (11/11/10-bit digits of the FP32 key of the scaled
// densities) of the ranks rank[] whose track is active, over every non-white
// pixel of `src`.  All blocks of a cooperative grid call it; it uses four
// grid barriers (counter `bar`, zeroed before the launch).  Block 0 writes the
// keys, the percentiles and the scale factors.  Returns false if a wait gave
// up (the error is recorded).
template <bool PINV, class Src>
__device__ bool radix_select(const Src& src, const char* lut, const Lasso& L, SelectState* s,
                             const u64 (&rank)[kTracks], const int (&active)[kTracks],
                             u64* ghist, unsigned* s_hist, unsigned* bar, int* err,
                             long long timeout_ns, double tgt0, double tgt1) {
  __shared__ unsigned s_prefix[kTracks];
  __shared__ u64 s_r[kTracks];
  __shared__ int s_act[kTracks];
  __shared__ int s_idx4[kTracks];
  __shared__ u64 s_before4[kTracks];
  __shared__ u64 s_tmp[33];
  if (threadIdx.x == 0) {
    for (int t = 0; t < kTracks; ++t) {
      s_act[t] = active[t];
      s_prefix[t] = 0u;
      s_r[t] = rank[t];
    }
  }
  const u64 gstride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < 3ull * kTracks * kRadixBins; i += gstride)
    ghist[i] = 0ull;
  unsigned target = gridDim.x;
  if (!grid_barrier(bar, target, &s->abort, err, timeout_ns)) return false;
  for (int d = 0; d < 3; ++d) {
    const int shift = d == 0 ? 21 : (d == 1 ? 10 : 0);
    const int hi = d == 0 ? 32 : (d == 1 ? 21 : 10);
    const unsigned mask = d == 2 ? 0x3FFu : 0x7FFu;
    for (int i = threadIdx.x; i < kTracks * kRadixBins; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    unsigned pre[kTracks];
    int act[kTracks], own[kTracks];
#pragma unroll
    for (int t = 0; t < kTracks; ++t) { pre[t] = s_prefix[t]; act[t] = s_act[t]; }
    // the two ranks of a stain share one histogram while their prefixes agree
#pragma unroll
    for (int t = 0; t < kTracks; ++t)
      own[t] = ((t & 1) && act[t] && act[t - 1] && pre[t] == pre[t - 1]) ? t - 1 : t;
    src.for_each([&](unsigned aR, unsigned aG, unsigned aB, bool nw) {
      float h1, h2;
      solve_one<PINV>(lut, aR, aG, aB, L, h1, h2);
      const unsigned key[2] = {PINV ? signed_key(__float_as_uint(h1)) : __float_as_uint(h1),
                               PINV ? signed_key(__float_as_uint(h2)) : __float_as_uint(h2)};
      const unsigned live = __activemask();
#pragma unroll
      for (int t = 0; t < kTracks; ++t) {
        if (own[t] != t || !act[t]) continue;   // uniform across the block
        const unsigned k = key[t >> 1];
        const bool in = nw && (((u64)k >> hi) == ((u64)pre[t] >> hi));
        // warp-aggregated increment: one atomic per distinct bin in the warp
        const unsigned bin = in ? ((k >> shift) & mask) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(live, bin);
        if (in && (__ffs(peers) - 1) == (int)(threadIdx.x & 31u))
          atomicAdd(s_hist + t * kRadixBins + bin, (unsigned)__popc(peers));
      }
    });
    __syncthreads();
    u64* gh = ghist + (size_t)d * kTracks * kRadixBins;
    for (int i = threadIdx.x; i < kTracks * kRadixBins; i += blockDim.x)
      if (s_hist[i]) atomicAdd(gh + i, (u64)s_hist[i]);
    target += gridDim.x;
    if (!grid_barrier(bar, target, &s->abort, err, timeout_ns)) return false;
    {   // the digit of every active track at once
      const u64* const hs[kTracks] = {gh + (size_t)own[0] * kRadixBins, gh + (size_t)own[1] * kRadixBins,
                                      gh + (size_t)own[2] * kRadixBins, gh + (size_t)own[3] * kRadixBins};
      const u64 rr[kTracks] = {s_r[0], s_r[1], s_r[2], s_r[3]};
      const int aa[kTracks] = {s_act[0], s_act[1], s_act[2], s_act[3]};
      block_find_rank4(hs, kRadixBins, rr, aa, s_idx4, s_before4, s_tmp);
    }
    if (threadIdx.x == 0) {
      for (int t = 0; t < kTracks; ++t) {
        if (!s_act[t]) continue;
        if (s_idx4[t] < 0) {     // fewer pixels than the rank: cannot happen
          record_error(err, SPCN_ERR_CUDA);
          s_act[t] = 0;
        } else {
          s_prefix[t] |= (unsigned)s_idx4[t] << shift;
          s_r[t] -= s_before4[t];
        }
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int t = 0; t < kTracks; ++t)
      if (s_act[t]) { s->key[t] = PINV ? signed_key_inv(s_prefix[t]) : s_prefix[t]; s->resolved[t] = 1; }
    finish_percentiles(s, tgt0, tgt1, L.hscale);
    __threadfence();
    s->all_resolved = 1;
  }
  return true;
}

// ------------------------------------------------------------ pass 2
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Four rounded values (byte 0 of each word) packed little-endian.
__device__ __forceinline__ unsigned pack4(unsigned a, unsigned b, unsigned c, unsigned d) {
  return __byte_perm(__byte_perm(a, b, 0x0040u), __byte_perm(c, d, 0x0040u), 0x5410u);
}

struct ReconConst {
  f2 M1[3], M2[3], L2[3];   // exponent: e_c = L2_c + M1_c h~1 + M2_c h~2 (both lanes equal)
};

// Eq. 1-2 projection of pass 2: d_j = sum_c pa[3j+c] v_c + pb[j], i.e. the
// projected table's s (W[:,j].v - lambda) / G_jj computed with FMAs from the
// optical densities (FP32; within a few ulp of the table's single rounding).
struct ProjConst {
  f2 A10, A11, A20, A21, B1, B2;   // pa[0], pa[1], pa[3], pa[4], pb[0], pb[1] in both lanes
  float a12, a22;                  // pa[2], pa[5]
};

__device__ __forceinline__ ProjConst proj_const(const Model* m) {
  ProjConst P;
  P.A10 = pk(m->pa[0], m->pa[0]);
  P.A11 = pk(m->pa[1], m->pa[1]);
  P.a12 = m->pa[2];
  P.A20 = pk(m->pa[3], m->pa[3]);
  P.A21 = pk(m->pa[4], m->pa[4]);
  P.a22 = m->pa[5];
  P.B1 = pk(m->pb[0], m->pb[0]);
  P.B2 = pk(m->pb[1], m->pb[1]);
  return P;
}

__device__ __forceinline__ float od_ld(const char* lut, unsigned off) {
  return *reinterpret_cast<const float*>(lut + off);
}

// The closed-form H-step of two pixels from the optical-density table.
template <bool PINV = false>
__device__ __forceinline__ void solve_pair_od(const char* lut, unsigned aRA, unsigned aGA,
                                              unsigned aBA, unsigned aRB, unsigned aGB,
                                              unsigned aBB, const ProjConst& P, f2 NR1, f2 NR2,
                                              float kappa, f2& H1, f2& H2) {
  const float vRA = od_ld(lut, aRA), vGA = od_ld(lut, aGA + kLutOffG), vBA = od_ld(lut, aBA + kLutOffB);
  const float vRB = od_ld(lut, aRB), vGB = od_ld(lut, aGB + kLutOffG), vBB = od_ld(lut, aBB + kLutOffB);
  const f2 VR = pk(vRA, vRB), VG = pk(vGA, vGB);
  const f2 S1 = fma2(P.A11, VG, fma2(P.A10, VR, P.B1));
  const f2 S2 = fma2(P.A21, VG, fma2(P.A20, VR, P.B2));
  if (PINV) {   // pinv(W) v with FMAs (B = 0): signed, no sparsity
    H1 = pk(fmaf(P.a12, vBA, lo_of(S1)), fmaf(P.a12, vBB, hi_of(S1)));
    H2 = pk(fmaf(P.a22, vBA, lo_of(S2)), fmaf(P.a22, vBB, hi_of(S2)));
    return;
  }
  const float D1A = fma_sat(P.a12, vBA, lo_of(S1)), D1B = fma_sat(P.a12, vBB, hi_of(S1));
  const float D2A = fma_sat(P.a22, vBA, lo_of(S2)), D2B = fma_sat(P.a22, vBB, hi_of(S2));
  const f2 P1 = pk(D1A, D1B), P2 = pk(D2A, D2B);
  const f2 Q1 = fma2(NR1, P2, P1);
  const f2 Q2 = fma2(NR2, P1, P2);
  const float t1A = mul_sat(kappa, lo_of(Q1)), t1B = mul_sat(kappa, hi_of(Q1));
  const float t2A = mul_sat(kappa, lo_of(Q2)), t2B = mul_sat(kappa, hi_of(Q2));
  H1 = pk(fminf(D1A, t1A), fminf(D1B, t1B));
  H2 = pk(fminf(D2A, t2A), fminf(D2B, t2B));
}

// Pass 2 on one chunk (optical-density table, lane register lane_reg_od()).
// With the lasso every exponent is <= log2(i0) <= 8, so the value stays in
// [0, 255]; signed pseudo-inverse densities can exceed i0 and are clamped.
template <bool PINV = false>
__device__ __forceinline__ void recon_chunk(const unsigned (&w)[12], const char* lut,
                                            unsigned lr, const ProjConst& P, f2 NR1, f2 NR2,
                                            float kappa, const ReconConst& K, unsigned (&o)[12]) {
  unsigned y[48];
#pragma unroll
  for (int p = 0; p < kChunk / 2; ++p) {
    const int kA = 2 * p, kB = 2 * p + 1;
    unsigned aRA, aGA, aBA, aRB, aGB, aBB;
    pixel_addr(w, kA, lr, aRA, aGA, aBA);
    pixel_addr(w, kB, lr, aRB, aGB, aBB);
    f2 H1, H2;
    solve_pair_od<PINV>(lut, aRA, aGA, aBA, aRB, aGB, aBB, P, NR1, NR2, kappa, H1, H2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // Eq. 3-4: i' = i0_t 2^(-log2e sum_j W_t[c,j] s_j h_j)
      const f2 E = fma2(K.M1[c], H1, fma2(K.M2[c], H2, K.L2[c]));
      // round half to even: adding 1.5*2^23 leaves round(x) in the low bits
      float xa = ex2_approx(lo_of(E)), xb = ex2_approx(hi_of(E));
      if (PINV) {
        xa = fminf(xa, 255.f);
        xb = fminf(xb, 255.f);
      }
      const f2 X = add2(pk(xa, xb), pk(12582912.0f, 12582912.0f));
      y[3 * kA + c] = __float_as_uint(lo_of(X));
      y[3 * kB + c] = __float_as_uint(hi_of(X));
    }
    // pack every output word whose four bytes are now known
#pragma unroll
    for (int i = 0; i < 12; ++i)
      if (4 * i + 3 <= 6 * p + 5 && 4 * i + 3 > 6 * p - 1)
        o[i] = pack4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
  }
}

// Pass-2 exponent coefficients of one image: M[3j+c] = -log2(e) W_t[c,j] s_j
// 2^hexp (Eq. 3-4 with the table's power-of-two scale folded in).  Computed in
// FP64 and rounded once, identically by every kernel that reconstructs.
__device__ __forceinline__ float recon_coef(const float* Wt, const double* scale, float hscale,
                                            int i) {
  const int c = i % 3, j = i / 3;
  return (float)(-(double)Wt[3 * j + c] * scale[j] * (double)hscale * 1.4426950408889634);
}

// P99 window of both stains and the constants of its exact tests:
// sat(h~ nk + lk) = [h~ < lo] and sat(h~ nh + hk) = [h~ < lo + nb].
struct Window {
  unsigned lo0, lo1, nb0, nb1;   // window start keys and widths (nb = 0: no window)
  float nk0, lk0, nk1, lk1;
  float nh0, hk0, nh1, hk1;
};

__host__ __device__ inline unsigned key_of(float f) {
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
}

// Constants of the exact test sat(h~ * nk + lk) = [h~ < key]: with key in
// [2^e, 2^(e+1)), any h~ < key is at least 2^(e-23) below it, so nk =
// -2^(24-e) makes the difference >= 1 before saturation.  Host and device
// (the same arithmetic on both).
__host__ __device__ inline void below_consts(unsigned key, float* nk, float* lk) {
  float f;
  memcpy(&f, &key, 4);
  int ex = 0;
  frexpf(f, &ex);                  // f in [2^(ex-1), 2^ex)
  const int K = 24 - (ex - 1);
  *nk = -ldexpf(1.f, K);
  *lk = ldexpf(f, K);
}

// Window [lo, lo+nb) of FP32 keys around a percentile hint h > 0 (in the
// units of the scaled densities): +-kWindowDelta relative, at most kWinBins
// keys; no window for a non-positive, non-finite or tiny hint.
__host__ __device__ inline void window_of(double hint, unsigned* lo, unsigned* nb, float* nk,
                                          float* lk, float* nh, float* hk) {
  *nk = -1.f;
  *lk = 0.f;
  *nh = -1.f;
  *hk = 0.f;
  if (!(hint > 0.0) || !(hint <= 1.7976931348623157e308) ||
      hint * (1.0 - kWindowDelta) < 0x1p-100) {
    *lo = 0u; *nb = 0u; return;
  }
  unsigned klo = key_of((float)(hint * (1.0 - kWindowDelta)));
  unsigned khi = key_of((float)(hint * (1.0 + kWindowDelta)));
  const unsigned kmid = key_of((float)hint);
  if (klo == 0u) klo = 1u;   // key 0 (h = 0) is counted below the window
  if (khi < klo) khi = klo;
  u64 width = (u64)khi - klo + 1;
  if (width > (u64)kWinBins) {
    klo = kmid > (unsigned)(kWinBins / 2) ? kmid - (unsigned)(kWinBins / 2) : 1u;
    width = kWinBins;
  }
  *lo = klo;
  *nb = (unsigned)width;
  below_consts(klo, nk, lk);
  below_consts(klo + (unsigned)width, nh, hk);
}

// Window [lo, lo+nb) of FP32 keys covering a band [blo, bhi] of scaled
// densities (the sample's order statistics around the percentile, see
// k_select_list), at most kWinBins keys: a wider band is narrowed to kWinBins
// keys centred on `mid`.  A band that does not start above 0 falls back to
// window_of(mid).
__host__ __device__ inline void window_band(double blo, double bhi, double mid, unsigned* lo,
                                            unsigned* nb, float* nk, float* lk, float* nh,
                                            float* hk) {
  if (!(blo > 0.0) || !(bhi >= blo) || !(bhi <= 1.7976931348623157e308) || blo < 0x1p-100) {
    window_of(mid, lo, nb, nk, lk, nh, hk);
    return;
  }
  unsigned klo = key_of((float)blo), khi = key_of((float)bhi);
  if (klo == 0u) klo = 1u;   // key 0 (h = 0) is counted below the window
  if (khi < klo) khi = klo;
  u64 width = (u64)khi - klo + 1;
  if (width > (u64)kWinBins) {
    const unsigned kmid = key_of((float)mid);
    klo = kmid > (unsigned)(kWinBins / 2) ? kmid - (unsigned)(kWinBins / 2) : 1u;
    width = kWinBins;
  }
  *lo = klo;
  *nb = (unsigned)width;
  below_consts(klo, nk, lk);
  below_consts(klo + (unsigned)width, nh, hk);
}

__host__ __device__ inline Window window_for(double hint0, double hint1) {
  Window w;
  window_of(hint0, &w.lo0, &w.nb0, &w.nk0, &w.lk0, &w.nh0, &w.hk0);
  window_of(hint1, &w.lo1, &w.nb1, &w.nk1, &w.lk1, &w.nh1, &w.hk1);
  return w;
}

// Host launchers that take a window (spcn_pixel.cu).
int launch_window_from_basis(Context* c, const Model* m, const Model* sample_model,
                             const SelectState* sample_sel, const int* basis_status, Window* w,
                             cudaStream_t st);
// Constants (wm, we) of the conservative all-white test of a full chunk of
// pass 1: the AND of its twelve words, masked by wm, equals we.
void white_test_consts(int white_thresh, unsigned* wm, unsigned* we);
// The Eq. 3 factors from a given source percentile (SPCN_FLAG_P99_SAMPLED):
// host values, or the basis estimation's sample percentile on the device.
int launch_scale_given(Context* c, const double* p99, const double* tgt, cudaStream_t st);
int launch_check_basis(Context* c, const Model* m, const int* basis_status, cudaStream_t st);
int launch_scale_from_basis(Context* c, const Model* m, const SelectState* sample_sel,
                            const int* basis_status, const double* tgt, cudaStream_t st);
int launch_percentile_passes_dev(Context* c, const Geometry& g, const Model* m, int white_thresh,
                                 double pct, const Window* wdev, const double* tgt_p99,
                                 cudaStream_t st, bool pinv = false);

}  // namespace spcn
