// Per-pixel passes of the improved SPCN (Eq. 1-4) on sm_103a.
//
// All passes stream the 8-bit RGB image in 16-pixel chunks (48 bytes = three
// 16-byte loads per thread) from a persistent grid sized to the SM count, look
// the optical densities up in a replicated shared-memory table (Eq. 1, already
// projected on the basis and shifted by lambda), and solve the Eq. 2 H-step in
// closed form (solve_pair / solve_one).  Nothing here is a dense contraction, so no
// tensor-core path is used: the passes are bound by HBM bandwidth and
// instruction issue.
#include <math.h>
#include <string.h>

#include <cmath>

#include "spcn_context.h"
#include "spcn_internal.cuh"

namespace spcn {

// ------------------------------------------------------------ Eq. 1 table
struct ModelIn {
  float W[6];
  float i0[3];
  float lambda;
  int hexp;          // power-of-two scale of the table; kHexpAuto: derive on the device
};

// Smallest e with 2^e >= 2 * (largest |d_j| any pixel can reach), so that
// every table sum s*d_j stays within [-1/2, 1/2].  |d_j| <= |v|/|w_j| +
// lambda/G_jj with |v_c| <= max(log i0_c, log(255/i0_c)).
__host__ __device__ inline int table_hexp(const float* W, const float* i0, float lambda) {
  double vv = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double a = log((double)i0[c]), b = log(255.0 / (double)i0[c]);
    const double m = a > b ? a : b;
    vv += m * m;
  }
  const double vn = sqrt(vv);
  double bound = 0.0;
  for (int j = 0; j < 2; ++j) {
    double g = 0.0;
    for (int c = 0; c < 3; ++c) g += (double)W[3 * j + c] * W[3 * j + c];
    if (g > 0.0) {
      const double bj = vn / sqrt(g) + (double)lambda / g;
      bound = bj > bound ? bj : bound;
    }
  }
  if (!(bound > 0.0)) bound = 1.0;
  int e = 0;
  frexp(bound, &e);       // bound < 2^e
  return e + 1;
}

// One thread per (channel, intensity): v = log(i0_c / max(i,1)) in FP64, the
// plain table and the scaled table of the closed-form H-step (rounded once to
// FP32, never -0).  Thread 0 derives the closed-form coefficients.
__global__ void k_build_model(Model* m, ModelIn in, const Model* from) {
  float W[6], i0[3];
  const Model* src = from;
  for (int i = 0; i < 6; ++i) W[i] = src ? src->W[i] : in.W[i];
  for (int i = 0; i < 3; ++i) i0[i] = src ? src->i0[i] : in.i0[i];
  double g11 = 0, g22 = 0, g12 = 0;
  for (int c = 0; c < 3; ++c) {
    g11 += (double)W[c] * W[c];
    g22 += (double)W[3 + c] * W[3 + c];
    g12 += (double)W[c] * W[3 + c];
  }
  const double det = g11 * g22 - g12 * g12;
  const bool ok = det > 1e-12 && g11 > 0.0 && g22 > 0.0;
  const int hexp = in.hexp == kHexpAuto ? table_hexp(W, i0, in.lambda) : in.hexp;
  const double s = ldexp(1.0, -hexp);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kLutEntries) {
    const int c = e >> 8, i = e & 255;
    const double v = log((double)i0[c] / (double)(i > 0 ? i : 1));
    const double lam = c == 0 ? (double)in.lambda : 0.0;
    float p0 = 0.f, p1 = 0.f;
    if (ok) {
      p0 = (float)(s * ((double)W[c] * v - lam) / g11);
      p1 = (float)(s * ((double)W[3 + c] * v - lam) / g22);
    }
    m->od[e] = (float)v;
    m->proj[e] = make_float2(p0 + 0.f, p1 + 0.f);   // + 0 turns -0 into +0
  }
  if (e == 0) {
    Lasso L;
    L.hexp = hexp;
    L.hscale = (float)ldexp(1.0, hexp);
    L.pad = 0;
    if (ok) {
      L.nrho1 = (float)(-g12 / g11);
      L.nrho2 = (float)(-g12 / g22);
      L.kappa = (float)(g11 * g22 / det);
      m->status = SPCN_OK;
    } else {
      L.nrho1 = L.nrho2 = L.kappa = 0.f;
      m->status = SPCN_ERR_DEGENERATE_BASIS;
    }
    m->lasso = L;
    if (from != m) {
      for (int i = 0; i < 6; ++i) m->W[i] = W[i];
      for (int i = 0; i < 3; ++i) m->i0[i] = i0[i];
    }
  }
}

int host_table_hexp(const float* W, const float* i0, float lambda) {
  return table_hexp(W, i0, lambda);
}

int launch_build_model(Context* c, Model* m, const float* W, const float* i0, float lambda,
                       const Model* from_device, cudaStream_t st) {
  ModelIn in;
  for (int i = 0; i < 6; ++i) in.W[i] = W ? W[i] : 0.f;
  for (int i = 0; i < 3; ++i) in.i0[i] = i0 ? i0[i] : 1.f;
  in.lambda = lambda;
  in.hexp = (W && i0 && !from_device) ? table_hexp(W, i0, lambda) : kHexpAuto;
  k_build_model<<<kLutEntries / 32, 32, 0, st>>>(m, in, from_device);   // one log per thread
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

// ------------------------------------------------------------ traversal
struct ChunkPos {
  u64 px;           // raster index of the chunk's first pixel
  int64_t src_off;  // byte offset in the source
  int64_t dst_off;  // byte offset in the destination
  int n;            // valid pixels (16 except at row ends)
};

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

__device__ __forceinline__ unsigned byte_at(const unsigned (&w)[12], int i) {
  return (w[i >> 2] >> ((i & 3) * 8)) & 0xFFu;
}

// Load a chunk into 12 little-endian words; STREAM selects the evict-first
// policy for data read for the last time.  Pixels past the end of a row read
// as white (0xFF bytes): they fall outside every count of pass 1, and their
// outputs are never stored, so every chunk takes the same unrolled path.
template <bool STREAM>
__device__ __forceinline__ void load_chunk(const Geometry& g, const ChunkPos& p,
                                           unsigned (&w)[12]) {
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

__device__ __forceinline__ void store_chunk(const Geometry& g, const ChunkPos& p,
                                            const unsigned (&o)[12]) {
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

// Persistent grid-stride loop over chunks; body(w, pos) is called for every
// chunk.  With PREFETCH the next chunk's loads are issued before the current
// chunk is processed (two register buffers, so no copies); the issue-bound
// pass 1 runs faster without it, the bandwidth-bound pass 2 with it.
template <bool STREAM, bool PREFETCH, class Body>
__device__ __forceinline__ void for_each_chunk(const Geometry& g, Body&& body) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 n = g.nchunks;
  u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x;
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

// ------------------------------------------------------------ pass 1
struct WindowArgs {
  Geometry g;
  const Model* m;
  SelectState* sel;
  u64* fine;
  u64* coarse;
  int* err;
  unsigned wthr;       // (white threshold + 1) << 8, compared with table offsets
  unsigned lo0, lo1;   // window start keys (scaled densities)
  unsigned nb0, nb1;   // window widths (0 = no window)
  float nk0, lk0;      // below-window test: sat(h~ * nk + lk) = [h~ < lo]
  float nk1, lk1;
  float nh0, hk0;      // below-window-end test: sat(h~ * nh + hk) = [h~ < lo + nb]
  float nh1, hk1;
  double pct;
  double tgt0, tgt1;   // target percentiles (for the scale factors)
};

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
    solve_pair(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, kappa, H1, H2);
    const bool nwA = aRA < a.wthr || aGA < a.wthr || aBA < a.wthr;
    const bool nwB = aRB < a.wthr || aGB < a.wthr || aBB < a.wthr;
    const f2 NW = pk(nwA ? 1.f : 0.f, nwB ? 1.f : 0.f);
    c_nw = add2(c_nw, NW);
    const float h1A = lo_of(H1), h1B = hi_of(H1), h2A = lo_of(H2), h2B = hi_of(H2);
    const f2 B0 = pk(fma_sat(h1A, a.nk0, a.lk0), fma_sat(h1B, a.nk0, a.lk0));
    const f2 B1 = pk(fma_sat(h2A, a.nk1, a.lk1), fma_sat(h2B, a.nk1, a.lk1));
    const f2 T0 = pk(fma_sat(h1A, a.nh0, a.hk0), fma_sat(h1B, a.nh0, a.hk0));
    const f2 T1 = pk(fma_sat(h2A, a.nh1, a.hk1), fma_sat(h2B, a.nh1, a.hk1));
    c_b0 = fma2(B0, NW, c_b0);
    c_b1 = fma2(B1, NW, c_b1);
    // T - B is 1 exactly for an in-window density
    const f2 X = add2(fma2(B0, M1, T0), fma2(B1, M1, T1));
    mask = fma2(mask, FOUR, mul2(X, NW));
  }
}

// Rank selection inside the window, run by the last block of pass 1.
__device__ void window_select(const WindowArgs& a) {
  SelectState* s = a.sel;
  __shared__ u64 s_tmp[33];
  __shared__ int s_idx, s_idx2;
  __shared__ u64 s_before, s_before2;
  __shared__ int s_res[kTracks];
  const u64 n = __ldcg(&s->n_nw);
  if (n == 0) {
    if (threadIdx.x == 0) {
      record_error(a.err, SPCN_ERR_NO_TISSUE);
      for (int t = 0; t < kTracks; ++t) { s->key[t] = 0; s->resolved[t] = 1; }
      s->p99[0] = s->p99[1] = 0.0;
      s->scale[0] = s->scale[1] = 1.0;
      s->t = 0.0;
      s->all_resolved = 1;
    }
    return;
  }
  if (threadIdx.x == 0) {
    set_ranks(s, n, a.pct);
    s->lo[0] = a.lo0; s->lo[1] = a.lo1; s->nb[0] = a.nb0; s->nb[1] = a.nb1;
  }
  __syncthreads();
  for (int t = 0; t < kTracks; ++t) {
    const int j = t >> 1;
    const unsigned nb = j ? a.nb1 : a.nb0;
    const unsigned lo = j ? a.lo1 : a.lo0;
    const u64 r = s->rank[t];
    const u64 below = __ldcg(&s->below[j]);
    if (threadIdx.x == 0) s_res[t] = 0;
    __syncthreads();
    if (nb == 0 || r < below) continue;
    const int ngroups = (int)((nb + kWinGroup - 1) >> kWinGroupBits);
    block_find_rank(a.coarse + j * kWinGroups, ngroups, r - below, &s_idx, &s_before, s_tmp);
    if (s_idx < 0) continue;
    const int gidx = s_idx;
    const u64 r2 = r - below - s_before;
    const unsigned gbeg = (unsigned)gidx << kWinGroupBits;
    const int nbins = (int)min((unsigned)kWinGroup, nb - gbeg);
    block_find_rank(a.fine + (size_t)j * kWinBins + gbeg, nbins, r2, &s_idx2, &s_before2, s_tmp);
    if (s_idx2 < 0) continue;   // cannot happen: the group count covers r2
    if (threadIdx.x == 0) {
      s->key[t] = lo + gbeg + (unsigned)s_idx2;
      s_res[t] = 1;
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int t = 0; t < kTracks; ++t) { s->resolved[t] = s_res[t]; all &= s_res[t]; }
    if (all) finish_percentiles(s, a.tgt0, a.tgt1, a.m->lasso.hscale);
    __threadfence();
    s->all_resolved = all;
  }
}

constexpr int kWarpQueue = 64;    // queued chunks per warp; drained once 32 are waiting, so the
                                  // re-read chunks are recent enough to still be in L2

// Window-histogram updates of the queued chunks: each entry is a chunk index
// and its two base-4 masks; only flagged pixels are recomputed (same
// arithmetic, same keys), reading their bytes again (still in L2).  Called by
// one warp for its own queue.
__device__ __forceinline__ void drain_queue(const uint2* queue, int count, const Geometry& g,
                                            const char* lut, unsigned lr, const Lasso& L,
                                            const WindowConst& a, unsigned* s_coarse) {
  for (int e = (int)(threadIdx.x & 31u); e < count; e += 32) {
    const uint2 ent = queue[e];
    const ChunkPos p = chunk_pos(g, (u64)ent.x);
    const uint8_t* src = g.src + p.src_off;
#pragma unroll 1
    for (int lane = 0; lane < 2; ++lane) {
      unsigned m = lane ? (ent.y >> 16) : (ent.y & 0xFFFFu);
#pragma unroll 1
      while (m) {
        const int bit = __ffs(m) - 1;
        const int pair = 7 - (bit >> 1);
        m &= ~(3u << (bit & ~1));
        const int k = 2 * pair + lane;
        const unsigned r = __ldg(src + 3 * k), gg = __ldg(src + 3 * k + 1), b = __ldg(src + 3 * k + 2);
        float h1, h2;
        solve_one(lut, (r << 8) | lr, (gg << 8) | lr, (b << 8) | lr, L, h1, h2);
        window_hit(a, s_coarse, __float_as_uint(h1) - a.lo0, __float_as_uint(h2) - a.lo1);
      }
    }
  }
}

__global__ void __launch_bounds__(kPassThreads, 1) k_pass_window(WindowArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_coarse = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);
  uint2* s_queue = reinterpret_cast<uint2*>(s_dyn + kLutSmemBytes + 2 * kWinGroups * sizeof(unsigned)) +
                   (threadIdx.x >> 5) * kWarpQueue;      // this warp's queue
  __shared__ u64 s_tmp[33];
  __shared__ unsigned s_ticket;
  for (int i = threadIdx.x; i < 2 * kWinGroups; i += blockDim.x) s_coarse[i] = 0u;
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  const Lasso L = a.m->lasso;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  f2 c_nw = pk(0.f, 0.f), c_b0 = pk(0.f, 0.f), c_b1 = pk(0.f, 0.f);
  const WindowConst C{a.fine, a.wthr, a.lo0, a.lo1, a.nb0, a.nb1, a.nk0, a.lk0, a.nk1, a.lk1,
                      a.nh0, a.hk0, a.nh1, a.hk1};
  const Geometry g = a.g;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  int qn = 0;   // entries in this warp's queue (warp-uniform)
  // every lane of a warp runs the same number of iterations (warp-uniform
  // loop), so the queue bookkeeping needs only warp-level operations
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < g.nchunks;
       base += stride) {
    const u64 q = base + lane;
    bool hit = false;
    unsigned packed = 0u;
    if (q < g.nchunks) {
      const ChunkPos p = chunk_pos(g, q);
      unsigned w[12];
      load_chunk<false>(g, p, w);
      f2 mask;
      window_chunk(w, lut, lr, NR1, NR2, L.kappa, C, c_nw, c_b0, c_b1, mask);
      const unsigned mA = (unsigned)lo_of(mask), mB = (unsigned)hi_of(mask);
      packed = mA | (mB << 16);
      hit = packed != 0u;
    }
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, hit);
    if (hit) s_queue[qn + __popc(ball & ((1u << lane) - 1u))] = make_uint2((unsigned)q, packed);
    qn += __popc(ball);
    if (qn >= 32 || base + stride >= g.nchunks) {
      __syncwarp();
      drain_queue(s_queue, qn, g, lut, lr, L, C, s_coarse);
      __syncwarp();
      qn = 0;
    }
  }
  // per-thread counts are exact in FP32 (fewer than 2^24 pixels per thread)
  const u64 t_nw = block_sum((u64)lo_of(c_nw) + (u64)hi_of(c_nw), s_tmp);
  const u64 t_b0 = block_sum((u64)lo_of(c_b0) + (u64)hi_of(c_b0), s_tmp);
  const u64 t_b1 = block_sum((u64)lo_of(c_b1) + (u64)hi_of(c_b1), s_tmp);
  if (threadIdx.x == 0) {
    if (t_nw) atomicAdd(&a.sel->n_nw, t_nw);
    if (t_b0) atomicAdd(&a.sel->below[0], t_b0);
    if (t_b1) atomicAdd(&a.sel->below[1], t_b1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kWinGroups; i += blockDim.x)
    if (s_coarse[i]) atomicAdd(a.coarse + i, (u64)s_coarse[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&a.sel->done_ctas, 1u);
  __syncthreads();
  if (s_ticket == gridDim.x - 1) {
    __threadfence();
    window_select(a);
  }
}

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
  const uint32_t* items;   // packed R | G<<8 | B<<16, all non-white
  u64 n;
  template <class F>
  __device__ __forceinline__ void for_each(F&& f) const {
    const unsigned lr = lane_reg();
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
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
template <class Src>
__device__ bool radix_select(const Src& src, const char* lut, const Lasso& L, SelectState* s,
                             const u64 (&rank)[kTracks], const int (&active)[kTracks],
                             u64* ghist, unsigned* s_hist, unsigned* bar, int* err,
                             long long timeout_ns, double tgt0, double tgt1) {
  __shared__ unsigned s_prefix[kTracks];
  __shared__ u64 s_r[kTracks];
  __shared__ int s_act[kTracks];
  __shared__ int s_idx;
  __shared__ u64 s_before;
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
      solve_one(lut, aR, aG, aB, L, h1, h2);
      const unsigned key[2] = {__float_as_uint(h1), __float_as_uint(h2)};
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
    for (int t = 0; t < kTracks; ++t) {
      if (!s_act[t]) continue;
      block_find_rank(gh + (size_t)own[t] * kRadixBins, kRadixBins, s_r[t], &s_idx, &s_before, s_tmp);
      if (threadIdx.x == 0) {
        if (s_idx < 0) {         // fewer pixels than the rank: cannot happen
          record_error(err, SPCN_ERR_CUDA);
          s_act[t] = 0;
        } else {
          s_prefix[t] |= (unsigned)s_idx << shift;
          s_r[t] -= s_before;
        }
      }
      __syncthreads();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int t = 0; t < kTracks; ++t)
      if (s_act[t]) { s->key[t] = s_prefix[t]; s->resolved[t] = 1; }
    finish_percentiles(s, tgt0, tgt1, L.hscale);
    __threadfence();
    s->all_resolved = 1;
  }
  return true;
}

struct SelectImageArgs {
  ImageSource src;
  const Model* m;
  SelectState* sel;
  u64* ghist;
  int* err;
  long long timeout_ns;
  double tgt0, tgt1;
};

__global__ void __launch_bounds__(kPassThreads, 1) k_select_image(SelectImageArgs a) {
  if (*(volatile int*)&a.sel->all_resolved) return;   // uniform: every block returns
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_hist = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);
  load_lut(a.m, s_dyn);
  const Lasso L = a.m->lasso;
  u64 rank[kTracks];
  int active[kTracks];
  for (int t = 0; t < kTracks; ++t) {
    rank[t] = __ldcg(&a.sel->rank[t]);
    active[t] = !__ldcg(&a.sel->resolved[t]);
  }
  radix_select(a.src, s_dyn, L, a.sel, rank, active, a.ghist, s_hist, &a.sel->barrier, a.err,
               a.timeout_ns, a.tgt0, a.tgt1);
}

struct SelectListArgs {
  const uint32_t* items;
  const u64* n_dev;
  const Model* m;
  SelectState* sel;
  u64* ghist;
  int* err;
  long long timeout_ns;
  double pct;
};

// Percentile of the densities of a packed list of non-white pixels (the basis
// sample, §3.1 item 2), radix select from scratch.
__global__ void __launch_bounds__(kPassThreads, 1) k_select_list(SelectListArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_hist = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);
  const u64 n = __ldcg(a.n_dev);
  if (n == 0 || a.m->status != SPCN_OK) return;   // uniform: every block returns
  u64 rank[kTracks];
  int active[kTracks];
  double t;
  type7_ranks(n, a.pct, &rank[0], &rank[1], &t);
  rank[2] = rank[0];
  rank[3] = rank[1];
  for (int i = 0; i < kTracks; ++i) active[i] = 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.sel->n_nw = n;
    a.sel->t = t;
    for (int i = 0; i < kTracks; ++i) a.sel->rank[i] = rank[i];
  }
  load_lut(a.m, s_dyn);
  const Lasso L = a.m->lasso;
  ListSource src{a.items, n};
  radix_select(src, s_dyn, L, a.sel, rank, active, a.ghist, s_hist, &a.sel->barrier, a.err,
               a.timeout_ns, 1.0, 1.0);
}

// ------------------------------------------------------------ pass 2
struct ReconArgs {
  Geometry g;
  const Model* m;
  const SelectState* sel;
  float Wt[6];       // target basis
  float l2i0[3];     // log2 of the target i0
};

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

__device__ __forceinline__ void recon_chunk(const unsigned (&w)[12], const char* lut,
                                            unsigned lr, f2 NR1, f2 NR2, float kappa,
                                            const ReconConst& K, unsigned (&o)[12]) {
  unsigned y[48];
#pragma unroll
  for (int p = 0; p < kChunk / 2; ++p) {
    const int kA = 2 * p, kB = 2 * p + 1;
    unsigned aRA, aGA, aBA, aRB, aGB, aBB;
    pixel_addr(w, kA, lr, aRA, aGA, aBA);
    pixel_addr(w, kB, lr, aRB, aGB, aBB);
    f2 H1, H2;
    solve_pair(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, kappa, H1, H2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // Eq. 3-4: i' = i0_t 2^(-log2e sum_j W_t[c,j] s_j h_j)
      const f2 E = fma2(K.M1[c], H1, fma2(K.M2[c], H2, K.L2[c]));
      // round half to even: adding 1.5*2^23 leaves round(x) in the low bits
      const f2 X = add2(pk(ex2_approx(lo_of(E)), ex2_approx(hi_of(E))), pk(12582912.0f, 12582912.0f));
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

__global__ void __launch_bounds__(kPassThreads, 1) k_pass_recon(ReconArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ float s_M[6];
  const Lasso L = a.m->lasso;
  if (threadIdx.x < 6) {
    const int c = threadIdx.x % 3, j = threadIdx.x / 3;
    const double sc = a.sel->scale[j];
    s_M[threadIdx.x] = (float)(-(double)a.Wt[3 * j + c] * sc * (double)L.hscale * 1.4426950408889634);
  }
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  ReconConst K;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    K.M1[c] = pk(s_M[c], s_M[c]);
    K.M2[c] = pk(s_M[3 + c], s_M[3 + c]);
    K.L2[c] = pk(a.l2i0[c], a.l2i0[c]);
  }
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  for_each_chunk<true, true>(a.g, [&](const unsigned (&w)[12], const ChunkPos& p) {
    unsigned o[12];
    recon_chunk(w, lut, lr, NR1, NR2, L.kappa, K, o);
    store_chunk(a.g, p, o);
  });
}

// ------------------------------------------------------------ densities
struct DensityArgs {
  Geometry g;
  const Model* m;
  float* H;
  int64_t stride;   // elements between the two planes
};

__global__ void __launch_bounds__(kPassThreads, 1) k_pass_density(DensityArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  const Lasso L = a.m->lasso;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  const f2 HS = pk(L.hscale, L.hscale);
  const bool vec_h = ((reinterpret_cast<uintptr_t>(a.H) & 15u) == 0) && ((a.stride & 3) == 0);
  for_each_chunk<true, true>(a.g, [&](const unsigned (&w)[12], const ChunkPos& p) {
    float* d0 = a.H + p.px;
    float* d1 = a.H + a.stride + p.px;
    const bool vec = p.n == kChunk && vec_h && (p.px & 3) == 0;
#pragma unroll
    for (int v = 0; v < kChunk / 4; ++v) {
      f2 H1[2], H2[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = 4 * v + 2 * q;
        unsigned aRA, aGA, aBA, aRB, aGB, aBB;
        pixel_addr(w, k, lr, aRA, aGA, aBA);
        pixel_addr(w, k + 1, lr, aRB, aGB, aBB);
        solve_pair(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, L.kappa, H1[q], H2[q]);
        H1[q] = mul2(H1[q], HS);     // exact: the scale is a power of two
        H2[q] = mul2(H2[q], HS);
      }
      const float4 h1 = make_float4(lo_of(H1[0]), hi_of(H1[0]), lo_of(H1[1]), hi_of(H1[1]));
      const float4 h2 = make_float4(lo_of(H2[0]), hi_of(H2[0]), lo_of(H2[1]), hi_of(H2[1]));
      if (vec) {
        __stcs(reinterpret_cast<float4*>(d0) + v, h1);
        __stcs(reinterpret_cast<float4*>(d1) + v, h2);
      } else {
        const float a1[4] = {h1.x, h1.y, h1.z, h1.w}, a2[4] = {h2.x, h2.y, h2.z, h2.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * v + k < p.n) { d0[4 * v + k] = a1[k]; d1[4 * v + k] = a2[k]; }
      }
    }
  });
}

// ------------------------------------------------------------ failure-detection hook
__global__ void k_debug_barrier(SelectState* s, int* err, int extra, long long timeout_ns) {
  grid_barrier(&s->barrier, gridDim.x + (unsigned)extra, &s->abort, err, timeout_ns);
}

// ------------------------------------------------------------ host launchers
static int grid_of(const Context* c, int occ) {
  return c->num_sms * (occ > 0 ? occ : 1);
}

int configure_pixel_kernels(Context* c) {
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_pass_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kWindowSmem));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_pass_recon, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLutSmemBytes));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_pass_density, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLutSmemBytes));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_select_image, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRadixSmem));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_select_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRadixSmem));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_window, k_pass_window,
                                                              kPassThreads, kWindowSmem));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_recon, k_pass_recon,
                                                              kPassThreads, kLutSmemBytes));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_density, k_pass_density,
                                                              kPassThreads, kLutSmemBytes));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_select, k_select_image,
                                                              kPassThreads, kRadixSmem));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_radix_list, k_select_list,
                                                              kPassThreads, kRadixSmem));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_debug, k_debug_barrier,
                                                              128, 0));
  if (c->occ_window < 1 || c->occ_recon < 1 || c->occ_density < 1 || c->occ_select < 1 ||
      c->occ_radix_list < 1 || c->occ_debug < 1)
    return SPCN_ERR_CUDA;
  return SPCN_OK;
}

// Window [lo, lo+nb) of FP32 keys around a percentile hint h > 0 (in the
// units of the scaled densities), and the constants of the exact
// below-window test sat(h~ * nk + lk) = [h~ < lo]: with lo in [2^e, 2^e+1),
// any h~ < lo is at least 2^(e-24) below it, so nk = -2^(24-e) makes the
// difference >= 1 before saturation.
static void below_consts(unsigned key, float* nk, float* lk) {
  float f;
  memcpy(&f, &key, 4);
  int ex = 0;
  frexpf(f, &ex);                  // f in [2^(ex-1), 2^ex)
  const int K = 24 - (ex - 1);
  *nk = -ldexpf(1.f, K);
  *lk = ldexpf(f, K);
}

static void window_of(double hint, unsigned* lo, unsigned* nb, float* nk, float* lk, float* nh,
                      float* hk) {
  *nk = -1.f;
  *lk = 0.f;
  *nh = -1.f;
  *hk = 0.f;
  if (!(hint > 0.0) || !std::isfinite(hint) || hint * (1.0 - kWindowDelta) < 0x1p-100) {
    *lo = 0u; *nb = 0u; return;
  }
  float flo = (float)(hint * (1.0 - kWindowDelta));
  float fhi = (float)(hint * (1.0 + kWindowDelta));
  unsigned klo, khi, kmid;
  float fmid = (float)hint;
  memcpy(&klo, &flo, 4);
  memcpy(&khi, &fhi, 4);
  memcpy(&kmid, &fmid, 4);
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

// Pass 1 + select (+ radix fallback when a rank fell outside the window).
int launch_percentile_passes(Context* c, const Geometry& g, const Model* m, int white_thresh,
                             double pct, const double* hint, int hexp, const double* tgt_p99,
                             cudaStream_t st) {
  WindowArgs a;
  a.g = g;
  a.m = m;
  a.sel = c->sel;
  a.fine = c->fine;
  a.coarse = c->coarse;
  a.err = c->err;
  a.wthr = ((unsigned)white_thresh + 1u) << 8;
  const double hs = ldexp(1.0, -hexp);
  window_of(hint ? hint[0] * hs : 0.0, &a.lo0, &a.nb0, &a.nk0, &a.lk0, &a.nh0, &a.hk0);
  window_of(hint ? hint[1] * hs : 0.0, &a.lo1, &a.nb1, &a.nk1, &a.lk1, &a.nh1, &a.hk1);
  a.pct = pct;
  a.tgt0 = tgt_p99 ? tgt_p99[0] : 1.0;
  a.tgt1 = tgt_p99 ? tgt_p99[1] : 1.0;
  SPCN_CUDA_TRY(cudaMemsetAsync(c->sel, 0, sizeof(SelectState), st));
  SPCN_CUDA_TRY(cudaMemsetAsync(c->coarse, 0, sizeof(u64) * 2 * kWinGroups, st));
  if (a.nb0) SPCN_CUDA_TRY(cudaMemsetAsync(c->fine, 0, sizeof(u64) * a.nb0, st));
  if (a.nb1) SPCN_CUDA_TRY(cudaMemsetAsync(c->fine + kWinBins, 0, sizeof(u64) * a.nb1, st));
  {
    TimedLaunch tl(c, SPCN_KERNEL_PASS1, st);
    k_pass_window<<<grid_of(c, c->occ_window), kPassThreads, kWindowSmem, st>>>(a);
  }
  SPCN_LAUNCH_CHECK(c);

  SelectImageArgs s;
  s.src.g = g;
  s.src.thr = (unsigned)white_thresh;
  s.m = m;
  s.sel = c->sel;
  s.ghist = c->rhist;
  s.err = c->err;
  s.timeout_ns = c->timeout_ns;
  s.tgt0 = a.tgt0;
  s.tgt1 = a.tgt1;
  void* args[] = {&s};
  {
    TimedLaunch tl(c, SPCN_KERNEL_SELECT, st);
    SPCN_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_select_image, grid_of(c, c->occ_select),
                                              kPassThreads, args, kRadixSmem, st));
  }
  c->launches++;
  return SPCN_OK;
}

int launch_select_list(Context* c, const uint32_t* items, const u64* n_dev, const Model* m,
                       SelectState* sel, u64* ghist, double pct, cudaStream_t st) {
  SelectListArgs a;
  a.items = items;
  a.n_dev = n_dev;
  a.m = m;
  a.sel = sel;
  a.ghist = ghist;
  a.err = c->err;
  a.timeout_ns = c->timeout_ns;
  a.pct = pct;
  SPCN_CUDA_TRY(cudaMemsetAsync(sel, 0, sizeof(SelectState), st));
  void* args[] = {&a};
  SPCN_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_select_list, grid_of(c, c->occ_radix_list),
                                            kPassThreads, args, kRadixSmem, st));
  c->launches++;
  return SPCN_OK;
}

int launch_recon(Context* c, const Geometry& g, const Model* m, const float* Wt, const float* i0t,
                 cudaStream_t st) {
  ReconArgs a;
  a.g = g;
  a.m = m;
  a.sel = c->sel;
  for (int i = 0; i < 6; ++i) a.Wt[i] = Wt[i];
  for (int i = 0; i < 3; ++i) a.l2i0[i] = (float)log2((double)i0t[i]);
  {
    TimedLaunch tl(c, SPCN_KERNEL_PASS2, st);
    k_pass_recon<<<grid_of(c, c->occ_recon), kPassThreads, kLutSmemBytes, st>>>(a);
  }
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

int launch_density(Context* c, const Geometry& g, const Model* m, float* H, int64_t stride,
                   cudaStream_t st) {
  DensityArgs a;
  a.g = g;
  a.m = m;
  a.H = H;
  a.stride = stride;
  {
    TimedLaunch tl(c, SPCN_KERNEL_DENSITY, st);
    k_pass_density<<<grid_of(c, c->occ_density), kPassThreads, kLutSmemBytes, st>>>(a);
  }
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

int launch_debug_barrier(Context* c, int extra, long long timeout_ns, cudaStream_t st) {
  SelectState* sel = c->sel;
  SPCN_CUDA_TRY(cudaMemsetAsync(c->sel, 0, sizeof(SelectState), st));
  int* err = c->err;
  void* args[] = {&sel, &err, &extra, &timeout_ns};
  SPCN_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_debug_barrier, c->num_sms, 128, args, 0, st));
  c->launches++;
  return SPCN_OK;
}

}  // namespace spcn
