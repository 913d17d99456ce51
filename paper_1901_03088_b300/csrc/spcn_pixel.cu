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
#include "spcn_pixel.cuh"

namespace spcn {

// ------------------------------------------------------------ Eq. 1 table
struct ModelIn {
  float W[6];
  float i0[3];
  float lambda;
  int hexp;          // power-of-two scale of the table; kHexpAuto: derive on the device
  int pinv;          // pseudo-inverse rows instead of the lasso's projections
};

// Smallest e with 2^e >= 2 * (largest |d_j| any pixel can reach), so that
// every table sum s*d_j stays within [-1/2, 1/2].  |d_j| <= |v|/|w_j| +
// lambda/G_jj with |v_c| <= max(log i0_c, log(255/i0_c)).  la[c] = log i0_c,
// lb[c] = log(255/i0_c) (computed apart, so that the device can take the six
// logarithms in parallel).
__host__ __device__ inline int table_hexp_from_logs(const float* W, const double* la,
                                                    const double* lb, float lambda) {
  double vv = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double m = la[c] > lb[c] ? la[c] : lb[c];
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

__host__ __device__ inline int table_hexp(const float* W, const float* i0, float lambda) {
  double la[3], lb[3];
  for (int c = 0; c < 3; ++c) {
    la[c] = log((double)i0[c]);
    lb[c] = log(255.0 / (double)i0[c]);
  }
  return table_hexp_from_logs(W, la, lb, lambda);
}

constexpr int kModelThreads = 128;   // table entries per block of k_build_model

// One thread per (channel, intensity): v = log(i0_c / max(i,1)) in FP64, the
// plain table and the scaled table of the closed-form H-step (rounded once to
// FP32, never -0).  The per-image scalars that need FP64 logarithms or
// divisions are spread over the lanes of warp 0 (FP64 latency, not
// throughput, bounds this kernel): each block takes the six logarithms of
// the table's scale in parallel, and block 0 derives the closed-form
// coefficients one per lane.
__global__ void __launch_bounds__(kModelThreads) k_build_model(Model* m, ModelIn in,
                                                               const Model* from) {
  __shared__ double s_lg[6];
  __shared__ int s_hexp;
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
  int hexp = in.hexp;
  if (hexp == kHexpAuto) {   // uniform
    if (threadIdx.x < 6) {
      const int c = threadIdx.x % 3;
      s_lg[threadIdx.x] = threadIdx.x < 3 ? log((double)i0[c]) : log(255.0 / (double)i0[c]);
    }
    __syncthreads();
    if (threadIdx.x == 0) s_hexp = table_hexp_from_logs(W, s_lg, s_lg + 3, in.lambda);
    __syncthreads();
    hexp = s_hexp;
  }
  const double s = ldexp(1.0, -hexp);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kLutEntries) {
    const int c = e >> 8, i = e & 255;
    const double v = log((double)i0[c] / (double)(i > 0 ? i : 1));
    const double lam = c == 0 ? (double)in.lambda : 0.0;
    float p0 = 0.f, p1 = 0.f;
    if (ok && in.pinv) {   // s (pinv(W))[j,c] v, pinv(W) = G^-1 W^T (§2.1)
      p0 = (float)(s * (((double)W[c] * g22 - (double)W[3 + c] * g12) / det) * v);
      p1 = (float)(s * (((double)W[3 + c] * g11 - (double)W[c] * g12) / det) * v);
    } else if (ok) {
      p0 = (float)(s * ((double)W[c] * v - lam) / g11);
      p1 = (float)(s * ((double)W[3 + c] * v - lam) / g22);
    }
    m->od[e] = (float)v;
    m->proj[e] = make_float2(p0 + 0.f, p1 + 0.f);   // + 0 turns -0 into +0
  }
  if (blockIdx.x != 0) return;
  // block 0, warp 0: lanes 0-5 the pass-2 projections pa, lanes 6-7 the
  // offsets pb, lane 8 the lasso record and the status, lane 9 the basis copy
  const int l = threadIdx.x;
  if (l < 6) {
    const int j = l / 3, c = l % 3;
    const double gjj = j ? g22 : g11;
    const double pj = in.pinv ? (j ? ((double)W[3 + c] * g11 - (double)W[c] * g12) / det
                                   : ((double)W[c] * g22 - (double)W[3 + c] * g12) / det)
                              : (double)W[3 * j + c] / gjj;
    m->pa[3 * j + c] = ok ? (float)(s * pj) + 0.f : 0.f;
  } else if (l < 8) {
    const int j = l - 6;
    const double gjj = j ? g22 : g11;
    m->pb[j] = (ok && !in.pinv) ? (float)(-s * (double)in.lambda / gjj) + 0.f : 0.f;
  } else if (l == 8) {
    Lasso L;
    L.hexp = hexp;
    L.hscale = (float)ldexp(1.0, hexp);
    L.pinv = in.pinv;
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
  } else if (l == 9 && from != m) {
    for (int i = 0; i < 6; ++i) m->W[i] = W[i];
    for (int i = 0; i < 3; ++i) m->i0[i] = i0[i];
  }
}

int host_table_hexp(const float* W, const float* i0, float lambda) {
  return table_hexp(W, i0, lambda);
}

int launch_build_model(Context* c, Model* m, const float* W, const float* i0, float lambda,
                       const Model* from_device, cudaStream_t st, bool pinv) {
  ModelIn in;
  in.pinv = pinv ? 1 : 0;
  for (int i = 0; i < 6; ++i) in.W[i] = W ? W[i] : 0.f;
  for (int i = 0; i < 3; ++i) in.i0[i] = i0 ? i0[i] : 1.f;
  in.lambda = lambda;
  in.hexp = (W && i0 && !from_device) ? table_hexp(W, i0, lambda) : kHexpAuto;
  k_build_model<<<kLutEntries / kModelThreads, kModelThreads, 0, st>>>(m, in, from_device);
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
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
  unsigned wm, we;     // all-white test of a full chunk: (AND of its words & wm) == we
  Window w;            // P99 window (scaled densities), unless wdev is set
  const Window* wdev;  // window computed on the device (read at the kernel's start)
  double pct;
  double tgt0, tgt1;   // target percentiles (for the scale factors)
};


// Rank selection inside the window, run by the last block of pass 1.
template <bool DEV>
__device__ void window_select(const WindowArgs& a) {
  const unsigned lo0 = DEV ? a.wdev->lo0 : a.w.lo0, lo1 = DEV ? a.wdev->lo1 : a.w.lo1;
  const unsigned nb0 = DEV ? a.wdev->nb0 : a.w.nb0, nb1 = DEV ? a.wdev->nb1 : a.w.nb1;
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
    s->lo[0] = lo0; s->lo[1] = lo1; s->nb[0] = nb0; s->nb[1] = nb1;
  }
  __syncthreads();
  for (int t = 0; t < kTracks; ++t) {
    const int j = t >> 1;
    const unsigned nb = j ? nb1 : nb0;
    const unsigned lo = j ? lo1 : lo0;
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


// Window-histogram updates of queued pixels: each entry is a chunk index and
// one pixel of that chunk that the packed window test flagged; the pixel is
// recomputed (same arithmetic, same keys) from its bytes, read again (still
// in L2).  Lane e takes entry e < count (count <= 32): one step of the warp.
template <bool PINV>
__device__ __forceinline__ void drain_pixels(const uint2* queue, int count, const Geometry& g,
                                             const char* lut, unsigned lr, const Lasso& L,
                                             const WindowConst& a, unsigned* s_coarse) {
  const int e = (int)(threadIdx.x & 31u);
  if (e >= count) return;
  const uint2 ent = queue[e];
  const ChunkPos p = chunk_pos(g, (u64)ent.x);
  const int64_t off = p.src_off + 3 * (int64_t)ent.y;
  if (!SPCN_CHECK(ent.x < g.nchunks && ent.y < (unsigned)kChunk && off >= 0 &&
                  off + 3 <= g.src_bytes, g.err))
    return;   // queued pixels belong to full chunks of the image
  const uint8_t* src = g.src + off;
  const unsigned r = __ldg(src), gg = __ldg(src + 1), b = __ldg(src + 2);
  float h1, h2;
  solve_one<PINV>(lut, (r << 8) | lr, (gg << 8) | lr, (b << 8) | lr, L, h1, h2);
  window_hit(a, s_coarse, __float_as_uint(h1) - a.lo0, __float_as_uint(h2) - a.lo1);
}

// Window arithmetic of one full chunk per lane (lanes with have = false take
// no part), then the hit queue: called by the whole warp.  Every flagged
// pixel becomes one queue entry; each time 32 are waiting they are drained
// in one step of the warp (the queue holds fewer than 32 before a round of
// appends, which adds at most 32).
template <bool PINV, bool WHITES_BELOW>
__device__ __forceinline__ void pass1_chunk(const unsigned (&w)[12], unsigned qi, bool have,
                                            const char* lut, unsigned lr, f2 NR1, f2 NR2,
                                            const Lasso& L, const WindowConst& C,
                                            const Geometry& g, uint2* s_queue,
                                            unsigned* s_coarse, int& qn, f2& c_nw, f2& c_b0,
                                            f2& c_b1) {
  // bit 2 (7 - p) + h: pixel 2 p + h lies in a window of either stain
  unsigned d = 0u;
  if (have) {
    f2 mask;
    window_chunk<PINV, WHITES_BELOW>(w, lut, lr, NR1, NR2, L.kappa, C, c_nw, c_b0, c_b1, mask);
    const unsigned m0 = (unsigned)lo_of(mask), m1 = (unsigned)hi_of(mask);
    d = ((m0 | (m0 >> 1)) & 0x5555u) | (((m1 | (m1 >> 1)) & 0x5555u) << 1);
  }
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  unsigned ball;
  while ((ball = __ballot_sync(0xFFFFFFFFu, d != 0u)) != 0u) {
    if (d) {
      const unsigned bit = (unsigned)__ffs(d) - 1u;
      d &= d - 1u;
      s_queue[qn + __popc(ball & lt)] = make_uint2(qi, 2u * (7u - (bit >> 1)) + (bit & 1u));
    }
    qn += __popc(ball);
    if (qn >= 32) {
      __syncwarp();
      drain_pixels<PINV>(s_queue, 32, g, lut, lr, L, C, s_coarse);
      // the rest (fewer than 32) moves to the front
      const bool mv = lane + 32u < (unsigned)qn;
      uint2 rest = make_uint2(0u, 0u);
      if (mv) rest = s_queue[lane + 32u];
      __syncwarp();
      if (mv) s_queue[lane] = rest;
      __syncwarp();
      qn -= 32;
    }
  }
}

// A row's last chunk when it holds fewer than 16 pixels: pixel by pixel with
// the same keys as the vector path, counting only the pixels that exist (the
// padding bytes are not pixels, whatever the white threshold).  The bytes are
// read again (L1 hits) so that no register array is indexed at run time.
template <bool PINV>
__device__ __forceinline__ void partial_chunk(const uint8_t* src, int n, const char* lut,
                                              unsigned lr, const Lasso& L, const WindowConst& C,
                                              unsigned* s_coarse, f2& c_nw, f2& c_b0, f2& c_b1) {
  float nw = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const unsigned aR = ((unsigned)__ldg(src + 3 * k) << 8) | lr;
    const unsigned aG = ((unsigned)__ldg(src + 3 * k + 1) << 8) | lr;
    const unsigned aB = ((unsigned)__ldg(src + 3 * k + 2) << 8) | lr;
    if (min(min(aR, aG), aB) >= C.wthr) continue;   // white
    float h1, h2;
    solve_one<PINV>(lut, aR, aG, aB, L, h1, h2);
    nw += 1.f;
    b0 += fma_sat(h1, C.nk0, C.lk0);   // [h~ < lo], the vector path's test
    b1 += fma_sat(h2, C.nk1, C.lk1);
    window_hit(C, s_coarse, __float_as_uint(h1) - C.lo0, __float_as_uint(h2) - C.lo1);
  }
  c_nw = add2(c_nw, pk(nw, 0.f));
  c_b0 = add2(c_b0, pk(b0, 0.f));
  c_b1 = add2(c_b1, pk(b1, 0.f));
}

// DEV: the window is read from device memory (computed there); otherwise it
// is a kernel parameter, which the pixel loop uses without holding it in
// registers.
//
// Each warp loads 32 chunks at a time; all-white chunks are dropped and the
// others wait on a per-warp stack (at most 31 deep, in shared memory) until
// a full warp of them is ready: lanes holding a tissue chunk take their own,
// the others pop one from the stack, so the window arithmetic runs on full
// warps of tissue.
template <bool DEV, bool PINV>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass_window(WindowArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_coarse = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);
  char* s_after = s_dyn + kLutSmemBytes + 2 * kWinGroups * sizeof(unsigned);
  uint2* s_queue = reinterpret_cast<uint2*>(s_after) + (threadIdx.x >> 5) * kWarpQueue;  // this warp's queue
  s_after += sizeof(uint2) * kWarpQueue * (kPassThreads / 32);
  uint4* s_stk = reinterpret_cast<uint4*>(s_after) + (threadIdx.x >> 5) * (3 * kChunkStack);
  s_after += sizeof(uint4) * 3 * kChunkStack * (kPassThreads / 32);
  unsigned* s_stq = reinterpret_cast<unsigned*>(s_after) + (threadIdx.x >> 5) * kChunkStack;
  __shared__ u64 s_tmp[33];
  __shared__ unsigned s_ticket;
  for (int i = threadIdx.x; i < 2 * kWinGroups; i += blockDim.x) s_coarse[i] = 0u;
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  const Lasso L = a.m->lasso;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  f2 c_nw = pk(0.f, 0.f), c_b0 = pk(0.f, 0.f), c_b1 = pk(0.f, 0.f);
  // field by field, straight from the parameter (no reference to it, which
  // would make the compiler copy the parameters to local memory)
#define SPCN_WF(f) (DEV ? a.wdev->f : a.w.f)
  const WindowConst C{a.fine,       a.wthr,       SPCN_WF(lo0), SPCN_WF(lo1), SPCN_WF(nb0),
                      SPCN_WF(nb1), SPCN_WF(nk0), SPCN_WF(lk0), SPCN_WF(nk1), SPCN_WF(lk1),
                      SPCN_WF(nh0), SPCN_WF(hk0), SPCN_WF(nh1), SPCN_WF(hk1)};
#undef SPCN_WF
  const Geometry g = a.g;
  if (!SPCN_CHECK(C.nb0 <= (unsigned)kWinBins && C.nb1 <= (unsigned)kWinBins, g.err)) return;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned wm = a.wm, we = a.we;
  const WhiteBytes wb = white_bytes((a.wthr >> 8) - 1u);
  // every white pixel below both window starts: the lasso of a tissue chunk
  // then skips the per-pixel non-white masks (the same on every thread)
  const bool wbelow = !PINV && whites_below((a.wthr >> 8) - 1u, lut, lr, C);
  int qn = 0;   // entries in this warp's hit queue (warp-uniform)
  int ns = 0;   // tissue chunks on this warp's stack (warp-uniform)
  // Counts of a full, not all-white chunk; true when it needs the window
  // arithmetic (not provably below both window starts).
  auto classify = [&](const unsigned (&w)[12]) -> bool {
    // the non-white count and the per-channel minima of the density bound
    // from the same regrouped words
    unsigned rg, bb;
    const float nw = chunk_nonwhite_min(w, wb, &rg, &bb);
    const bool below = !PINV && below_bound(rg, bb, lut, lr, C);   // counts only, no lasso
    if (below || wbelow) {
      // with wbelow a tissue chunk's lasso counts all 16 pixels below both
      // windows (its white ones included), so its white pixels are taken
      // off here
      const f2 nb = pk(below ? nw : nw - (float)kChunk, 0.f);
      c_nw = add2(c_nw, pk(nw, 0.f));
      c_b0 = add2(c_b0, nb);
      c_b1 = add2(c_b1, nb);
    }
    return !below;
  };
  // The warp's step after each lane classified its chunk: tissue chunks wait
  // on the stack until a full warp of them is ready, which then runs the
  // window arithmetic.
  auto warp_step = [&](bool tissue, unsigned (&w)[12], unsigned qi) {
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, tissue);
    const int cnt = __popc(ball);
    __syncwarp();   // the stack's previous reads and writes are done
    if (ns + cnt < 32) {   // not a full warp yet: stack them
      if (tissue) stack_put(s_stk, s_stq, ns + __popc(ball & lt), w, qi);
      ns += cnt;
      return;
    }
    if (!tissue) stack_get(s_stk, s_stq, ns - 1 - __popc(~ball & lt), w, qi);
    ns -= 32 - cnt;
    if (wbelow)
      pass1_chunk<PINV, true>(w, qi, true, lut, lr, NR1, NR2, L, C, g, s_queue, s_coarse, qn, c_nw, c_b0, c_b1);
    else
      pass1_chunk<PINV, false>(w, qi, true, lut, lr, NR1, NR2, L, C, g, s_queue, s_coarse, qn, c_nw, c_b0, c_b1);
  };
  // every lane of a warp runs the same number of iterations (warp-uniform
  // loops), so the queue and stack bookkeeping needs only warp-level operations
  if (flat_fast(g)) {
    // one long row, 16-byte aligned, fewer than 2^31 full chunks: 32-bit
    // chunk indices, no per-chunk position arithmetic; the row's partial
    // last chunk is counted after the loop
    const unsigned nfull = (unsigned)((u64)g.npx / kChunk);
    const unsigned stride32 = gridDim.x * blockDim.x;
    const uint4* src4 = reinterpret_cast<const uint4*>(g.src);
    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nfull;
         base += stride32) {
      const unsigned q = base + lane;
      unsigned w[12];
      bool tissue = false;
      if (q < nfull && SPCN_CHECK((int64_t)(q + 1ull) * (3 * kChunk) <= g.src_bytes, g.err)) {
        const uint4* v = src4 + 3ull * q;
        const uint4 x = __ldg(v), y = __ldg(v + 1), z = __ldg(v + 2);
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
        w[4] = y.x; w[5] = y.y; w[6] = y.z; w[7] = y.w;
        w[8] = z.x; w[9] = z.y; w[10] = z.z; w[11] = z.w;
        tissue = !chunk_white(w, wm, we) && classify(w);
      }
      warp_step(tissue, w, q);
    }
    const int tail = (int)((u64)g.npx % kChunk);
    if (tail && (u64)blockIdx.x * blockDim.x + threadIdx.x == (u64)nfull % stride) {
      const int64_t off = (int64_t)nfull * (3 * kChunk);
      if (SPCN_CHECK(off + 3 * (int64_t)tail <= g.src_bytes, g.err))
        partial_chunk<PINV>(g.src + off, tail, lut, lr, L, C, s_coarse, c_nw, c_b0, c_b1);
    }
  } else {
    for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < g.nchunks;
         base += stride) {
      const u64 q = base + lane;
      unsigned w[12];
      bool tissue = false;
      if (q < g.nchunks) {
        const ChunkPos p = chunk_pos(g, q);
        load_chunk<false>(g, p, w);
        if (p.n != kChunk) {
          if (SPCN_CHECK(p.src_off >= 0 && p.src_off + 3 * (int64_t)p.n <= g.src_bytes, g.err))
            partial_chunk<PINV>(g.src + p.src_off, p.n, lut, lr, L, C, s_coarse, c_nw, c_b0, c_b1);
        } else {
          tissue = !chunk_white(w, wm, we) && classify(w);
        }
      }
      warp_step(tissue, w, (unsigned)q);
    }
  }
  __syncwarp();
  if (ns > 0) {   // the rest of the stack (fewer than 32)
    const bool have = lane < (unsigned)ns;
    unsigned w[12];
    unsigned qi = 0u;
    if (have) stack_get(s_stk, s_stq, (int)lane, w, qi);
    if (wbelow)
      pass1_chunk<PINV, true>(w, qi, have, lut, lr, NR1, NR2, L, C, g, s_queue, s_coarse, qn, c_nw, c_b0, c_b1);
    else
      pass1_chunk<PINV, false>(w, qi, have, lut, lr, NR1, NR2, L, C, g, s_queue, s_coarse, qn, c_nw, c_b0, c_b1);
  }
  if (qn > 0) {
    __syncwarp();
    drain_pixels<PINV>(s_queue, qn, g, lut, lr, L, C, s_coarse);
  }
  // per-thread counts are exact in FP32 (fewer than 2^24 pixels per thread).
  // A thread's below counts can be negative (a tissue chunk's white pixels
  // are taken off by the lane that classified it, and counted by the lane
  // that runs its lasso); the sums wrap modulo 2^64 to the block's exact total.
  auto as_u64 = [](float x) { return (u64)(long long)x; };
  const u64 t_nw = block_sum((u64)lo_of(c_nw) + (u64)hi_of(c_nw), s_tmp);
  const u64 t_b0 = block_sum(as_u64(lo_of(c_b0)) + as_u64(hi_of(c_b0)), s_tmp);
  const u64 t_b1 = block_sum(as_u64(lo_of(c_b1)) + as_u64(hi_of(c_b1)), s_tmp);
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
    window_select<DEV>(a);
  }
}


struct SelectImageArgs {
  ImageSource src;
  const Model* m;
  SelectState* sel;
  u64* ghist;
  u64* fallbacks;   // counts the launches that had a rank to resolve (or null)
  int* err;
  long long timeout_ns;
  double tgt0, tgt1;
};

template <bool PINV>
__global__ void __launch_bounds__(kPassThreads, 1) k_select_image(SelectImageArgs a) {
  if (*(volatile int*)&a.sel->all_resolved) return;   // uniform: every block returns
  if (a.fallbacks && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.fallbacks, 1ull);
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
  radix_select<PINV>(a.src, s_dyn, L, a.sel, rank, active, a.ghist, s_hist, &a.sel->barrier, a.err,
               a.timeout_ns, a.tgt0, a.tgt1);
}

// ------------------------------------------------------------ window-miss recovery
// When a rank fell outside pass 1's window it is found by counting passes
// instead of the radix select over every key.  A round counts, for each stain
// with an unresolved rank, the non-white pixels in 32 consecutive key ranges
// of 2^shift keys each (a ladder), with warp ballots into per-lane counters:
// no atomics per pixel.  The ranges are walked with the exact count of pixels
// below them to find the range that holds each unresolved rank; the union of
// a stain's ranges is the next round's span.  Once a stain's span is at most
// kWinBins keys, one more pass histograms the keys of that span exactly (as
// pass 1 does its window) and the ranks are selected there.  The first round
// starts next to the missed window: descending from its start, or ascending
// from its end (with no window, descending from the key of 1.0, above every
// scaled lasso density).  Every pixel's key is computed by pass 1's
// arithmetic, so the keys are those of every other pass, bit for bit.  A rank
// not found this way (ranks far apart, or a failed wait) is left to the radix
// select that follows.  Not for the pseudo-inverse (signed keys).
constexpr int kLadderBins = 32;
constexpr int kLadderRounds = 6;
constexpr unsigned kKeyInf = 0x7F800000u;    // +inf: above every density
constexpr unsigned kKeyOne = 0x3F800000u;    // 1.0: above every scaled lasso density
constexpr size_t kLadderSmem = kLutSmemBytes + sizeof(unsigned) * 2 * kWinGroups;
// scratch of the recovery inside the context's radix histograms
constexpr int kLadderCountOff = 0;                                  // [rounds][2][32] u64
constexpr int kLadderCoarseOff = 2 * kLadderBins * kLadderRounds;   // [2][kWinGroups] u64
constexpr int kLadderScratch = kLadderCoarseOff + 2 * kWinGroups;
static_assert(kLadderScratch <= 3 * kTracks * kRadixBins, "recovery scratch fits");

struct LadderArgs {
  Geometry g;
  unsigned wthr;        // (white threshold + 1) << 8, compared with table offsets
  unsigned wm, we;      // all-white test of a full chunk, as in pass 1
  const Model* m;
  SelectState* sel;
  const u64* win_coarse;   // pass 1's window counts [2][kWinGroups] (read before any write)
  u64* scratch;         // kLadderScratch u64 (counts, final coarse bins)
  u64* fine;            // [2][kWinBins], the final span's exact bins
  u64* misses;          // launches that had a rank to find
  int* err;
  long long timeout_ns;
  double tgt0, tgt1;
};

// Per stain: the key span [lo, hi) that holds its unresolved ranks, the exact
// count of non-white pixels below lo, and the ladder of the next round.
struct LadderSpan {
  unsigned lo, hi;
  u64 below_lo;         // pixels with key < lo
  u64 below_hi;         // pixels with key < hi (descending ladders)
  int dir;              // -1: ranges [hi - (b+1) 2^shift, hi - b 2^shift); +1: [lo + b 2^shift, ...)
  int shift;
  int state;            // 0: nothing to find, 1: counting, 2: final (hi - lo <= kWinBins), 3: given up
};

// Ranges of ladder bin b (64-bit, clamped to [0, kKeyInf]).
__device__ __forceinline__ void ladder_range(const LadderSpan& s, int b, long long* lo,
                                             long long* hi) {
  const long long w = 1ll << s.shift;
  if (s.dir < 0) {
    *hi = (long long)s.hi - (long long)b * w;
    *lo = *hi - w;
  } else {
    *lo = (long long)s.lo + (long long)b * w;
    *hi = *lo + w;
  }
  if (*lo < 0) *lo = 0;
  if (*hi > (long long)kKeyInf) *hi = kKeyInf;
}

__device__ __forceinline__ int shift_for(u64 width) {
  int s = 0;
  while (((u64)kLadderBins << s) < width) ++s;
  return s;
}

// Find the range of each unresolved track of stain j from a round's counts
// and narrow the stain's span to their union.
__device__ void ladder_update(LadderSpan& S, const u64* cnt, const SelectState* s, int j) {
  long long nlo = -1, nhi = -1;
  u64 nbelow = 0;
  for (int t = 2 * j; t < 2 * j + 2; ++t) {
    if (__ldcg(&s->resolved[t])) continue;
    const u64 r = __ldcg(&s->rank[t]);
    long long blo = -1, bhi = -1;
    u64 bb = 0;
    if (S.dir < 0) {
      u64 c = S.below_hi;
      for (int b = 0; b < kLadderBins; ++b) {
        c -= __ldcg(cnt + b);
        if (r >= c) { ladder_range(S, b, &blo, &bhi); bb = c; break; }
      }
      if (blo < 0) {   // below the ladder
        long long l0, h0;
        ladder_range(S, kLadderBins - 1, &l0, &h0);
        blo = 0; bhi = l0; bb = 0;
      }
    } else {
      u64 c = S.below_lo;
      for (int b = 0; b < kLadderBins; ++b) {
        const u64 x = __ldcg(cnt + b);
        if (r < c + x) { ladder_range(S, b, &blo, &bhi); bb = c; break; }
        c += x;
      }
      if (blo < 0) {   // above the ladder
        long long l0, h0;
        ladder_range(S, kLadderBins - 1, &l0, &h0);
        blo = h0; bhi = kKeyInf; bb = c;
      }
    }
    if (nlo < 0 || blo < nlo) { nlo = blo; nbelow = bb; }
    if (bhi > nhi) nhi = bhi;
  }
  if (nlo < 0 || nhi <= nlo) { S.state = 3; return; }   // cannot happen for valid counts
  S.lo = (unsigned)nlo;
  S.hi = (unsigned)nhi;
  S.below_lo = nbelow;
  S.dir = 1;
  const u64 width = (u64)(nhi - nlo);
  if (width <= (u64)kWinBins) { S.state = 2; return; }
  S.shift = shift_for(width);
}

// Warp-uniform traversal of the pixels that may matter: a chunk is skipped
// when it is all white or when its density bound (every pixel's key is at
// most the bound's, see below_bound) lies below low0 and low1, the lowest
// keys the caller counts for each stain; a warp skips its 32 chunks when none
// is kept.  Otherwise every lane calls body for each of the 16 pixel slots of
// its chunk (nw is false for slots without a counted pixel), so body may use
// warp-wide operations.
template <class Body>
__device__ __forceinline__ void ladder_pixels(const LadderArgs& a, const char* lut, const Lasso& L,
                                              unsigned low0, unsigned low1, Body&& body) {
  const Geometry& g = a.g;
  const unsigned lr = lane_reg();
  const unsigned lane = threadIdx.x & 31u;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < g.nchunks;
       base += stride) {
    const u64 q = base + lane;
    unsigned w[12];
    int n = 0;
    if (q < g.nchunks) {
      const ChunkPos p = chunk_pos(g, q);
      load_chunk<false>(g, p, w);
      if (!chunk_white(w, a.wm, a.we)) {   // padding bytes read white and lower no minimum
        unsigned b1, b2;
        chunk_bound_keys(w, lut, lr, &b1, &b2);
        if (b1 >= low0 || b2 >= low1) n = p.n;
      }
    }
    if (!__any_sync(0xFFFFFFFFu, n > 0)) continue;
#pragma unroll
    for (int k = 0; k < kChunk; k += 2) {   // two pixels per packed lasso (same arithmetic)
      unsigned aRA, aGA, aBA, aRB, aGB, aBB;
      pixel_addr(w, k, lr, aRA, aGA, aBA);
      pixel_addr(w, k + 1, lr, aRB, aGB, aBB);
      const bool nwA = k < n && min(min(aRA, aGA), aBA) < a.wthr;
      const bool nwB = k + 1 < n && min(min(aRB, aGB), aBB) < a.wthr;
      f2 H1, H2;
      solve_pair<false>(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, L.kappa, H1, H2);
      body(nwA, __float_as_uint(lo_of(H1)), __float_as_uint(lo_of(H2)));
      body(nwB, __float_as_uint(hi_of(H1)), __float_as_uint(hi_of(H2)));
    }
  }
}

// Lane b of the warp adds the number of lanes whose bin is b (bins >= 32 are
// not counted): the lanes with a bin, then one ballot per bit of the bin,
// each kept or inverted by the matching bit of the lane's own index (flip[i]
// is all ones where bit i of the lane index is 0).
__device__ __forceinline__ void ballot_count(unsigned bin, const unsigned (&flip)[5],
                                             unsigned& cnt) {
  unsigned m = __ballot_sync(0xFFFFFFFFu, bin < (unsigned)kLadderBins);
#pragma unroll
  for (int i = 0; i < 5; ++i) m &= __ballot_sync(0xFFFFFFFFu, (bin >> i) & 1u) ^ flip[i];
  cnt += (unsigned)__popc(m);
}

__global__ void __launch_bounds__(kPassThreads, 1) k_select_ladder(LadderArgs a) {
  SelectState* s = a.sel;
  if (*(volatile int*)&s->all_resolved) return;   // uniform: every block returns
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.misses, 1ull);
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_coarse = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);   // [2][kWinGroups]
  __shared__ unsigned s_cnt[2][kLadderBins];
  __shared__ u64 s_tmp[33];
  __shared__ int s_idx, s_idx2;
  __shared__ u64 s_before, s_before2;
  const u64 n = __ldcg(&s->n_nw);
  // pass 1's in-window counts (its coarse groups), one block sum per stain
  u64 inwin[2];
  for (int j = 0; j < 2; ++j) {
    u64 part = 0;
    for (int i = threadIdx.x; i < kWinGroups; i += blockDim.x)
      part += __ldcg(a.win_coarse + j * kWinGroups + i);
    inwin[j] = block_sum(part, s_tmp);
  }
  // first spans, from pass 1's outcome (the same in every block)
  LadderSpan S[2];
  for (int j = 0; j < 2; ++j) {
    LadderSpan& X = S[j];
    X.state = 0;
    const int u0 = !__ldcg(&s->resolved[2 * j]), u1 = !__ldcg(&s->resolved[2 * j + 1]);
    if (!u0 && !u1) continue;
    const unsigned lo = __ldcg(&s->lo[j]), nb = __ldcg(&s->nb[j]);
    const u64 below = __ldcg(&s->below[j]);
    bool under = true, over = true;
    for (int t = 2 * j; t < 2 * j + 2; ++t) {
      if (__ldcg(&s->resolved[t])) continue;
      const u64 r = __ldcg(&s->rank[t]);
      under = under && r < below;
      over = over && r >= below + inwin[j];
    }
    X.state = 1;
    if (nb == 0) {                     // no window: below the key of 1.0, 8 binades
      X.lo = 0; X.hi = kKeyOne; X.below_lo = 0; X.below_hi = n; X.dir = -1; X.shift = 21;
    } else if (under) {                // below the window: two binades under its start
      X.lo = 0; X.hi = lo; X.below_lo = 0; X.below_hi = below; X.dir = -1; X.shift = 19;
    } else if (over) {                 // above the window: two binades over its end
      X.lo = lo + nb; X.hi = kKeyInf; X.below_lo = below + inwin[j]; X.below_hi = n;
      X.dir = 1; X.shift = 19;
    } else {                           // cannot happen (adjacent ranks); search everything
      X.lo = 0; X.hi = kKeyInf; X.below_lo = 0; X.below_hi = n; X.dir = 1;
      X.shift = shift_for(kKeyInf);
    }
  }
  // zero the counts and the final bins (pass 1's are no longer needed)
  const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 gstride = (u64)gridDim.x * blockDim.x;
  for (u64 i = gtid; i < (u64)kLadderScratch; i += gstride) a.scratch[i] = 0ull;
  for (u64 i = gtid; i < 2ull * kWinBins; i += gstride) a.fine[i] = 0ull;
  unsigned target = gridDim.x;
  if (!grid_barrier(&s->barrier2, target, &s->abort, a.err, a.timeout_ns)) return;
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const Lasso L = a.m->lasso;
  const unsigned lane = threadIdx.x & 31u;
  unsigned flip[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) flip[i] = ((lane >> i) & 1u) ? 0u : 0xFFFFFFFFu;
  for (int round = 0; round < kLadderRounds; ++round) {
    if (S[0].state != 1 && S[1].state != 1) break;   // uniform
    for (int i = threadIdx.x; i < 2 * kLadderBins; i += blockDim.x) (&s_cnt[0][0])[i] = 0u;
    __syncthreads();
    unsigned c0 = 0u, c1 = 0u;
    // each stain's ladder as bin = (key - base) >> shift (ascending) or
    // (base - key) >> shift (descending, base = hi - 1), in plain registers
    const unsigned base0 = S[0].dir < 0 ? S[0].hi - 1u : S[0].lo;
    const unsigned base1 = S[1].dir < 0 ? S[1].hi - 1u : S[1].lo;
    const unsigned sh0 = (unsigned)S[0].shift, sh1 = (unsigned)S[1].shift;
    const bool desc0 = S[0].dir < 0, desc1 = S[1].dir < 0;
    const bool on0 = S[0].state == 1, on1 = S[1].state == 1;
    // lowest key each stain's ladder counts (none: above every key)
    const unsigned low0 = !on0 ? 0xFFFFFFFFu : (desc0 ? (unsigned)max(0ll, (long long)base0 + 1ll -
                                                                       (32ll << sh0)) : base0);
    const unsigned low1 = !on1 ? 0xFFFFFFFFu : (desc1 ? (unsigned)max(0ll, (long long)base1 + 1ll -
                                                                       (32ll << sh1)) : base1);
    // distance from the ladder's base in its direction: keys on the other
    // side wrap around to huge distances and land beyond bin 31
    const unsigned mul0 = desc0 ? 0xFFFFFFFFu : 1u, mul1 = desc1 ? 0xFFFFFFFFu : 1u;
    ladder_pixels(a, lut, L, low0, low1, [&](bool nw, unsigned k1, unsigned k2) {
      const unsigned b1 = nw ? min(((k1 - base0) * mul0) >> sh0, 32u) : 32u;
      const unsigned b2 = nw ? min(((k2 - base1) * mul1) >> sh1, 32u) : 32u;
      if (on0 && __any_sync(0xFFFFFFFFu, b1 < 32u)) ballot_count(b1, flip, c0);
      if (on1 && __any_sync(0xFFFFFFFFu, b2 < 32u)) ballot_count(b2, flip, c1);
    });
    if (c0) atomicAdd(&s_cnt[0][lane], c0);
    if (c1) atomicAdd(&s_cnt[1][lane], c1);
    __syncthreads();
    u64* cnt = a.scratch + kLadderCountOff + (size_t)round * 2 * kLadderBins;
    if (threadIdx.x < 2 * kLadderBins) {
      const unsigned v = (&s_cnt[0][0])[threadIdx.x];
      if (v) atomicAdd(cnt + threadIdx.x, (u64)v);
    }
    target += gridDim.x;
    if (!grid_barrier(&s->barrier2, target, &s->abort, a.err, a.timeout_ns)) return;
    for (int j = 0; j < 2; ++j)
      if (S[j].state == 1) ladder_update(S[j], cnt + j * kLadderBins, s, j);
  }
  // the final spans: exact bins of every key, coarse groups per block
  if (S[0].state != 2 && S[1].state != 2) return;   // uniform: left to the radix select
  for (int i = threadIdx.x; i < 2 * kWinGroups; i += blockDim.x) s_coarse[i] = 0u;
  __syncthreads();
  {
    const unsigned lo0 = S[0].state == 2 ? S[0].lo : 0u, lo1 = S[1].state == 2 ? S[1].lo : 0u;
    unsigned w0 = S[0].state == 2 ? S[0].hi - S[0].lo : 0u;
    unsigned w1 = S[1].state == 2 ? S[1].hi - S[1].lo : 0u;
    if (!SPCN_CHECK(w0 <= (unsigned)kWinBins && w1 <= (unsigned)kWinBins, a.err)) w0 = w1 = 0u;
    u64* fine = a.fine;
    ladder_pixels(a, lut, L, w0 ? lo0 : 0xFFFFFFFFu, w1 ? lo1 : 0xFFFFFFFFu,
                  [&](bool nw, unsigned k1, unsigned k2) {
      if (!nw) return;
      const unsigned r1 = k1 - lo0, r2 = k2 - lo1;
      if (r1 < w0) {
        red_add_global(fine + r1, 1ull);
        red_add_shared(s_coarse + (r1 >> kWinGroupBits), 1u);
      }
      if (r2 < w1) {
        red_add_global(fine + kWinBins + r2, 1ull);
        red_add_shared(s_coarse + kWinGroups + (r2 >> kWinGroupBits), 1u);
      }
    });
  }
  __syncthreads();
  u64* coarse = a.scratch + kLadderCoarseOff;
  for (int i = threadIdx.x; i < 2 * kWinGroups; i += blockDim.x)
    if (s_coarse[i]) atomicAdd(coarse + i, (u64)s_coarse[i]);
  target += gridDim.x;
  if (!grid_barrier(&s->barrier2, target, &s->abort, a.err, a.timeout_ns)) return;
  if (blockIdx.x != 0) return;
  for (int t = 0; t < kTracks; ++t) {
    const int j = t >> 1;
    if (S[j].state != 2 || __ldcg(&s->resolved[t])) continue;   // uniform within the block
    const u64 r = __ldcg(&s->rank[t]) - S[j].below_lo;
    const unsigned width = S[j].hi - S[j].lo;
    const int ngroups = (int)((width + kWinGroup - 1) >> kWinGroupBits);
    block_find_rank(coarse + j * kWinGroups, ngroups, r, &s_idx, &s_before, s_tmp);
    if (s_idx < 0) continue;
    const unsigned gbeg = (unsigned)s_idx << kWinGroupBits;
    const int nbins = (int)min((unsigned)kWinGroup, width - gbeg);
    block_find_rank(a.fine + (size_t)j * kWinBins + gbeg, nbins, r - s_before, &s_idx2,
                    &s_before2, s_tmp);
    if (s_idx2 < 0) continue;
    if (threadIdx.x == 0) {
      s->key[t] = S[j].lo + gbeg + (unsigned)s_idx2;
      s->resolved[t] = 1;
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int t = 0; t < kTracks; ++t) all &= s->resolved[t];
    if (all) {
      finish_percentiles(s, a.tgt0, a.tgt1, L.hscale);
      __threadfence();
      s->all_resolved = 1;
    }
  }
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
  unsigned sub;      // 1: the whole list; s > 1: every s-th group of four (a hint only)
  int band;          // select the ends of the binomial band instead of ranks k, k+1
  const int* units;  // independent sampling units (kept patches), or null: every item
};

// The band of a hint: a population quantile p lies, with probability about
// 1 - 6e-5, between the sample's order statistics at p -/+ delta, delta =
// z sqrt(p (1 - p) / m_eff) with z = 4 (the binomial count below the quantile
// in an i.i.d. sample).  m_eff is the number of independent sampling units:
// the visited items of a pixel sample, the kept patches of a patch sample
// (pixels of one patch are not independent).  delta is capped at kBandMax, so
// that the window stays affordable when the sample says little.
constexpr double kBandZ = 4.0;
constexpr u64 kListMinVisited = 1ull << 18;
constexpr double kBandMax = 0.002;
__device__ __forceinline__ void band_ranks(u64 n, double pct, double m_eff, u64* r_lo, u64* r_hi) {
  const double p = pct / 100.0;
  double d = kBandZ * sqrt(p * (1.0 - p) / fmax(m_eff, 1.0));
  if (d > kBandMax) d = kBandMax;
  const double span = (double)(n - 1);
  double lo = floor((p - d) * span), hi = ceil((p + d) * span);
  if (lo < 0.0) lo = 0.0;
  if (hi > span) hi = span;
  if (lo > hi) lo = hi;
  *r_lo = (u64)lo;
  *r_hi = (u64)hi;
}

// Percentile of the densities of a packed list of non-white pixels (the basis
// sample, §3.1 item 2), radix select from scratch; with sub > 1 of a regular
// sub-sample of the list (used only as the search window's hint).
template <bool PINV>
__global__ void __launch_bounds__(kPassThreads, 1) k_select_list(SelectListArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_hist = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);
  const u64 n_all = __ldcg(a.n_dev);
  if (n_all == 0 || a.m->status != SPCN_OK) return;   // uniform: every block returns
  // a regular sub-sample keeps at least kListMinVisited items (a smaller
  // list is visited whole), so that the band's binomial width stays small
  const u64 most = n_all / kListMinVisited;
  const unsigned sub = (unsigned)(most < 1ull ? 1ull : (most < (u64)a.sub ? most : (u64)a.sub));
  const u64 n = ListSource::visited(n_all, sub);
  u64 rank[kTracks];
  int active[kTracks];
  double t;
  if (a.band) {   // tracks 2j, 2j+1: the band's ends; p99 = their midpoint
    const double m_eff = a.units ? (double)min((u64)max(*a.units, 1), n) : (double)n;
    band_ranks(n, a.pct, m_eff, &rank[0], &rank[1]);
    t = 0.5;
  } else {
    type7_ranks(n, a.pct, &rank[0], &rank[1], &t);
  }
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
  ListSource src{a.items, n_all, sub};
  radix_select<PINV>(src, s_dyn, L, a.sel, rank, active, a.ghist, s_hist, &a.sel->barrier, a.err,
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


template <bool PINV>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass_recon(ReconArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ float s_M[6];
  const Lasso L = a.m->lasso;
  if (threadIdx.x < 6) {
    s_M[threadIdx.x] = recon_coef(a.Wt, a.sel->scale, L.hscale, threadIdx.x);
  }
  load_od_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg_od();
  const ProjConst P = proj_const(a.m);
  ReconConst K;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    K.M1[c] = pk(s_M[c], s_M[c]);
    K.M2[c] = pk(s_M[3 + c], s_M[3 + c]);
    K.L2[c] = pk(a.l2i0[c], a.l2i0[c]);
  }
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  const Geometry& g = a.g;
  if (flat_fast(g) && g.vec_dst) {
    // one long row, source and output 16-byte aligned, fewer than 2^31 full
    // chunks: 32-bit chunk indices and plain vector accesses, the next
    // chunk's loads in flight while the current one is computed (two
    // register buffers); the row's partial last chunk after the loop
    const unsigned nfull = (unsigned)((u64)g.npx / kChunk);
    const unsigned stride32 = gridDim.x * blockDim.x;
    const uint4* src4 = reinterpret_cast<const uint4*>(g.src);
    uint4* dst4 = reinterpret_cast<uint4*>(g.dst);
    auto ld = [&](unsigned q, unsigned (&w)[12]) {
      if (!SPCN_CHECK((int64_t)(q + 1ull) * (3 * kChunk) <= g.src_bytes, g.err)) {
#pragma unroll
        for (int i = 0; i < 12; ++i) w[i] = 0xFFFFFFFFu;
        return;
      }
      const uint4* v = src4 + 3ull * q;
      const uint4 x = __ldcs(v), y = __ldcs(v + 1), z = __ldcs(v + 2);
      w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
      w[4] = y.x; w[5] = y.y; w[6] = y.z; w[7] = y.w;
      w[8] = z.x; w[9] = z.y; w[10] = z.z; w[11] = z.w;
    };
    auto run = [&](unsigned q, const unsigned (&w)[12]) {
      unsigned o[12];
      recon_chunk<PINV>(w, lut, lr, P, NR1, NR2, L.kappa, K, o);
      if (!SPCN_CHECK((int64_t)(q + 1ull) * (3 * kChunk) <= g.dst_bytes, g.err)) return;
      uint4* v = dst4 + 3ull * q;
      __stcs(v, make_uint4(o[0], o[1], o[2], o[3]));
      __stcs(v + 1, make_uint4(o[4], o[5], o[6], o[7]));
      __stcs(v + 2, make_uint4(o[8], o[9], o[10], o[11]));
    };
    unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned wa[12], wb[12];
    if (q < nfull) ld(q, wa);
    while (q < nfull) {
      unsigned qn = q + stride32;
      if (qn < nfull) ld(qn, wb);
      run(q, wa);
      q = qn;
      if (q >= nfull) break;
      qn = q + stride32;
      if (qn < nfull) ld(qn, wa);
      run(q, wb);
      q = qn;
    }
    if ((u64)g.npx % kChunk && (u64)blockIdx.x * blockDim.x + threadIdx.x == nfull % stride32) {
      const ChunkPos p = chunk_pos(g, (u64)nfull);
      unsigned w[12], o[12];
      load_chunk<true>(g, p, w);
      recon_chunk<PINV>(w, lut, lr, P, NR1, NR2, L.kappa, K, o);
      store_chunk(g, p, o);
    }
    return;
  }
  for_each_chunk<true, true>(g, [&](const unsigned (&w)[12], const ChunkPos& p) {
    unsigned o[12];
    recon_chunk<PINV>(w, lut, lr, P, NR1, NR2, L.kappa, K, o);
    store_chunk(g, p, o);
  });
}

// ------------------------------------------------------------ densities
struct DensityArgs {
  Geometry g;
  const Model* m;
  float* H;
  int64_t stride;   // elements between the two planes
};

// Densities of the pixels of one chunk (lane), scaled back (exact: the scale
// is a power of two): h1[k], h2[k] for pixel k of the chunk.
template <bool PINV>
__device__ __forceinline__ void density_chunk(const unsigned (&w)[12], const char* lut,
                                              unsigned lr, f2 NR1, f2 NR2, float kappa, f2 HS,
                                              float (&h1)[kChunk], float (&h2)[kChunk]) {
#pragma unroll
  for (int q = 0; q < kChunk / 2; ++q) {
    unsigned aRA, aGA, aBA, aRB, aGB, aBB;
    pixel_addr(w, 2 * q, lr, aRA, aGA, aBA);
    pixel_addr(w, 2 * q + 1, lr, aRB, aGB, aBB);
    f2 H1, H2;
    solve_pair<PINV>(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, kappa, H1, H2);
    H1 = mul2(H1, HS);
    H2 = mul2(H2, HS);
    h1[2 * q] = lo_of(H1);
    h1[2 * q + 1] = hi_of(H1);
    h2[2 * q] = lo_of(H2);
    h2[2 * q + 1] = hi_of(H2);
  }
}

// One plane of a warp's 32 consecutive full chunks (512 pixels from px0),
// staged through shared memory so that each store writes 512 contiguous
// bytes (the lanes' own 64-byte runs would each half-fill 32 sectors).
// The 16-byte slots are XOR-swizzled so that every 8-lane phase of both the
// lane-strided writes and the contiguous reads hits 8 distinct bank groups:
// slot 4L+v (lane L's vector v) lives at (4L+v) ^ ((L>>1)&3).
__device__ __forceinline__ void store_plane_coalesced(float* dst, const float (&h)[kChunk],
                                                      float4* stage, unsigned lane) {
  const unsigned sw = (lane >> 1) & 3u;
#pragma unroll
  for (int v = 0; v < 4; ++v)
    stage[(4u * lane + v) ^ sw] = make_float4(h[4 * v], h[4 * v + 1], h[4 * v + 2], h[4 * v + 3]);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 4; ++k)
    __stcs(reinterpret_cast<float4*>(dst) + 32 * k + lane, stage[(32u * k + lane) ^ (lane >> 3)]);
  __syncwarp();
}

template <bool PINV>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass_density(DensityArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  float4* stage = reinterpret_cast<float4*>(s_dyn + kLutSmemBytes) + (threadIdx.x >> 5) * 128;
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  const unsigned lane = threadIdx.x & 31u;
  const Lasso L = a.m->lasso;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  const f2 HS = pk(L.hscale, L.hscale);
  const bool vec_h = ((reinterpret_cast<uintptr_t>(a.H) & 15u) == 0) && ((a.stride & 3) == 0);
  const Geometry g = a.g;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  // warp-uniform loop: a warp handles 32 consecutive chunks per iteration
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < g.nchunks;
       base += stride) {
    const u64 q = base + lane;
    const bool have = q < g.nchunks;
    ChunkPos p;
    p.px = 0;
    p.n = 0;
    float h1[kChunk], h2[kChunk];
    if (have) {
      p = chunk_pos(g, q);
      unsigned w[12];
      load_chunk<true>(g, p, w);
      density_chunk<PINV>(w, lut, lr, NR1, NR2, L.kappa, HS, h1, h2);
    }
    const u64 px0 = __shfl_sync(0xFFFFFFFFu, p.px, 0);
#ifdef SPCN_CHECKED
    const bool inside = !have || SPCN_CHECK(p.px + (u64)p.n <= (u64)g.npx, g.err);
    if (!__all_sync(0xFFFFFFFFu, inside)) continue;   // a plane index beyond the image: no store
#endif
    const bool run = __all_sync(0xFFFFFFFFu, have && p.n == kChunk && p.px == px0 + 16u * lane);
    if (run && vec_h && (px0 & 3) == 0) {
      store_plane_coalesced(a.H + px0, h1, stage, lane);
      store_plane_coalesced(a.H + a.stride + px0, h2, stage, lane);
    } else if (have) {
      float* d0 = a.H + p.px;
      float* d1 = a.H + a.stride + p.px;
      if (p.n == kChunk && vec_h && (p.px & 3) == 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          __stcs(reinterpret_cast<float4*>(d0) + v,
                 make_float4(h1[4 * v], h1[4 * v + 1], h1[4 * v + 2], h1[4 * v + 3]));
          __stcs(reinterpret_cast<float4*>(d1) + v,
                 make_float4(h2[4 * v], h2[4 * v + 1], h2[4 * v + 2], h2[4 * v + 3]));
        }
      } else {
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
          if (k < p.n) { d0[k] = h1[k]; d1[k] = h2[k]; }
      }
    }
  }
}

// ------------------------------------------------------------ failure-detection hook
__global__ void k_debug_barrier(SelectState* s, int* err, int extra, long long timeout_ns) {
  grid_barrier(&s->barrier, gridDim.x + (unsigned)extra, &s->abort, err, timeout_ns);
}

// ------------------------------------------------------------ host launchers
static int grid_of(const Context* c, int occ) {
  return c->num_sms * (occ > 0 ? occ : 1);
}

// Shared-memory limit of a kernel and its blocks per SM (the smaller over the
// instantiations that share one grid size).
template <class K>
static int smem_attr(K* k, size_t smem) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess ? SPCN_OK : SPCN_ERR_CUDA;
}
template <class K>
static int occ_min(int* occ, K* k, int threads, size_t smem) {
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, threads, smem) != cudaSuccess)
    return SPCN_ERR_CUDA;
  if (*occ == 0 || o < *occ) *occ = o;
  return SPCN_OK;
}

int configure_pixel_kernels(Context* c) {
  int rc = 0;
  rc |= smem_attr(k_pass_window<false, false>, kWindowSmem);
  rc |= smem_attr(k_pass_window<true, false>, kWindowSmem);
  rc |= smem_attr(k_pass_window<false, true>, kWindowSmem);
  rc |= smem_attr(k_pass_window<true, true>, kWindowSmem);
  rc |= smem_attr(k_pass_recon<false>, kLutSmemBytes);
  rc |= smem_attr(k_pass_recon<true>, kLutSmemBytes);
  rc |= smem_attr(k_pass_density<false>, kDensitySmem);
  rc |= smem_attr(k_pass_density<true>, kDensitySmem);
  rc |= smem_attr(k_select_image<false>, kRadixSmem);
  rc |= smem_attr(k_select_image<true>, kRadixSmem);
  rc |= smem_attr(k_select_list<false>, kRadixSmem);
  rc |= smem_attr(k_select_list<true>, kRadixSmem);
  rc |= smem_attr(k_select_ladder, kLadderSmem);
  if (rc) return SPCN_ERR_CUDA;
  c->occ_window = c->occ_recon = c->occ_density = c->occ_select = c->occ_radix_list = 0;
  c->occ_debug = 0;
  rc |= occ_min(&c->occ_window, k_pass_window<false, false>, kPassThreads, kWindowSmem);
  rc |= occ_min(&c->occ_window, k_pass_window<true, false>, kPassThreads, kWindowSmem);
  rc |= occ_min(&c->occ_window, k_pass_window<false, true>, kPassThreads, kWindowSmem);
  rc |= occ_min(&c->occ_window, k_pass_window<true, true>, kPassThreads, kWindowSmem);
  rc |= occ_min(&c->occ_recon, k_pass_recon<false>, kPassThreads, kLutSmemBytes);
  rc |= occ_min(&c->occ_recon, k_pass_recon<true>, kPassThreads, kLutSmemBytes);
  rc |= occ_min(&c->occ_density, k_pass_density<false>, kPassThreads, kDensitySmem);
  rc |= occ_min(&c->occ_density, k_pass_density<true>, kPassThreads, kDensitySmem);
  rc |= occ_min(&c->occ_select, k_select_image<false>, kPassThreads, kRadixSmem);
  rc |= occ_min(&c->occ_select, k_select_image<true>, kPassThreads, kRadixSmem);
  rc |= occ_min(&c->occ_select, k_select_ladder, kPassThreads, kLadderSmem);
  rc |= occ_min(&c->occ_radix_list, k_select_list<false>, kPassThreads, kRadixSmem);
  rc |= occ_min(&c->occ_radix_list, k_select_list<true>, kPassThreads, kRadixSmem);
  rc |= occ_min(&c->occ_debug, k_debug_barrier, 128, 0);
  if (rc) return SPCN_ERR_CUDA;
  if (c->occ_window < 1 || c->occ_recon < 1 || c->occ_density < 1 || c->occ_select < 1 ||
      c->occ_radix_list < 1 || c->occ_debug < 1)
    return SPCN_ERR_CUDA;
  return SPCN_OK;
}

// Window of the source's P99 from the basis estimated on the device (the
// sample percentile as the hint, in the units of the source table), so that a
// normalisation can follow a basis estimation without a host round trip.  A
// failed estimation is recorded in the error word and leaves no window (the
// exact fallback then runs; the outputs are computed but the call reports
// the error).
// The sample select ran in band mode: per stain, keys 2j and 2j+1 are the
// sample's order statistics at the ends of the binomial band around the
// percentile, p99[j] the band's midpoint (all in the sample model's scaled
// units); the window covers the band in the image model's units.
__global__ void k_window_from_basis(const Model* m, const Model* sample_model,
                                    const SelectState* sample_sel, const int* basis_status,
                                    Window* w, int* err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int st = *basis_status;
  if (st == SPCN_OK) st = m->status;
  if (st != SPCN_OK) record_error(err, st);
  if (st != SPCN_OK) {
    *w = window_for(0.0, 0.0);
    return;
  }
  const double hs = ldexp(1.0, -m->lasso.hexp);
  const double hb = (double)sample_model->lasso.hscale;   // sample keys -> densities
  Window r;
  unsigned* lo[2] = {&r.lo0, &r.lo1};
  unsigned* nb[2] = {&r.nb0, &r.nb1};
  float* nk[2] = {&r.nk0, &r.nk1};
  float* lk[2] = {&r.lk0, &r.lk1};
  float* nh[2] = {&r.nh0, &r.nh1};
  float* hk[2] = {&r.hk0, &r.hk1};
  for (int j = 0; j < 2; ++j)
    window_band((double)__uint_as_float(sample_sel->key[2 * j]) * hb * hs,
                (double)__uint_as_float(sample_sel->key[2 * j + 1]) * hb * hs,
                sample_sel->p99[j] * hs, lo[j], nb[j], nk[j], lk[j], nh[j], hk[j]);
  *w = r;
}

int launch_window_from_basis(Context* c, const Model* m, const Model* sample_model,
                             const SelectState* sample_sel, const int* basis_status, Window* w,
                             cudaStream_t st) {
  k_window_from_basis<<<1, 32, 0, st>>>(m, sample_model, sample_sel, basis_status, w, c->err);
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

// SPCN_FLAG_P99_SAMPLED: the source percentile is not measured but given,
// either by the caller or by the basis estimation on the device; the Eq. 3
// factors are then formed exactly as after a measured percentile.
__device__ __forceinline__ void set_given_percentiles(SelectState* s, double p0, double p1,
                                                      double t0, double t1) {
  const double p[2] = {p0, p1}, tg[2] = {t0, t1};
  for (int j = 0; j < 2; ++j) {
    s->p99[j] = p[j];
    s->scale[j] = (p[j] != 0.0) ? tg[j] / p[j] : 1.0;
  }
  s->all_resolved = 1;
}

__global__ void k_scale_given(SelectState* s, double p0, double p1, double t0, double t1) {
  if (blockIdx.x == 0 && threadIdx.x == 0) set_given_percentiles(s, p0, p1, t0, t1);
}

// From the basis estimation left on the device; a failed estimation is
// recorded in the error word and leaves scale 1.
__global__ void k_scale_from_basis(const Model* m, const SelectState* sample_sel,
                                   const int* basis_status, SelectState* s, double t0, double t1,
                                   int* err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int st = *basis_status;
  if (st == SPCN_OK) st = m->status;
  if (st != SPCN_OK) record_error(err, st);
  set_given_percentiles(s, st == SPCN_OK ? sample_sel->p99[0] : 0.0,
                        st == SPCN_OK ? sample_sel->p99[1] : 0.0, t0, t1);
}

// A failed basis estimation left on the device goes to the error word (for
// calls whose later kernels do not read its percentile).
__global__ void k_check_basis(const Model* m, const int* basis_status, int* err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int st = *basis_status;
  if (st == SPCN_OK) st = m->status;
  if (st != SPCN_OK) record_error(err, st);
}

int launch_check_basis(Context* c, const Model* m, const int* basis_status, cudaStream_t st) {
  k_check_basis<<<1, 32, 0, st>>>(m, basis_status, c->err);
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

int launch_scale_given(Context* c, const double* p99, const double* tgt, cudaStream_t st) {
  k_scale_given<<<1, 32, 0, st>>>(c->sel, p99[0], p99[1], tgt[0], tgt[1]);
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

int launch_scale_from_basis(Context* c, const Model* m, const SelectState* sample_sel,
                            const int* basis_status, const double* tgt, cudaStream_t st) {
  k_scale_from_basis<<<1, 32, 0, st>>>(m, sample_sel, basis_status, c->sel, tgt[0], tgt[1],
                                       c->err);
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

// Constants of the conservative all-white test of a full chunk: every byte
// has its top k bits set, with k the smallest for which that puts a byte
// above the threshold T (256 - 2^(8-k) > T).  With T = 255 nothing is white
// and the test never passes (mask 0, expected 1).
void white_test_consts(int T, unsigned* wm, unsigned* we) {
  *wm = 0u;
  *we = 1u;
  for (int k = 1; k <= 8; ++k) {
    if (256 - (1 << (8 - k)) > T) {
      const unsigned byte = (0xFFu << (8 - k)) & 0xFFu;
      *wm = *we = byte * 0x01010101u;
      return;
    }
  }
}

// Pass 1 + select (+ radix fallback when a rank fell outside the window).
// The window comes from a host hint, or (wdev) from device memory.
static int percentile_passes(Context* c, const Geometry& g, const Model* m, int white_thresh,
                             double pct, const Window& w, const Window* wdev,
                             const double* tgt_p99, cudaStream_t st, bool pinv) {
  WindowArgs a;
  a.g = g;
  a.m = m;
  a.sel = c->sel;
  a.fine = c->fine;
  a.coarse = c->coarse;
  a.err = c->err;
  a.wthr = ((unsigned)white_thresh + 1u) << 8;
  white_test_consts(white_thresh, &a.wm, &a.we);
  a.w = w;
  a.wdev = wdev;
  a.pct = pct;
  a.tgt0 = tgt_p99 ? tgt_p99[0] : 1.0;
  a.tgt1 = tgt_p99 ? tgt_p99[1] : 1.0;
  SPCN_CUDA_TRY(cudaMemsetAsync(c->sel, 0, sizeof(SelectState), st));
  SPCN_CUDA_TRY(cudaMemsetAsync(c->coarse, 0, sizeof(u64) * 2 * kWinGroups, st));
  // the window's bins (all of them when the width is known on the device only)
  const unsigned nb0 = wdev ? (unsigned)kWinBins : w.nb0, nb1 = wdev ? (unsigned)kWinBins : w.nb1;
  if (nb0) SPCN_CUDA_TRY(cudaMemsetAsync(c->fine, 0, sizeof(u64) * nb0, st));
  if (nb1) SPCN_CUDA_TRY(cudaMemsetAsync(c->fine + kWinBins, 0, sizeof(u64) * nb1, st));
  {
    TimedLaunch tl(c, SPCN_KERNEL_PASS1, st);
    const int grid = grid_of(c, c->occ_window);
    if (wdev && pinv)
      k_pass_window<true, true><<<grid, kPassThreads, kWindowSmem, st>>>(a);
    else if (wdev)
      k_pass_window<true, false><<<grid, kPassThreads, kWindowSmem, st>>>(a);
    else if (pinv)
      k_pass_window<false, true><<<grid, kPassThreads, kWindowSmem, st>>>(a);
    else
      k_pass_window<false, false><<<grid, kPassThreads, kWindowSmem, st>>>(a);
  }
  SPCN_LAUNCH_CHECK(c);

  if (!pinv) {   // a rank outside the window: counting passes first
    LadderArgs l;
    l.g = g;
    l.wthr = a.wthr;
    l.wm = a.wm;
    l.we = a.we;
    l.m = m;
    l.sel = c->sel;
    l.win_coarse = c->coarse;
    l.scratch = c->rhist;
    l.fine = c->fine;
    l.misses = c->fallbacks;
    l.err = c->err;
    l.timeout_ns = c->timeout_ns;
    l.tgt0 = a.tgt0;
    l.tgt1 = a.tgt1;
    void* largs[] = {&l};
    TimedLaunch tl(c, SPCN_KERNEL_LADDER, st);
    SPCN_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_select_ladder, grid_of(c, c->occ_select),
                                              kPassThreads, largs, kLadderSmem, st));
    c->launches++;
  }
  SelectImageArgs s;
  s.src.g = g;
  s.src.thr = (unsigned)white_thresh;
  s.m = m;
  s.sel = c->sel;
  s.ghist = c->rhist;
  s.fallbacks = pinv ? c->fallbacks : nullptr;   // the lasso's misses are counted by the recovery
  s.err = c->err;
  s.timeout_ns = c->timeout_ns;
  s.tgt0 = a.tgt0;
  s.tgt1 = a.tgt1;
  void* args[] = {&s};
  {
    TimedLaunch tl(c, SPCN_KERNEL_SELECT, st);
    SPCN_CUDA_TRY(cudaLaunchCooperativeKernel(
        pinv ? (void*)k_select_image<true> : (void*)k_select_image<false>,
        grid_of(c, c->occ_select), kPassThreads, args, kRadixSmem, st));
  }
  c->launches++;
  return SPCN_OK;
}

int launch_percentile_passes(Context* c, const Geometry& g, const Model* m, int white_thresh,
                             double pct, const double* hint, int hexp, const double* tgt_p99,
                             cudaStream_t st, bool pinv) {
  const double hs = ldexp(1.0, -hexp);
  const Window w = window_for(hint ? hint[0] * hs : 0.0, hint ? hint[1] * hs : 0.0);
  return percentile_passes(c, g, m, white_thresh, pct, w, nullptr, tgt_p99, st, pinv);
}

int launch_percentile_passes_dev(Context* c, const Geometry& g, const Model* m, int white_thresh,
                                 double pct, const Window* wdev, const double* tgt_p99,
                                 cudaStream_t st, bool pinv) {
  return percentile_passes(c, g, m, white_thresh, pct, window_for(0.0, 0.0), wdev, tgt_p99, st,
                           pinv);
}

int launch_select_list(Context* c, const uint32_t* items, const u64* n_dev, const Model* m,
                       SelectState* sel, u64* ghist, double pct, cudaStream_t st, bool pinv,
                       unsigned sub, bool band, const int* units) {
  SelectListArgs a;
  a.band = band ? 1 : 0;
  a.units = units;
  a.items = items;
  a.n_dev = n_dev;
  a.m = m;
  a.sel = sel;
  a.ghist = ghist;
  a.err = c->err;
  a.timeout_ns = c->timeout_ns;
  a.pct = pct;
  a.sub = sub < 1 ? 1 : sub;
  SPCN_CUDA_TRY(cudaMemsetAsync(sel, 0, sizeof(SelectState), st));
  void* args[] = {&a};
  SPCN_CUDA_TRY(cudaLaunchCooperativeKernel(
      pinv ? (void*)k_select_list<true> : (void*)k_select_list<false>,
      grid_of(c, c->occ_radix_list), kPassThreads, args, kRadixSmem, st));
  c->launches++;
  return SPCN_OK;
}

int launch_recon(Context* c, const Geometry& g, const Model* m, const float* Wt, const float* i0t,
                 cudaStream_t st, bool pinv) {
  ReconArgs a;
  a.g = g;
  a.m = m;
  a.sel = c->sel;
  for (int i = 0; i < 6; ++i) a.Wt[i] = Wt[i];
  for (int i = 0; i < 3; ++i) a.l2i0[i] = (float)log2((double)i0t[i]);
  {
    TimedLaunch tl(c, SPCN_KERNEL_PASS2, st);
    if (pinv)
      k_pass_recon<true><<<grid_of(c, c->occ_recon), kPassThreads, kLutSmemBytes, st>>>(a);
    else
      k_pass_recon<false><<<grid_of(c, c->occ_recon), kPassThreads, kLutSmemBytes, st>>>(a);
  }
  SPCN_LAUNCH_CHECK(c);
  return SPCN_OK;
}

int launch_density(Context* c, const Geometry& g, const Model* m, float* H, int64_t stride,
                   cudaStream_t st, bool pinv) {
  DensityArgs a;
  a.g = g;
  a.m = m;
  a.H = H;
  a.stride = stride;
  {
    TimedLaunch tl(c, SPCN_KERNEL_DENSITY, st);
    if (pinv)
      k_pass_density<true><<<grid_of(c, c->occ_density), kPassThreads, kDensitySmem, st>>>(a);
    else
      k_pass_density<false><<<grid_of(c, c->occ_density), kPassThreads, kDensitySmem, st>>>(a);
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
