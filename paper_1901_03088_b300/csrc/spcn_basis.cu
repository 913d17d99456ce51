// Basis estimation of the improved SPCN on sm_103a (§3.1 items 1-3, §3.2
// item 2, Eq. 2):
//   sampling       all pixels / SplitMix64 draws / non-background patches,
//                  packed as R | G<<8 | B<<16 in sample order;
//   compaction     stable split of the sample into non-white and bright lists;
//   i0             80th percentile per channel of <= 100000 bright pixels;
//   sparse NMF     one cooperative persistent kernel: per-pixel closed-form
//                  H-step, Gram sums added exactly in 64-bit fixed point, a
//                  grid barrier, and the exact column update of W computed
//                  identically by every block;
//   ordering       hematoxylin = larger OD(red) - OD(blue);
//   sample P99     exact radix select over the non-white sample.
#include <math.h>

#include "spcn_context.h"
#include "spcn_internal.cuh"

namespace spcn {

int launch_select_list(Context* c, const uint32_t* items, const u64* n_dev, const Model* m,
                       SelectState* sel, u64* ghist, double pct, cudaStream_t st,
                       bool pinv = false, unsigned sub = 1, bool band = false,
                       const int* units = nullptr);

constexpr int kCompactBlock = 4096;
constexpr int kCompactThreads = 512;
constexpr int kCompactPer = kCompactBlock / kCompactThreads;
constexpr int kSnmfThreads = 512;
constexpr int kMaxSnmfGrid = 4096;

// ------------------------------------------------------------ SplitMix64
// Published definition (Steele, Lea & Flood 2014): state += gamma; output
// mix(state).  Output n of a generator seeded with s is mix(s + (n+1) gamma).
__device__ __forceinline__ u64 sm64_mix(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ u64 sm64_output(u64 seed, u64 n) {
  return sm64_mix(seed + (n + 1ull) * 0x9E3779B97F4A7C15ull);
}

// Lemire's multiply-high range reduction of output n to [0, bound).
__device__ __forceinline__ u64 sm64_below(u64 seed, u64 n, u64 bound) {
  return __umul64hi(sm64_output(seed, n), bound);
}

__device__ __forceinline__ uint32_t load_pixel(const uint8_t* data, int64_t pitch, u64 x, u64 y) {
  const uint8_t* p = data + (int64_t)y * pitch + (int64_t)(x * 3);
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
}

__device__ __forceinline__ bool packed_nonwhite(uint32_t v, unsigned thr) {
  const unsigned r = v & 0xFFu, g = (v >> 8) & 0xFFu, b = (v >> 16) & 0xFFu;
  return min(r, min(g, b)) <= thr;
}

// ------------------------------------------------------------ sampling
struct SampleArgs {
  const uint8_t* data;
  int64_t pitch;
  int64_t width, height;
  u64 seed;
  uint32_t* out;
  u64 m;     // draws (all / hash)
  u64 cap;   // sample entries allocated
  int* err;
  u64* m_out;   // the estimation's sample size, written here on the device (no host
                // operand in the stream, so the call can be captured into a CUDA graph)
};

__global__ void k_sample_all(SampleArgs a) {
  const u64 n = (u64)a.width * a.height;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.m_out = a.m;
  if (!SPCN_CHECK(n <= a.cap, a.err)) return;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    a.out[i] = load_pixel(a.data, a.pitch, i % a.width, i / a.width);
}

__global__ void k_sample_hash(SampleArgs a) {
  const u64 n = (u64)a.width * a.height;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.m_out = a.m;
  if (!SPCN_CHECK(a.m <= a.cap, a.err)) return;
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < a.m; k += (u64)gridDim.x * blockDim.x) {
    const u64 idx = sm64_below(a.seed, k, n);
    if (!SPCN_CHECK(idx < n, a.err)) continue;
    a.out[k] = load_pixel(a.data, a.pitch, idx % a.width, idx / a.width);
  }
}

struct PatchArgs {
  const uint8_t* data;
  int64_t pitch;
  int64_t width, height;
  u64 seed;
  int P;
  int n_patches;
  int n_cand;
  unsigned thr;
  int* cand;          // [n_cand] non-white counts, then [n_patches] accepted candidates
  BasisState* bs;
  uint32_t* out;
  u64 cap;            // sample entries allocated
  int* err;
  // per-patch compaction (null: the sample is gathered and compacted apart):
  int ng;             // row groups of kPatchGroupRows rows per patch
  int* gcnt;          // [n_cand][ng] non-white pixels per row group
  u64* goff;          // [2][n_patches] list offsets of each kept patch (non-white, bright)
  uint32_t* nw;       // the non-white and bright lists
  uint32_t* br;
};

__device__ __forceinline__ void patch_origin(const PatchArgs& a, int k, u64* x0, u64* y0) {
  *x0 = sm64_below(a.seed, 2ull * (u64)k, (u64)(a.width - a.P + 1));
  *y0 = sm64_below(a.seed, 2ull * (u64)k + 1ull, (u64)(a.height - a.P + 1));
}

// Rows per group of the per-patch compaction: one warp compacts one group.
constexpr int kPatchGroupRows = 4;
constexpr int kRowBatch = 8;   // 32-pixel pieces of a row loaded at once by a compacting warp

// Pieces j0 .. j0 + kRowBatch - 1 of a patch row (lane: pixel x = 32 j +
// lane), packed R | G<<8 | B<<16, and whether each pixel exists (x < P).
__device__ __forceinline__ void load_row_batch(const uint8_t* row, int P, int j0, unsigned lane,
                                               uint32_t (&v)[kRowBatch], unsigned& have) {
  have = 0u;
#pragma unroll
  for (int j = 0; j < kRowBatch; ++j) {
    const int x = 32 * (j0 + j) + (int)lane;
    v[j] = 0u;
    if (x < P) {
      v[j] = (uint32_t)row[3 * x] | ((uint32_t)row[3 * x + 1] << 8) |
             ((uint32_t)row[3 * x + 2] << 16);
      have |= 1u << j;
    }
  }
}

// One block per candidate patch: its non-white pixel count (row groups by
// warps, columns by lanes, no per-pixel division), and with gcnt the count
// of every row group.
__global__ void k_patch_count(PatchArgs a) {
  __shared__ u64 s_tmp[33];
  const int k = blockIdx.x;
  u64 x0, y0;
  patch_origin(a, k, &x0, &y0);
  if (!SPCN_CHECK(x0 + (u64)a.P <= (u64)a.width && y0 + (u64)a.P <= (u64)a.height, a.err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int ng = (a.P + kPatchGroupRows - 1) / kPatchGroupRows;
  unsigned cnt = 0;
  for (int gi = warp; gi < ng; gi += nwarps) {
    unsigned gc = 0;
    const int y1 = min(a.P, (gi + 1) * kPatchGroupRows);
    for (int y = gi * kPatchGroupRows; y < y1; ++y) {
      const uint8_t* row = a.data + (int64_t)(y0 + (u64)y) * a.pitch + (int64_t)(x0 * 3);
      for (int x = lane; x < a.P; x += 32) {
        const unsigned r = row[3 * x], g = row[3 * x + 1], b = row[3 * x + 2];
        gc += min(r, min(g, b)) <= a.thr ? 1u : 0u;
      }
    }
    gc = __reduce_add_sync(0xFFFFFFFFu, gc);
    if (a.gcnt && lane == 0) a.gcnt[(size_t)k * ng + gi] = (int)gc;
    cnt += lane == 0 ? gc : 0u;
  }
  const u64 tot = block_sum(cnt, s_tmp);
  if (threadIdx.x == 0) a.cand[k] = (int)tot;
}

// Keep candidates, in order, while at least half their pixels are non-white:
// warp 0 scans them 32 at a time (ballot + prefix counts), the same list as
// a sequential scan.  With goff the whole block then places every kept row
// group in the non-white and bright lists: exclusive prefix sums of the
// groups' counts in sample order (kept patches in order, groups in order).
constexpr int kAcceptThreads = 1024;
__global__ void __launch_bounds__(kAcceptThreads) k_patch_accept(PatchArgs a) {
  __shared__ u64 s_tmp[33];
  __shared__ int s_n;
  const unsigned lane = threadIdx.x & 31u;
  const long long need = (long long)a.P * a.P;
  if (threadIdx.x < 32) {
    int n = 0;
    for (int k0 = 0; k0 < a.n_cand && n < a.n_patches; k0 += 32) {
      const int k = k0 + (int)lane;
      const bool ok = k < a.n_cand && 2ll * a.cand[k] >= need;
      const unsigned ball = __ballot_sync(0xFFFFFFFFu, ok);
      const int pos = n + __popc(ball & ((1u << lane) - 1u));
      if (ok && pos < a.n_patches) a.cand[a.n_cand + pos] = k;
      n += __popc(ball);
    }
    if (n > a.n_patches) n = a.n_patches;
    if (lane == 0) {
      s_n = n;
      a.bs->n_acc = n;
      a.bs->m = (u64)n * (u64)need;
      if (n == 0) a.bs->status = SPCN_ERR_NO_TISSUE;
    }
  }
  __syncthreads();
  if (!a.goff) return;
  // per kept patch, in order: non-white pixels = the candidate's count
  const int n = s_n;
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int p0 = min(n, (int)threadIdx.x * per), p1 = min(n, p0 + per);
  u64 lnw = 0;
  for (int q = p0; q < p1; ++q) lnw += (u64)a.cand[a.cand[a.n_cand + q]];
  u64 tnw;
  u64 onw = block_excl_scan(lnw, s_tmp, &tnw);
  u64 obr = (u64)p0 * (u64)need - onw;   // the rest of the earlier patches' pixels
  for (int q = p0; q < p1; ++q) {
    const u64 c = (u64)a.cand[a.cand[a.n_cand + q]];
    a.goff[q] = onw;
    a.goff[a.n_patches + q] = obr;
    onw += c;
    obr += (u64)need - c;
  }
  if (threadIdx.x == 0) {
    a.bs->n_nw = tnw;
    a.bs->n_br = (u64)n * (u64)need - tnw;
  }
}

// One warp per kept row group: its pixels in raster order, each appended to
// the non-white or the bright list (ballot + prefix counts) after the
// patch's earlier groups (their counts summed by the warp), so both lists are
// the stable split of the gathered sample.
constexpr int kCompactWarps = 8;
__global__ void __launch_bounds__(32 * kCompactWarps) k_patch_compact(PatchArgs a) {
  const unsigned lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
  const u64 idx = (u64)blockIdx.x * kCompactWarps + (threadIdx.x >> 5);
  const int p = (int)(idx / (u64)a.ng), gi = (int)(idx % (u64)a.ng);
  if (p >= a.bs->n_acc) return;
  const int k = a.cand[a.n_cand + p];
  u64 x0, y0;
  patch_origin(a, k, &x0, &y0);
  unsigned before = 0;   // non-white pixels of the patch's groups before this one
  for (int g = (int)lane; g < gi; g += 32) before += (unsigned)a.gcnt[(size_t)k * a.ng + g];
  before = __reduce_add_sync(0xFFFFFFFFu, before);
  u64 onw = a.goff[p] + before;
  u64 obr = a.goff[a.n_patches + p] + (u64)gi * kPatchGroupRows * (u64)a.P - before;
  if (!SPCN_CHECK(x0 + (u64)a.P <= (u64)a.width && y0 + (u64)a.P <= (u64)a.height &&
                  onw <= a.bs->n_nw && obr <= a.bs->n_br, a.err))
    return;
  const int y1 = min(a.P, (gi + 1) * kPatchGroupRows);
  for (int y = gi * kPatchGroupRows; y < y1; ++y) {
    const uint8_t* row = a.data + (int64_t)(y0 + (u64)y) * a.pitch + (int64_t)(x0 * 3);
    for (int j0 = 0; 32 * j0 < a.P; j0 += kRowBatch) {
      uint32_t v[kRowBatch];
      unsigned have;
      load_row_batch(row, a.P, j0, lane, v, have);
#pragma unroll
      for (int j = 0; j < kRowBatch; ++j) {
        const bool in_nw = ((have >> j) & 1u) && packed_nonwhite(v[j], a.thr);
        const bool in_br = ((have >> j) & 1u) && !in_nw;
        const unsigned bn = __ballot_sync(0xFFFFFFFFu, in_nw);
        const unsigned bb = __ballot_sync(0xFFFFFFFFu, in_br);
        if (in_nw && SPCN_CHECK(onw + __popc(bn & lt) < a.bs->n_nw, a.err))
          a.nw[onw + __popc(bn & lt)] = v[j];
        if (in_br && SPCN_CHECK(obr + __popc(bb & lt) < a.bs->n_br, a.err))
          a.br[obr + __popc(bb & lt)] = v[j];
        onw += __popc(bn);
        obr += __popc(bb);
      }
    }
  }
}

// Eight blocks per kept patch (interleaved rows): copy its pixels, raster
// order, into the sample.
constexpr int kGatherSplit = 8;
__global__ void k_patch_gather(PatchArgs a) {
  const int p = blockIdx.x / kGatherSplit, part = blockIdx.x % kGatherSplit;
  if (p >= a.bs->n_acc) return;
  u64 x0, y0;
  patch_origin(a, a.cand[a.n_cand + p], &x0, &y0);
  if (!SPCN_CHECK(x0 + (u64)a.P <= (u64)a.width && y0 + (u64)a.P <= (u64)a.height &&
                  (u64)(p + 1) * (u64)a.P * (u64)a.P <= a.cap, a.err))
    return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint32_t* out = a.out + (u64)p * (u64)a.P * (u64)a.P;
  for (int y = warp * kGatherSplit + part; y < a.P; y += nwarps * kGatherSplit) {
    const uint8_t* row = a.data + (int64_t)(y0 + (u64)y) * a.pitch + (int64_t)(x0 * 3);
    for (int x = lane; x < a.P; x += 32)
      out[(u64)y * a.P + x] = (uint32_t)row[3 * x] | ((uint32_t)row[3 * x + 1] << 8) |
                              ((uint32_t)row[3 * x + 2] << 16);
  }
}

// ------------------------------------------------------------ stable compaction
struct CompactArgs {
  const uint32_t* sample;
  BasisState* bs;
  unsigned thr;
  unsigned* blk;    // [2][cap]
  u64* blk_off;     // [2][cap]
  u64 cap;
  uint32_t* nw;
  uint32_t* br;
};

__global__ void __launch_bounds__(kCompactThreads) k_classify_count(CompactArgs a) {
  __shared__ u64 s_tmp[33];
  const u64 m = a.bs->m;
  const u64 base = (u64)blockIdx.x * kCompactBlock;
  if (base >= m) return;
  unsigned cnw = 0, cbr = 0;
  for (int i = 0; i < kCompactPer; ++i) {
    const u64 e = base + (u64)threadIdx.x * kCompactPer + i;
    if (e < m) {
      const bool nw = packed_nonwhite(a.sample[e], a.thr);
      cnw += nw ? 1u : 0u;
      cbr += nw ? 0u : 1u;
    }
  }
  const u64 tnw = block_sum(cnw, s_tmp);
  const u64 tbr = block_sum(cbr, s_tmp);
  if (threadIdx.x == 0) {
    a.blk[blockIdx.x] = (unsigned)tnw;
    a.blk[a.cap + blockIdx.x] = (unsigned)tbr;
  }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(CompactArgs a) {
  __shared__ u64 s_tmp[33];
  const u64 m = a.bs->m;
  const u64 nblk = (m + kCompactBlock - 1) / kCompactBlock;
  for (int list = 0; list < 2; ++list) {
    u64 run = 0;
    for (u64 b0 = 0; b0 < nblk; b0 += blockDim.x) {
      const u64 b = b0 + threadIdx.x;
      const u64 v = b < nblk ? a.blk[list * a.cap + b] : 0ull;
      u64 total;
      const u64 ex = block_excl_scan(v, s_tmp, &total);
      if (b < nblk) a.blk_off[list * a.cap + b] = run + ex;
      run += total;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (list == 0) a.bs->n_nw = run;
      else a.bs->n_br = run;
    }
  }
}

__global__ void __launch_bounds__(kCompactThreads) k_compact(CompactArgs a) {
  __shared__ u64 s_tmp[33];
  const u64 m = a.bs->m;
  const u64 base = (u64)blockIdx.x * kCompactBlock;
  if (base >= m) return;
  uint32_t v[kCompactPer];
  unsigned fl = 0, cnw = 0, cbr = 0;
  for (int i = 0; i < kCompactPer; ++i) {
    const u64 e = base + (u64)threadIdx.x * kCompactPer + i;
    v[i] = 0;
    if (e < m) {
      v[i] = a.sample[e];
      if (packed_nonwhite(v[i], a.thr)) { fl |= 1u << i; ++cnw; }
      else { fl |= 1u << (i + 16); ++cbr; }
    }
  }
  u64 tot;
  u64 onw = block_excl_scan(cnw, s_tmp, &tot) + a.blk_off[blockIdx.x];
  u64 obr = block_excl_scan(cbr, s_tmp, &tot) + a.blk_off[a.cap + blockIdx.x];
  for (int i = 0; i < kCompactPer; ++i) {
    if (fl & (1u << i)) a.nw[onw++] = v[i];
    else if (fl & (1u << (i + 16))) a.br[obr++] = v[i];
  }
}

// ------------------------------------------------------------ i0 (§3.1 item 1)
struct I0Args {
  const uint32_t* br;
  BasisState* bs;
  Model* m;
  unsigned* hist;     // [3][256] global counts, zeroed before the launch
  unsigned* ticket;   // zeroed before the launch
  int cap;
  double pct;
  int fixed255;       // §2.1 Eq. 1's original i0 = 255 instead of the estimate
  double w0[6];       // the initial basis: column-normalised Ruifrok-Johnston H&E vectors
};

constexpr int kI0Threads = 256;
constexpr int kI0Blocks = 64;

// Per channel, the type-7 percentile of every ceil(n/cap)-th bright sample
// pixel (sample order), from 256-bin histograms (exact for 8-bit values).
// Blocks count into per-warp bins, merge into global bins, and the last block
// computes the percentiles.  Also initialises the basis to the
// column-normalised Ruifrok-Johnston H&E vectors, the starting point of the
// dictionary learning.
__global__ void __launch_bounds__(kI0Threads) k_i0(I0Args a) {
  __shared__ unsigned s_h[kI0Threads / 32][3][256];
  __shared__ unsigned s_last;
  unsigned* my = &s_h[threadIdx.x >> 5][0][0];
  for (int i = threadIdx.x; i < (kI0Threads / 32) * 768; i += blockDim.x) (&s_h[0][0][0])[i] = 0u;
  __syncthreads();
  const u64 nb = a.bs->n_br;
  const u64 stride = nb ? (nb + (u64)a.cap - 1) / (u64)a.cap : 1;
  const u64 kept = nb ? (nb + stride - 1) / stride : 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < kept; i += (u64)gridDim.x * blockDim.x) {
    const uint32_t v = a.br[i * stride];
    atomicAdd(my + (v & 0xFFu), 1u);
    atomicAdd(my + 256 + ((v >> 8) & 0xFFu), 1u);
    atomicAdd(my + 512 + ((v >> 16) & 0xFFu), 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 768; i += blockDim.x) {
    unsigned t = 0;
    for (int w = 0; w < kI0Threads / 32; ++w) t += (&s_h[w][0][0])[i];
    if (t) atomicAdd(a.hist + i, t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: thread v holds bin v of each channel; a block scan gives
  // every bin's cumulative count, and the thread whose bin holds rank k (and
  // k + 1) of a channel records its value
  __shared__ unsigned s_wt[3][kI0Threads / 32];
  __shared__ int s_rv[3][2];
  const int v = threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double pos = kept > 0 ? (double)(kept - 1) * (a.pct / 100.0) : 0.0;
  u64 k = (u64)floor(pos);
  if (kept > 0 && k > kept - 1) k = kept - 1;
  unsigned cnt[3], incl[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cnt[c] = __ldcg(a.hist + 256 * c + v);
    unsigned x = cnt[c];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    incl[c] = x;
    if (lane == 31) s_wt[c][warp] = x;
  }
  if (v < 6) s_rv[v / 2][v % 2] = 255;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u64 before = 0;
    for (int w = 0; w < warp; ++w) before += s_wt[c][w];
    const u64 hi = before + incl[c], lo = hi - cnt[c];
    for (int j = 0; j < 2; ++j) {
      const u64 r = k + (u64)j;
      if (cnt[c] > 0 && lo <= r && r < hi) s_rv[c][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int c = threadIdx.x;
    double val = 255.0;
    if (kept > 0 && !a.fixed255) {
      const double t = pos - (double)k;
      const double lo = (double)s_rv[c][0];
      const double hi = (k + 1 < kept) ? (double)s_rv[c][1] : lo;
      val = (k + 1 < kept) ? __dadd_rn(lo, __dmul_rn(t, __dsub_rn(hi, lo))) : lo;
    }
    a.m->i0[c] = (float)val;
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {   // static indices: the parameter stays in parameter space
      a.bs->W[i] = a.w0[i];
      a.m->W[i] = (float)a.w0[i];
    }
  }
}

// ------------------------------------------------------------ sparse NMF (Eq. 2)
struct SnmfArgs {
  const uint32_t* nw;
  BasisState* bs;
  Model* m;
  unsigned long long* tot;   // [3][kAcc] fixed-point totals, zeroed before the launch
  unsigned* bar;
  int* abort;
  int* err;
  float lambda;
  int max_iter;
  double tol;
  long long timeout_ns;
  int order_blue;     // the original ordering heuristic (larger blue OD is hematoxylin)
};

// Reduced sums, in this order: A11 A12 A22 | B[R,0] B[R,1] B[G,0] B[G,1]
// B[B,0] B[B,1] | sum h1, sum h2 | sum |v|^2.
// The W update runs on one thread per block after the grid barrier, so its
// dependent chain is on the critical path of every iteration; it runs in
// FP32 from the FP64 totals (FP64 operations are slow and long in latency on
// this GPU).

__global__ void __launch_bounds__(kSnmfThreads) k_snmf(SnmfArgs a) {
  __shared__ float s_od[kLutEntries];
  __shared__ float s_W[6];
  __shared__ double s_tot[kAcc];
  __shared__ float s_coef[12];
  __shared__ float s_red[kSnmfThreads / 32][kAcc];
  __shared__ int s_shift;      // fixed-point scale of this iteration's sums
  __shared__ int s_flag;
  __shared__ double s_obj;
  __shared__ float s_Wp[6];    // the basis the last H-step used (for the objective)
  __shared__ int s_have;
  const u64 n = a.bs->n_nw;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.bs->status = SPCN_ERR_NO_TISSUE;
    return;   // uniform
  }
  for (int i = threadIdx.x; i < kLutEntries; i += blockDim.x) s_od[i] = a.m->od[i];
  if (threadIdx.x < 6) s_W[threadIdx.x] = (float)a.bs->W[threadIdx.x];
  if (threadIdx.x == 0) { s_flag = 0; s_obj = 0.0; s_have = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 gstride = (u64)gridDim.x * blockDim.x;
  unsigned target = 0;
  int it;
  // closed-form H-step coefficients of the current basis (thread 0); -1 in
  // s_flag when the basis is degenerate.  FP32 throughout (the coefficients
  // are FP32 anyway); the determinant g11 g22 - g12^2 takes the rounding
  // error of g12^2 back with an FMA, so it stays accurate when the two
  // columns are nearly parallel (exactly 0 for equal columns)
  auto set_coef = [&]() {
    float g11 = 0.f, g22 = 0.f, g12 = 0.f;
    for (int c = 0; c < 3; ++c) {
      g11 = fmaf(s_W[c], s_W[c], g11);
      g22 = fmaf(s_W[3 + c], s_W[3 + c], g22);
      g12 = fmaf(s_W[c], s_W[3 + c], g12);
    }
    const float q = g12 * g12;
    const float det = fmaf(g11, g22, -q) - fmaf(g12, g12, -q);
    if (!(det > 1e-12f)) {
      s_flag = -1;
    } else {
      const float id = 1.f / det;
      for (int i = 0; i < 6; ++i) s_coef[i] = s_W[i];
      s_coef[6] = g22 * id;
      s_coef[7] = -g12 * id;
      s_coef[8] = -g12 * id;
      s_coef[9] = g11 * id;
      s_coef[10] = 1.f / g11;
      s_coef[11] = 1.f / g22;
      // per-pixel bound of the summands: |v_c| <= log 256, and an H-step
      // density is at most (1/g_jj) log 256 sum_c w_cj (W >= 0)
      const float vmax = 5.5452f;
      float hb = 0.f;
      for (int j = 0; j < 2; ++j) {
        const float l1 = fabsf(s_W[3 * j]) + fabsf(s_W[3 * j + 1]) + fabsf(s_W[3 * j + 2]);
        hb = fmaxf(hb, s_coef[10 + j] * vmax * l1);
      }
      const float per = fmaxf(fmaxf(hb * hb, vmax * hb), fmaxf(hb, 3.f * vmax * vmax));
      const float bound = (float)n * per * 1.0001f + 1.f;
      int e = 128;                   // a bound beyond FP32 (a near-singular basis)
      if (bound < 3.0e38f) frexpf(bound, &e);   // every |total| < 2^e
      s_shift = max(61 - e, -120);   // 2^s_shift stays a normal FP32 number
    }
  };
  if (threadIdx.x == 0) set_coef();
  __syncthreads();
  for (it = 1; it <= a.max_iter; ++it) {
    if (s_flag < 0) break;
    const float w00 = s_coef[0], w10 = s_coef[1], w20 = s_coef[2];
    const float w01 = s_coef[3], w11 = s_coef[4], w21 = s_coef[5];
    const float a11 = s_coef[6], a12 = s_coef[7], a21 = s_coef[8], a22 = s_coef[9];
    const float u1 = s_coef[10], u2 = s_coef[11];
    float acc[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) acc[i] = 0.f;
    auto step = [&](uint32_t v) {
      const float v0 = s_od[v & 0xFFu], v1 = s_od[256 + ((v >> 8) & 0xFFu)],
                  v2 = s_od[512 + ((v >> 16) & 0xFFu)];
      const float d1 = fmaf(w20, v2, fmaf(w10, v1, w00 * v0)) - a.lambda;
      const float d2 = fmaf(w21, v2, fmaf(w11, v1, w01 * v0)) - a.lambda;
      const float t1 = fmaf(a12, fmaxf(d2, 0.f), a11 * d1);
      const float t2 = fmaf(a21, fmaxf(d1, 0.f), a22 * d2);
      const float h1 = fmaxf(0.f, fminf(u1 * d1, t1));
      const float h2 = fmaxf(0.f, fminf(u2 * d2, t2));
      acc[0] = fmaf(h1, h1, acc[0]);
      acc[1] = fmaf(h1, h2, acc[1]);
      acc[2] = fmaf(h2, h2, acc[2]);
      acc[3] = fmaf(v0, h1, acc[3]);
      acc[4] = fmaf(v0, h2, acc[4]);
      acc[5] = fmaf(v1, h1, acc[5]);
      acc[6] = fmaf(v1, h2, acc[6]);
      acc[7] = fmaf(v2, h1, acc[7]);
      acc[8] = fmaf(v2, h2, acc[8]);
      acc[9] += h1;
      acc[10] += h2;
      acc[11] = fmaf(v0, v0, fmaf(v1, v1, fmaf(v2, v2, acc[11])));
    };
    // Two pixels per packed FP32x2 instruction: each lane rounds exactly as
    // the scalar step does; the lanes accumulate apart and are added at the end.
    const f2 W00 = pk(w00, w00), W10 = pk(w10, w10), W20 = pk(w20, w20);
    const f2 W01 = pk(w01, w01), W11 = pk(w11, w11), W21 = pk(w21, w21);
    const f2 A11 = pk(a11, a11), A12 = pk(a12, a12), A21 = pk(a21, a21), A22 = pk(a22, a22);
    const f2 U1 = pk(u1, u1), U2 = pk(u2, u2), NL = pk(-a.lambda, -a.lambda);
    f2 pacc[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) pacc[i] = 0ull;
    auto step2 = [&](uint32_t v, uint32_t u) {
      const f2 V0 = pk(s_od[v & 0xFFu], s_od[u & 0xFFu]);
      const f2 V1 = pk(s_od[256 + ((v >> 8) & 0xFFu)], s_od[256 + ((u >> 8) & 0xFFu)]);
      const f2 V2 = pk(s_od[512 + ((v >> 16) & 0xFFu)], s_od[512 + ((u >> 16) & 0xFFu)]);
      const f2 D1 = add2(fma2(W20, V2, fma2(W10, V1, mul2(W00, V0))), NL);
      const f2 D2 = add2(fma2(W21, V2, fma2(W11, V1, mul2(W01, V0))), NL);
      const f2 T1 = fma2(A12, pk(fmaxf(lo_of(D2), 0.f), fmaxf(hi_of(D2), 0.f)), mul2(A11, D1));
      const f2 T2 = fma2(A21, pk(fmaxf(lo_of(D1), 0.f), fmaxf(hi_of(D1), 0.f)), mul2(A22, D2));
      const f2 X1 = mul2(U1, D1), X2 = mul2(U2, D2);
      const f2 H1 = pk(fmaxf(0.f, fminf(lo_of(X1), lo_of(T1))), fmaxf(0.f, fminf(hi_of(X1), hi_of(T1))));
      const f2 H2 = pk(fmaxf(0.f, fminf(lo_of(X2), lo_of(T2))), fmaxf(0.f, fminf(hi_of(X2), hi_of(T2))));
      pacc[0] = fma2(H1, H1, pacc[0]);
      pacc[1] = fma2(H1, H2, pacc[1]);
      pacc[2] = fma2(H2, H2, pacc[2]);
      pacc[3] = fma2(V0, H1, pacc[3]);
      pacc[4] = fma2(V0, H2, pacc[4]);
      pacc[5] = fma2(V1, H1, pacc[5]);
      pacc[6] = fma2(V1, H2, pacc[6]);
      pacc[7] = fma2(V2, H1, pacc[7]);
      pacc[8] = fma2(V2, H2, pacc[8]);
      pacc[9] = add2(pacc[9], H1);
      pacc[10] = add2(pacc[10], H2);
      pacc[11] = fma2(V0, V0, fma2(V1, V1, fma2(V2, V2, pacc[11])));
    };
    // four pixels per 16-byte load (the list is 16-byte aligned), then the tail
    const uint4* nw4 = reinterpret_cast<const uint4*>(a.nw);
    const u64 n4 = n >> 2;
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + gstride < n4; i += 2 * gstride) {   // two loads in flight
      const uint4 v = __ldg(nw4 + i), u = __ldg(nw4 + i + gstride);
      step2(v.x, v.y);
      step2(v.z, v.w);
      step2(u.x, u.y);
      step2(u.z, u.w);
    }
    if (i < n4) {
      const uint4 v = __ldg(nw4 + i);
      step2(v.x, v.y);
      step2(v.z, v.w);
    }
#pragma unroll
    for (int i = 0; i < kAcc; ++i) acc[i] = lo_of(pacc[i]) + hi_of(pacc[i]);
    for (u64 i = (n4 << 2) + (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gstride)
      step(__ldg(a.nw + i));
    // warp sums in FP32 (a fixed shuffle tree), then fixed point: each warp
    // sum times 2^s_shift rounded to a 64-bit integer, added exactly over the
    // block and, with one atomic per sum and block, over the grid.  Integer
    // sums do not depend on the order, so every block reads the same totals
    // and reruns are bitwise equal; s_shift leaves the largest total the
    // basis allows below 2^61, and the rounding (2^-s_shift per warp) is far
    // below the FP32 warp sums' own
#pragma unroll
    for (int i = 0; i < kAcc; ++i) {
      float x = acc[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) s_red[warp][i] = x;
    }
    __syncthreads();
    unsigned long long* tot = a.tot + (size_t)(it % 3) * kAcc;
    if (threadIdx.x < kAcc) {
      // x 2^s is exact in FP32 (a power of two), then rounded to an integer
      const float sc = ldexpf(1.f, s_shift);
      long long v = 0;
#pragma unroll
      for (int w = 0; w < kSnmfThreads / 32; ++w) v += __float2ll_rn(s_red[w][threadIdx.x] * sc);
      atomicAdd(tot + threadIdx.x, (unsigned long long)v);
    }
    target += gridDim.x;
    if (!grid_barrier(a.bar, target, a.abort, a.err, a.timeout_ns)) return;
    if (threadIdx.x < kAcc) {
      s_tot[threadIdx.x] = (double)(long long)__ldcg(tot + threadIdx.x) * ldexp(1.0, -s_shift);
      // the buffer of iteration it + 2, read by every block before this barrier
      if (blockIdx.x == 0) a.tot[(size_t)((it + 2) % 3) * kAcc + threadIdx.x] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // The column update in FP32 from the FP64 totals: at the totals'
      // magnitude its rounding moves W by about 1e-7, far inside the
      // convergence tolerance and the 1e-5 agreement with the FP64 oracle,
      // while this serial step runs on one thread of every block and FP64
      // operations are slow and long in latency on this GPU.
      const float A[2][2] = {{(float)s_tot[0], (float)s_tot[1]}, {(float)s_tot[1], (float)s_tot[2]}};
      float B[3][2];
      for (int c = 0; c < 3; ++c) {
        B[c][0] = (float)s_tot[3 + 2 * c];
        B[c][1] = (float)s_tot[4 + 2 * c];
      }
      float W[3][2], Wp[3][2];
      for (int c = 0; c < 3; ++c) { W[c][0] = Wp[c][0] = s_W[c]; W[c][1] = Wp[c][1] = s_W[3 + c]; }
      for (int i = 0; i < 6; ++i) s_Wp[i] = s_W[i];   // objective taken at the end
      s_have = 1;
      int flag = 0;
      for (int j = 0; j < 2 && flag == 0; ++j) {
        if (!(A[j][j] > 0.f)) continue;
        const float iA = 1.f / A[j][j];
        float u[3], nu = 0.f;
        for (int c = 0; c < 3; ++c) {
          u[c] = fmaf(B[c][j] - fmaf(W[c][0], A[0][j], W[c][1] * A[1][j]), iA, W[c][j]);
          u[c] = u[c] > 0.f ? u[c] : 0.f;
          nu = fmaf(u[c], u[c], nu);
        }
        if (!(nu > 0.f)) { flag = -1; break; }
        const float r = 1.f / sqrtf(nu);
        for (int c = 0; c < 3; ++c) W[c][j] = u[c] * r;
      }
      float dmax = 0.f;
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 2; ++j) dmax = fmaxf(dmax, fabsf(W[c][j] - Wp[c][j]));
      for (int c = 0; c < 3; ++c) { s_W[c] = W[c][0]; s_W[3 + c] = W[c][1]; }
      if (flag == 0 && (double)dmax < a.tol) flag = 1;
      s_flag = flag;
      if (flag == 0) set_coef();   // the next iteration's coefficients
    }
    __syncthreads();
    if (s_flag != 0) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (s_have) {   // objective of the last H-step taken (1/2-scaled Eq. 2)
      double g11 = 0, g22 = 0, g12 = 0, wb = 0;
      for (int c = 0; c < 3; ++c) {
        g11 += s_Wp[c] * s_Wp[c];
        g22 += s_Wp[3 + c] * s_Wp[3 + c];
        g12 += s_Wp[c] * s_Wp[3 + c];
        wb += s_Wp[c] * s_tot[3 + 2 * c] + s_Wp[3 + c] * s_tot[4 + 2 * c];
      }
      s_obj = 0.5 * s_tot[11] - wb +
              0.5 * (g11 * s_tot[0] + 2.0 * g12 * s_tot[1] + g22 * s_tot[2]) +
              (double)a.lambda * (s_tot[9] + s_tot[10]);
    }
    int status = SPCN_OK;
    double g11 = 0, g22 = 0, g12 = 0;
    for (int c = 0; c < 3; ++c) {
      g11 += s_W[c] * s_W[c];
      g22 += s_W[3 + c] * s_W[3 + c];
      g12 += s_W[c] * s_W[3 + c];
    }
    if (s_flag < 0 || !(g11 * g22 - g12 * g12 > 1e-12)) status = SPCN_ERR_DEGENERATE_BASIS;
    // §3.1 item 3: hematoxylin is the stain with the larger OD(red) - OD(blue);
    // the original heuristic compares the blue OD alone
    const double d0 = a.order_blue ? s_W[2] : s_W[0] - s_W[2];
    const double d1 = a.order_blue ? s_W[5] : s_W[3] - s_W[5];
    double Wo[6];
    for (int c = 0; c < 3; ++c) {
      Wo[c] = d1 > d0 ? s_W[3 + c] : s_W[c];
      Wo[3 + c] = d1 > d0 ? s_W[c] : s_W[3 + c];
    }
    for (int i = 0; i < 6; ++i) { a.bs->W[i] = Wo[i]; a.m->W[i] = (float)Wo[i]; }
    a.bs->iters = it > a.max_iter ? a.max_iter : it;
    a.bs->objective = s_obj;
    a.bs->status = status;
  }
}

// ------------------------------------------------------------ median of per-patch percentiles
// §3.2 item 4 (SPCN_FLAG_P99_PATCH_MEDIAN): for every kept patch the exact
// type-7 percentile of each stain's density over the patch's non-white
// pixels, then per stain the median (type-7 50th percentile) of those values
// over the patches.  The non-white list is the stable compaction of the
// sample, which holds the kept patches one after another, so patch p's
// non-white pixels are one segment of it, placed by the candidates' counts.
constexpr int kPatchSelThreads = 1024;
constexpr int kPatchSelBins = 2048;   // 11/11/10-bit digits of the FP32 key
constexpr size_t kPatchSelSmem = kLutSmemBytes + sizeof(unsigned) * 4 * kPatchSelBins;
constexpr int kMaxMedianPatches = 4096;

struct PatchP99Args {
  const uint32_t* nw;
  const int* cand;     // [n_cand] non-white counts, then the accepted candidates
  int n_cand;
  const BasisState* bs;
  const Model* m;
  double pct;
  double* per_patch;   // [n_acc][2]
};

// The bin of a shared 2048-bin histogram that holds rank r (-1 if none) and
// the count before it.  Whole block.
__device__ void shared_rank_bin(const unsigned* h, u64 r, int* s_idx, u64* s_before,
                                u64* s_tmp) {
  const int per = (kPatchSelBins + (int)blockDim.x - 1) / (int)blockDim.x;
  const int beg = threadIdx.x * per, end = min(kPatchSelBins, beg + per);
  u64 local = 0;
  for (int i = beg; i < end; ++i) local += h[i];
  u64 total;
  const u64 excl = block_excl_scan(local, s_tmp, &total);
  if (threadIdx.x == 0) *s_idx = -1;
  __syncthreads();
  if (local > 0 && excl <= r && r < excl + local) {
    u64 c = excl;
    for (int i = beg; i < end; ++i) {
      if (r < c + h[i]) { *s_idx = i; *s_before = c; break; }
      c += h[i];
    }
  }
  __syncthreads();
}

// One block per kept patch: radix select (11/11/10-bit digits of the FP32
// key of the scaled density; order-preserving signed keys for the
// pseudo-inverse) of ranks k and k+1 of both stains over the patch's segment
// of the non-white list.
template <bool PINV>
__global__ void __launch_bounds__(kPatchSelThreads, 1) k_patch_p99(PatchP99Args a) {
  extern __shared__ __align__(16) char s_dyn[];
  unsigned* s_hist = reinterpret_cast<unsigned*>(s_dyn + kLutSmemBytes);   // [4][bins]
  __shared__ u64 s_tmp[33];
  __shared__ unsigned s_pre[4];
  __shared__ u64 s_r[4];
  __shared__ int s_idx;
  __shared__ u64 s_before;
  const int p = blockIdx.x;
  if (p >= a.bs->n_acc || a.bs->status != SPCN_OK || a.m->status != SPCN_OK) return;   // uniform
  u64 part = 0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) part += (u64)a.cand[a.cand[a.n_cand + i]];
  const u64 off = block_sum(part, s_tmp);
  const u64 n = (u64)a.cand[a.cand[a.n_cand + p]];   // >= 1: a kept patch is half non-white
  u64 k, k1;
  double t;
  type7_ranks(n, a.pct, &k, &k1, &t);
  if (threadIdx.x < 4) {
    s_pre[threadIdx.x] = 0u;
    s_r[threadIdx.x] = (threadIdx.x & 1) ? k1 : k;
  }
  load_lut(a.m, s_dyn);
  const char* lut = s_dyn;
  const unsigned lr = lane_reg();
  const Lasso L = a.m->lasso;
  const uint32_t* items = a.nw + off;
  for (int d = 0; d < 3; ++d) {
    const int shift = d == 0 ? 21 : (d == 1 ? 10 : 0);
    const int hi = d == 0 ? 32 : (d == 1 ? 21 : 10);
    const unsigned mask = d == 2 ? 0x3FFu : 0x7FFu;
    for (int i = threadIdx.x; i < 4 * kPatchSelBins; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    unsigned pre[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) pre[q] = s_pre[q];
    for (u64 i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t v = __ldg(items + i);
      float h1, h2;
      solve_one<PINV>(lut, lut_addr(v, lr, 0), lut_addr(v, lr, 1), lut_addr(v, lr, 2), L, h1, h2);
      const unsigned key[2] = {PINV ? signed_key(__float_as_uint(h1)) : __float_as_uint(h1),
                               PINV ? signed_key(__float_as_uint(h2)) : __float_as_uint(h2)};
      const unsigned live = __activemask();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned kk = key[q >> 1];
        const bool in = ((u64)kk >> hi) == ((u64)pre[q] >> hi);
        // warp-aggregated increment: one shared atomic per distinct bin
        const unsigned bin = in ? ((kk >> shift) & mask) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(live, bin);
        if (in && (__ffs(peers) - 1) == (int)(threadIdx.x & 31u))
          atomicAdd(s_hist + q * kPatchSelBins + bin, (unsigned)__popc(peers));
      }
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      shared_rank_bin(s_hist + q * kPatchSelBins, s_r[q], &s_idx, &s_before, s_tmp);
      if (threadIdx.x == 0 && s_idx >= 0) {
        s_pre[q] |= (unsigned)s_idx << shift;
        s_r[q] -= s_before;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < 2) {
    const int j = threadIdx.x;
    const unsigned ka = PINV ? signed_key_inv(s_pre[2 * j]) : s_pre[2 * j];
    const unsigned kb = PINV ? signed_key_inv(s_pre[2 * j + 1]) : s_pre[2 * j + 1];
    a.per_patch[2 * p + j] = interp_type7(__fmul_rn(__uint_as_float(ka), L.hscale),
                                          __fmul_rn(__uint_as_float(kb), L.hscale), t);
  }
}

// Per stain, the type-7 50th percentile of the per-patch values, written as
// the reported sample percentile: one block sorts them (bitonic, in shared
// memory; at most 4096 patches).
__global__ void __launch_bounds__(1024) k_patch_median(const double* per_patch, BasisState* bs,
                                                       const Model* m) {
  __shared__ double s_v[kMaxMedianPatches];
  const int n = bs->n_acc;
  if (n <= 0 || n > kMaxMedianPatches || bs->status != SPCN_OK || m->status != SPCN_OK) return;
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int j = 0; j < 2; ++j) {
    for (int i = threadIdx.x; i < np2; i += blockDim.x)
      s_v[i] = i < n ? per_patch[2 * i + j] : __longlong_as_double(0x7FF0000000000000ll);
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < np2; i += blockDim.x) {
          const int o = i ^ stride;
          if (o > i) {
            const bool up = (i & size) == 0;
            const double x = s_v[i], y = s_v[o];
            if ((x > y) == up) { s_v[i] = y; s_v[o] = x; }
          }
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) {
      const double pos = (double)(n - 1) * 0.5;
      const int k = (int)floor(pos);
      const int k1 = k + 1 <= n - 1 ? k + 1 : k;
      const double t = pos - (double)k;
      const double lo = s_v[k], hi = s_v[k1];
      bs->sel.p99[j] = __dadd_rn(lo, __dmul_rn(t, __dsub_rn(hi, lo)));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ host driver
static int grid_for(const Context* c, int occ) { return c->num_sms * (occ > 0 ? occ : 1); }

int configure_basis_kernels(Context* c) {
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_snmf, k_snmf,
                                                              kSnmfThreads, 0));
  if (c->occ_snmf < 1) return SPCN_ERR_CUDA;
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_patch_p99<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPatchSelSmem));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_patch_p99<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPatchSelSmem));
  if (grid_for(c, c->occ_snmf) > kMaxSnmfGrid) c->occ_snmf = kMaxSnmfGrid / c->num_sms;
  return SPCN_OK;
}

// Every launch of a basis estimation (sampling, i0, sparse NMF, stain order,
// sample percentile) on `st`, without waiting: the results stay on the
// device (c->bs, c->model_b) until finish_estimate_basis reads them.
int launch_estimate_basis(Context* c, const spcn_image* img, const spcn_params* p,
                          cudaStream_t st, bool hint_only) {
  const int64_t W = img->width, H = img->height;
  const u64 N = (u64)W * (u64)H;
  u64 cap = 0, m = 0;
  int n_cand = 0;
  if (p->sample_mode == SPCN_SAMPLE_ALL) {
    cap = m = N;
  } else if (p->sample_mode == SPCN_SAMPLE_HASH) {
    m = (u64)floor((double)p->sample_rate * (double)N + 0.5);
    if (m == 0) return SPCN_ERR_INVALID_ARG;
    cap = m;
  } else {
    if (p->patch_size > W || p->patch_size > H) return SPCN_ERR_INVALID_ARG;
    cap = (u64)p->n_patches * (u64)p->patch_size * (u64)p->patch_size;
    n_cand = 4 * p->n_patches;
  }
  int rc = ensure_sample_capacity(c, (size_t)cap);
  if (rc) return rc;
  if (n_cand) { rc = ensure_candidate_capacity(c, n_cand + p->n_patches); if (rc) return rc; }

  BasisState* bs = c->bs;
  bool per_patch = false;   // patch sampling compacted patch by patch (below)
  SPCN_CUDA_TRY(cudaMemsetAsync(bs, 0, sizeof(BasisState), st));
  const int big_grid = c->num_sms * 8;
  if (p->sample_mode != SPCN_SAMPLE_PATCHES) {
    SampleArgs s{img->data, img->pitch_bytes, W, H, p->seed, c->sample, m, (u64)c->sample_cap,
                 c->err, &bs->m};
    if (p->sample_mode == SPCN_SAMPLE_ALL) k_sample_all<<<big_grid, 256, 0, st>>>(s);
    else k_sample_hash<<<big_grid, 256, 0, st>>>(s);
    SPCN_LAUNCH_CHECK(c);
  } else {
    PatchArgs pa{img->data, img->pitch_bytes, W, H, p->seed, p->patch_size, p->n_patches,
                 n_cand, (unsigned)p->white_thresh, c->cand, bs, c->sample, (u64)c->sample_cap,
                 c->err, 0, nullptr, nullptr, c->nw, c->br};
    // Per-patch compaction: the kept patches' row groups go straight into
    // the two lists, so the whole sample is never written.  Its buffer (n
    // patches of P^2 entries) holds the patch offsets and the group counts
    // instead (4 n + 4 n ceil(P/4) 32-bit words, which fit for P >= 3).
    const int ng = (p->patch_size + kPatchGroupRows - 1) / kPatchGroupRows;
    const u64 words = 4ull * (u64)p->n_patches * (1ull + (u64)ng);
    per_patch = words <= cap;
    if (per_patch) {
      pa.ng = ng;
      pa.goff = reinterpret_cast<u64*>(c->sample);
      pa.gcnt = reinterpret_cast<int*>(c->sample + 4ull * (u64)p->n_patches);
    }
    k_patch_count<<<n_cand, 256, 0, st>>>(pa);
    SPCN_LAUNCH_CHECK(c);
    k_patch_accept<<<1, kAcceptThreads, 0, st>>>(pa);
    SPCN_LAUNCH_CHECK(c);
    if (per_patch) {
      const u64 groups = (u64)p->n_patches * (u64)ng;
      k_patch_compact<<<(unsigned)((groups + kCompactWarps - 1) / kCompactWarps), 32 * kCompactWarps,
                        0, st>>>(pa);
      SPCN_LAUNCH_CHECK(c);
    } else {
      k_patch_gather<<<p->n_patches * kGatherSplit, 256, 0, st>>>(pa);
      SPCN_LAUNCH_CHECK(c);
    }
  }
  if (!per_patch) {
    const u64 nblk = (cap + kCompactBlock - 1) / kCompactBlock;
    CompactArgs ca{c->sample, bs, (unsigned)p->white_thresh, c->blk, c->blk_off,
                   (u64)c->blk_cap, c->nw, c->br};
    k_classify_count<<<(unsigned)nblk, kCompactThreads, 0, st>>>(ca);
    SPCN_LAUNCH_CHECK(c);
    k_scan_blocks<<<1, 1024, 0, st>>>(ca);
    SPCN_LAUNCH_CHECK(c);
    k_compact<<<(unsigned)nblk, kCompactThreads, 0, st>>>(ca);
    SPCN_LAUNCH_CHECK(c);
  }
  SPCN_CUDA_TRY(cudaMemsetAsync(bs->i0_hist, 0, sizeof(bs->i0_hist) + sizeof(bs->i0_ticket), st));
  I0Args ia{c->br, bs, c->model_b, bs->i0_hist, &bs->i0_ticket, p->i0_max_samples,
            (double)p->i0_pct, (p->flags & SPCN_FLAG_I0_255) ? 1 : 0, {}};
  {   // §3.1: the Ruifrok-Johnston H&E vectors, each normalised to unit length
    const double h[3] = {0.650, 0.704, 0.286}, e[3] = {0.072, 0.990, 0.105};
    const double nh = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    const double ne = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    for (int c = 0; c < 3; ++c) {
      ia.w0[c] = h[c] / nh;
      ia.w0[3 + c] = e[c] / ne;
    }
  }
  k_i0<<<kI0Blocks, kI0Threads, 0, st>>>(ia);
  SPCN_LAUNCH_CHECK(c);
  rc = launch_build_model(c, c->model_b, nullptr, nullptr, p->lambda, c->model_b, st);
  if (rc) return rc;
  // sparse NMF, one cooperative launch
  SnmfArgs sa;
  sa.nw = c->nw;
  sa.bs = bs;
  sa.m = c->model_b;
  sa.tot = reinterpret_cast<unsigned long long*>(c->partials);
  SPCN_CUDA_TRY(cudaMemsetAsync(sa.tot, 0, sizeof(unsigned long long) * 3 * kAcc, st));
  sa.bar = &c->sel->barrier;
  sa.abort = &c->sel->abort;
  sa.err = c->err;
  sa.lambda = p->lambda;
  sa.max_iter = p->max_iter;
  sa.tol = (double)p->tol;
  sa.timeout_ns = c->timeout_ns;
  sa.order_blue = (p->flags & SPCN_FLAG_ORDER_BLUE) ? 1 : 0;
  SPCN_CUDA_TRY(cudaMemsetAsync(c->sel, 0, sizeof(SelectState), st));
  void* args[] = {&sa};
  SPCN_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_snmf, grid_for(c, c->occ_snmf), kSnmfThreads,
                                            args, 0, st));
  c->launches++;
  // the final table: the learnt basis, and the densities that are scaled
  const bool pinv = (p->flags & SPCN_FLAG_H_PINV) != 0;
  rc = launch_build_model(c, c->model_b, nullptr, nullptr, p->lambda, c->model_b, st, pinv);
  if (rc) return rc;
  if (p->flags & SPCN_FLAG_P99_PATCH_MEDIAN) {   // patches sampling (checked by the caller)
    SPCN_CUDA_TRY(cudaMemsetAsync(&bs->sel, 0, sizeof(SelectState), st));
    PatchP99Args pp{c->nw, c->cand, n_cand, bs, c->model_b, (double)p->stain_pct, c->partials};
    if (pinv)
      k_patch_p99<true><<<p->n_patches, kPatchSelThreads, kPatchSelSmem, st>>>(pp);
    else
      k_patch_p99<false><<<p->n_patches, kPatchSelThreads, kPatchSelSmem, st>>>(pp);
    SPCN_LAUNCH_CHECK(c);
    k_patch_median<<<1, 1024, 0, st>>>(c->partials, bs, c->model_b);
    SPCN_LAUNCH_CHECK(c);
    return SPCN_OK;
  }
  // hint_only: the sample only places the search window of an exact
  // whole-image percentile (a binomial band around the percentile); a
  // regular sub-sample (at most every 16th group of four sample pixels, at
  // least 2^18 of them) suffices
  return launch_select_list(c, c->nw, &bs->n_nw, c->model_b, &bs->sel, c->rhist_b,
                            (double)p->stain_pct, st, pinv, hint_only ? 16u : 1u, hint_only,
                            p->sample_mode == SPCN_SAMPLE_PATCHES ? &bs->n_acc : nullptr);
}

// Wait for the estimation launched on `st` and fill the host record.
int finish_estimate_basis(Context* c, spcn_stats* out, cudaStream_t st) {
  BasisState* bs = c->bs;
  BasisState h;
  Model hm;
  int herr = 0;
  SPCN_CUDA_TRY(cudaMemcpyAsync(&h, bs, sizeof(BasisState), cudaMemcpyDeviceToHost, st));
  SPCN_CUDA_TRY(cudaMemcpyAsync(&hm.W, &c->model_b->W, sizeof(hm.W) + sizeof(hm.i0),
                                cudaMemcpyDeviceToHost, st));
  SPCN_CUDA_TRY(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPCN_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < 6; ++i) out->W[i] = hm.W[i];
  for (int i = 0; i < 3; ++i) out->i0[i] = hm.i0[i];
  out->p99[0] = h.sel.p99[0];
  out->p99[1] = h.sel.p99[1];
  out->iters = h.iters;
  out->n_sample = (int64_t)h.m;
  out->n_nonwhite = (int64_t)h.n_nw;
  out->n_bright = (int64_t)h.n_br;
  out->objective = h.objective;
  int status = h.status;
  if (status == SPCN_OK && herr != 0) status = herr;
  if (status == SPCN_OK && h.n_nw == 0) status = SPCN_ERR_NO_TISSUE;
  out->status = status;
  if (herr != 0) SPCN_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), st));
  return status;
}

int run_estimate_basis(Context* c, const spcn_image* img, const spcn_params* p, spcn_stats* out,
                       cudaStream_t st) {
  const int rc = launch_estimate_basis(c, img, p, st);
  if (rc) return rc;
  return finish_estimate_basis(c, out, st);
}

}  // namespace spcn
