// Batched normalisation: many tiles, each with its own source statistics,
// normalised to one target in one cooperative persistent launch (the batch
// form of §3.2, "sources normalised to one target").  Per tile the launch
// computes exactly what the single-image path computes (Eq. 1-4 with the
// exact non-white P99 of Eq. 3): the same tables, the same closed-form H-step,
// the same keys and the same reconstruction, so every output byte and every
// percentile equals that of spcn_normalize on the tile alone.
//
// Schedule.  The launch works through one queue of work items (a range of a
// tile's 16-pixel chunks and a pass), claimed with an atomic ticket:
//   pass-1 item  densities of every pixel, non-white and below-window counts,
//                and the FP32 keys at or above the tile's window start,
//                appended to the tile's key lists (per-warp shared-memory
//                buffers, flushed with one atomic reservation each);
//   tile select  the block finishing a tile's last pass-1 item selects the
//                wanted ranks from the key lists (radix select with 12-bit
//                digits over key - start) and publishes the scale factors;
//   pass-2 item  waits (bounded) for its tile's scale, then reconstructs.
// Every pass-1 item of a tile precedes its pass-2 items in the queue, so the
// waits end without any grid-wide barrier.
//
// Window.  Tiles of one slide share the slide's statistics, but each tile's
// own P99 differs from the slide's by up to about +-25% (tissue content varies
// from tile to tile), so a narrow two-sided window around the hint misses
// often.  The window here is open-ended: [lo, +inf), where lo comes from a
// pilot sample of the tile itself (k_batch_pilot, launched before the batch
// kernel), or is kOpenLow * hint when the sample is too small.  Only ranks
// whose density lies below the window start (or a list that overflowed)
// leave a tile to the exact radix select over its pixels, run by the whole
// grid after the queue, followed by the tile's pass 2.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "spcn_context.h"
#include "spcn_internal.cuh"
#include "spcn_pixel.cuh"

namespace spcn {

#ifndef SPCN_BATCH_THREADS
#define SPCN_BATCH_THREADS 1024
#endif
constexpr int kBatchThreads = SPCN_BATCH_THREADS;   // one block per SM (shared memory)
constexpr int kKeyBuf = 128;       // keys per stain buffered per warp before a flush
constexpr int kSelBits = 12;       // digit width of the in-list select
constexpr int kSelBins = 1 << kSelBits;
constexpr double kOpenLow = 0.75;  // window start, relative to the hint
constexpr int kWarps = kBatchThreads / 32;
constexpr size_t kBatchQueueBytes = sizeof(uint2) * kWarpQueue * kWarps;
constexpr size_t cmax(size_t x, size_t y) { return x > y ? x : y; }
// per-warp queues and key buffers (pass 1), overlaid by the select and the
// fallback's radix histograms
constexpr size_t kBatchWork = cmax(kBatchQueueBytes + sizeof(unsigned) * 2 * kKeyBuf * kWarps,
                                   cmax(sizeof(unsigned) * kTracks * kRadixBins,
                                        sizeof(unsigned) * 2 * kSelBins));
constexpr size_t kBatchSmem = kLutSmemBytes + kBatchWork;
static_assert(kBatchWork >= sizeof(unsigned) * kTracks * kRadixBins, "radix histograms overlay the pass-1 buffers");
static_assert(kBatchWork >= sizeof(unsigned) * 2 * kSelBins, "select histograms overlay the pass-1 buffers");

// One tile of the batch (device, read-only during a run).
struct BatchTile {
  Geometry g;
  unsigned model;          // index of the tile's table
  unsigned n_items1;       // pass-1 items of the tile
  unsigned lo[2];          // window start key per stain (keys >= lo are listed); set by the pilot
  unsigned win[2];         // 0: no window (no hint): the stain takes the exact fallback
  float nk[2], lk[2];      // exact [h~ < lo] test (nk = 0, lk = 1 without a window)
  unsigned hlo[2], hwin[2];   // the same from the hint alone (kOpenLow * hint)
  float hnk[2], hlk[2];
  unsigned hkey[2];        // key of the hint itself (the pilot's design-effect threshold)
  unsigned* keys;          // stain-0 key list; stain 1 at keys + list_cap
  u64 list_cap;            // keys per stain
};

// Per-tile state of a run (zeroed before every run).
struct BatchTileState {
  SelectState sel;         // counts, ranks, keys, percentiles, scale; fallback barrier
  u64 list_n[2];           // keys appended (may exceed list_cap: overflow)
  unsigned done1;          // finished pass-1 items
  int ready;               // 0: pass 1 running, 1: scale known, 2: exact fallback needed
  int status;              // SPCN_OK or SPCN_ERR_NO_TISSUE
  int fallback;            // 1: the percentile needed the exact fallback
  float M[6];              // pass-2 coefficients (recon_coef), set with ready = 1
  int pad2[2];
  u64 srank[kTracks];      // grid-wide select: each track's rank within its first-digit bin
  int sbin[kTracks];       // and that bin (-1: the track is not resolved from the lists)
};

// Run-wide state (zeroed before every run).
struct BatchRunState {
  unsigned next;           // work-queue ticket (staged schedule: pass-1 items)
  unsigned next2;          // staged schedule: pass-2 items
  unsigned n_fallback;     // tiles left to the exact fallback (counted by the selects)
  unsigned barrier;        // grid barrier counter of the fallback phase
  unsigned barrier2;       // grid barrier counter of the persistent launch's phases
  int abort;               // a wait gave up
  int err;                 // first error of the run
};

struct BatchItem {
  unsigned tile;           // ~0u: no item (end of the queue)
  unsigned pass;           // 1 or 2
  unsigned model;          // the tile's table
  unsigned n_items1;       // pass-1 items of the tile
  u64 c0, c1;              // chunk range [c0, c1) of the tile
};

struct BatchArgs {
  const BatchTile* tiles;
  BatchTileState* state;
  const BatchItem* items;
  const Model* models;
  unsigned* hist1;         // per tile and stain: first-digit histogram of listed keys
  unsigned* hist2;         // grid-wide select: per tile and track, second-digit histogram
  const BatchItem* p1_items;  // staged pass 1: each block's segments (chunk ranges of one tile),
  const unsigned* p1_first;   // block b's at [p1_first[b], p1_first[b + 1])
  const BatchItem* p2_items;  // staged pass 2: the same for its grid
  const unsigned* p2_first;
  u64* rhist;
  BatchRunState* run;
  unsigned n_items, n_tiles;
  unsigned wthr;           // (white threshold + 1) << 8, compared with table offsets
  unsigned thr;            // white threshold
  unsigned wm, we;         // all-white test of a full chunk: (AND of its words & wm) == we
  double pct;
  double tgt0, tgt1;       // target percentiles
  float Wt[6];             // target basis
  float l2i0[3];           // log2 of the target i0
  long long timeout_ns;
};

// 32-byte item descriptor, global -> shared, without holding registers.
__device__ __forceinline__ void copy_item_async(BatchItem* dst, const BatchItem* src) {
  static_assert(sizeof(BatchItem) == 32, "two 16-byte copies");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const char* g = reinterpret_cast<const char*>(src);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"(d), "l"(g) : "memory");
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"(d + 16u), "l"(g + 16) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Bounded wait of one thread for a tile's ready word.  Returns the word (1
// or 2), or -1 when the run was aborted or the wait gave up (then the abort
// word and TIMEOUT are recorded).
__device__ int wait_ready(const int* ready, int* abort, int* err, long long timeout_ns) {
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    const int v = ld_acquire_s32(ready);
    if (v != 0) return v;
    if (*(volatile int*)abort != 0) return -1;
    if ((long long)(global_timer_ns() - t0) > timeout_ns) {
      atomicExch(abort, 1);
      record_error(err, SPCN_ERR_TIMEOUT);
      return -1;
    }
    __nanosleep(256);
  }
}

// Append a warp's buffered keys to a tile's list: one atomic reservation,
// then coalesced stores; keys past the capacity are counted but dropped.
// Every key also counts in the tile's first-digit histogram of d = key - lo
// (bin min(d >> 12, 4095), fire-and-forget reductions spread over all
// blocks), so the select needs only one pass over the list.  kc is
// warp-uniform.
__device__ __forceinline__ void red_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void flush_keys(const unsigned* kb, int kc, unsigned* list, u64 cap,
                                           u64* list_n, unsigned* hist1, unsigned lo) {
  if (kc == 0) return;
  const unsigned lane = threadIdx.x & 31u;
  u64 base = 0;
  if (lane == 0) base = atomicAdd(list_n, (u64)kc);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  for (int i = (int)lane; i < kc; i += 32) {
    const unsigned k = kb[i];
    if (base + (u64)i < cap) list[base + i] = k;
    red_add_u32(hist1 + min((k - lo) >> kSelBits, (unsigned)(kSelBins - 1)), 1u);
  }
}

// Keys of the queued chunks' flagged pixels (same arithmetic as pass 1, so
// the same keys), appended to the warp's key buffers.  The flagged pixels of
// up to 32 queue entries are numbered by a warp prefix sum, and each step
// gives every lane one of them (its entry by a binary search over the
// prefix sums, its pixel as the n-th set bit of the entry's mask), so no
// lane idles while another entry still has pixels left.  Warp-uniform.  The
// tile's list pointers are read here, not held by the pixel loop.
template <class G>
__device__ __noinline__ void batch_drain(const uint2* queue, int count, u64 c0, const G& g,
                                         const char* lut, unsigned lr, const Lasso& L,
                                         unsigned* kb0, unsigned* kb1, int& kc0, int& kc1,
                                         const BatchTile* T, BatchTileState* S, unsigned* h1) {
  const u64 cap = T->list_cap;
  unsigned* list0 = T->keys;
  unsigned* list1 = list0 + cap;
  const unsigned lo0 = T->win[0] ? T->lo[0] : 0xFFFFFFFFu;
  const unsigned lo1 = T->win[1] ? T->lo[1] : 0xFFFFFFFFu;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  for (int e0 = 0; e0 < count; e0 += 32) {
    // d: bit 2i set when digit i of the entry's mask is non-zero (digits
    // 0-7: even pixels, pair 7-i; digits 8-15: odd pixels, pair 15-i)
    unsigned d = 0u, q = 0u;
    if (e0 + (int)lane < count) {
      const uint2 ent = queue[e0 + lane];
      q = ent.x;
      d = (ent.y | (ent.y >> 1)) & 0x55555555u;
    }
    const unsigned n = __popc(d);
    unsigned incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if ((int)lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const unsigned excl = incl - n;
    for (unsigned s0 = 0; s0 < total; s0 += 32) {
      const unsigned sl = s0 + lane;
      // owner entry: the first lane whose inclusive sum exceeds sl
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned v = __shfl_sync(0xFFFFFFFFu, incl, j + step - 1);
        if (v <= sl) j += step;
      }
      const unsigned dj = __shfl_sync(0xFFFFFFFFu, d, j & 31);
      const unsigned qj = __shfl_sync(0xFFFFFFFFu, q, j & 31);
      const unsigned ej = __shfl_sync(0xFFFFFFFFu, excl, j & 31);
      unsigned k0 = 0u, k1 = 0u;
      bool in0 = false, in1 = false;
      if (sl < total) {
        const int i = (int)__fns(dj, 0u, (int)(sl - ej) + 1) >> 1;
        const int k = 2 * (7 - (i & 7)) + (i >> 3);
        const ChunkPos p = chunk_pos(g, c0 + qj);
        const uint8_t* src = g.src + p.src_off + 3 * k;
        const bool inside = SPCN_CHECK(k < p.n && p.src_off + 3 * (int64_t)k + 3 <= g.src_bytes,
                                       g.err);
        const unsigned r = inside ? __ldg(src) : 255u, gg = inside ? __ldg(src + 1) : 255u,
                       b = inside ? __ldg(src + 2) : 255u;
        float h1, h2;
        solve_one(lut, (r << 8) | lr, (gg << 8) | lr, (b << 8) | lr, L, h1, h2);
        k0 = __float_as_uint(h1);
        k1 = __float_as_uint(h2);
        in0 = k0 >= lo0;
        in1 = k1 >= lo1;
      }
      const unsigned b0 = __ballot_sync(0xFFFFFFFFu, in0), b1 = __ballot_sync(0xFFFFFFFFu, in1);
      if (in0) kb0[kc0 + __popc(b0 & lt)] = k0;
      if (in1) kb1[kc1 + __popc(b1 & lt)] = k1;
      kc0 += __popc(b0);
      kc1 += __popc(b1);
      if (kc0 > kKeyBuf - 32 || kc1 > kKeyBuf - 32) {
        __syncwarp();
        flush_keys(kb0, kc0, list0, cap, S->list_n, h1, lo0);
        flush_keys(kb1, kc1, list1, cap, S->list_n + 1, h1 + kSelBins, lo1);
        __syncwarp();
        kc0 = 0;
        kc1 = 0;
      }
    }
  }
}

// First bin whose inclusive prefix exceeds r in a shared histogram of n
// counts.  *s_idx = -1 if the total is <= r.
__device__ __forceinline__ void smem_find_rank(const unsigned* hist, int n, u64 r, int* s_idx,
                                               u64* s_before, u64* s_tmp) {
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per);
  const int cnt = min(per, n - beg);
  u64 local = 0;
  for (int i = 0; i < cnt; ++i) local += hist[beg + i];
  u64 total;
  const u64 excl = block_excl_scan(local, s_tmp, &total);
  if (threadIdx.x == 0) *s_idx = -1;
  __syncthreads();
  if (local > 0 && excl <= r && r < excl + local) {
    u64 c = excl;
    for (int i = 0; i < cnt; ++i) {
      const u64 x = hist[beg + i];
      if (r < c + x) { *s_idx = beg + i; *s_before = c; break; }
      c += x;
    }
  }
  __syncthreads();
}

// Percentile of one tile from its key lists, by the block that finished the
// tile's pass 1.  Rank r of the non-white densities is rank r - below among
// the listed keys when below <= r < below + count and the list is complete.
// Its first 12-bit digit of d = key - lo comes from the histogram built
// during pass 1, its last 12 bits from one pass over the list.  Ranks
// outside, or in the histogram's top (overflow) bin, leave the tile to the
// exact fallback.
__device__ void batch_select(const BatchArgs& a, unsigned tile, unsigned* s_hist, u64* s_tmp) {
  const BatchTile* T = a.tiles + tile;
  BatchTileState* S = a.state + tile;
  SelectState* s = &S->sel;
  __shared__ int s_idx;
  __shared__ u64 s_before;
  __shared__ int s_bin[2];
  __shared__ u64 s_rr[2];
  __shared__ int s_res[kTracks];
  const u64 n = __ldcg(&s->n_nw);
  if (n == 0) {
    if (threadIdx.x == 0) {
      S->status = SPCN_ERR_NO_TISSUE;
      for (int t = 0; t < kTracks; ++t) { s->key[t] = 0; s->resolved[t] = 1; }
      s->p99[0] = s->p99[1] = 0.0;
      s->scale[0] = s->scale[1] = 1.0;
      s->t = 0.0;
      s->all_resolved = 1;
      const float hs = a.models[T->model].lasso.hscale;
      for (int i = 0; i < 6; ++i) S->M[i] = recon_coef(a.Wt, s->scale, hs, i);
      __threadfence();
      st_release_s32(&S->ready, 1);
    }
    return;
  }
  if (threadIdx.x == 0) {
    set_ranks(s, n, a.pct);
    for (int j = 0; j < 2; ++j) { s->lo[j] = T->lo[j]; s->nb[j] = 0u; }
    for (int t = 0; t < kTracks; ++t) s_res[t] = 0;
  }
  __syncthreads();
  const u64 cap = T->list_cap;
  for (int j = 0; j < 2; ++j) {
    const unsigned lo = T->lo[j];
    const u64 cnt = __ldcg(&S->list_n[j]);
    const u64 below = __ldcg(&s->below[j]);
    const unsigned* list = T->keys + (u64)j * cap;
    bool in[2];
    for (int u = 0; u < 2; ++u) {
      const u64 r = s->rank[2 * j + u];
      in[u] = T->win[j] && cnt <= cap && r >= below && r - below < cnt;
    }
    if (!in[0] && !in[1]) continue;   // uniform across the block
    // first digit: the pass-1 histogram
    const unsigned* h1 = a.hist1 + ((size_t)tile * 2 + j) * kSelBins;
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) s_hist[i] = __ldcg(h1 + i);
    if (threadIdx.x == 0)
      for (int u = 0; u < 2; ++u) s_rr[u] = s->rank[2 * j + u] - below;
    __syncthreads();
    for (int u = 0; u < 2; ++u) {
      if (!in[u]) continue;
      smem_find_rank(s_hist, kSelBins, s_rr[u], &s_idx, &s_before, s_tmp);
      if (threadIdx.x == 0) {
        s_bin[u] = s_idx;
        if (s_idx >= 0) s_rr[u] -= s_before;
      }
      __syncthreads();
    }
    bool ok[2];
    for (int u = 0; u < 2; ++u) ok[u] = in[u] && s_bin[u] >= 0 && s_bin[u] < kSelBins - 1;
    if (!ok[0] && !ok[1]) { __syncthreads(); continue; }
    // second digit: one pass over the list, counting the keys of each
    // track's first-digit bin (one histogram when both bins agree)
    const int b0 = ok[0] ? s_bin[0] : -1, b1 = ok[1] ? s_bin[1] : -1;
    const bool share = b0 == b1 || b0 < 0 || b1 < 0;
    const int bb = b0 >= 0 ? b0 : b1;
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kSelBins; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    auto count = [&](unsigned key) {
      const unsigned d = key - lo;
      const int hb = (int)min(d >> kSelBits, (unsigned)(kSelBins - 1));
      const unsigned low = d & (kSelBins - 1);
      if (hb == bb) atomicAdd(s_hist + low, 1u);
      else if (!share && hb == b1) atomicAdd(s_hist + kSelBins + low, 1u);
    };
    // 16-byte loads, eight keys per thread and step (the lists start on
    // 16-byte boundaries; the last partial vector is read key by key)
    const uint4* v = reinterpret_cast<const uint4*>(list);
    const u64 nv = cnt / 4;
    for (u64 i = threadIdx.x; i < nv; i += 2 * blockDim.x) {
      const uint4 x = __ldcg(v + i);
      const bool two = i + blockDim.x < nv;
      uint4 y = make_uint4(0u, 0u, 0u, 0u);
      if (two) y = __ldcg(v + i + blockDim.x);
      count(x.x); count(x.y); count(x.z); count(x.w);
      if (two) { count(y.x); count(y.y); count(y.z); count(y.w); }
    }
    for (u64 i = nv * 4 + threadIdx.x; i < cnt; i += blockDim.x) count(__ldcg(list + i));
    __syncthreads();
    for (int u = 0; u < 2; ++u) {
      if (!ok[u]) continue;
      const unsigned* h = s_hist + ((share || u == 0) ? 0 : kSelBins);
      smem_find_rank(h, kSelBins, s_rr[u], &s_idx, &s_before, s_tmp);
      if (threadIdx.x == 0 && s_idx >= 0) {
        s->key[2 * j + u] = lo + ((unsigned)s_bin[u] << kSelBits) + (unsigned)s_idx;
        s_res[2 * j + u] = 1;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    int all = 1;
    for (int t = 0; t < kTracks; ++t) { s->resolved[t] = s_res[t]; all &= s_res[t]; }
    if (all) {
      const float hs = a.models[T->model].lasso.hscale;
      finish_percentiles(s, a.tgt0, a.tgt1, hs);
      for (int i = 0; i < 6; ++i) S->M[i] = recon_coef(a.Wt, s->scale, hs, i);
    }
    s->all_resolved = all;
    if (!all) atomicAdd(&a.run->n_fallback, 1u);
    __threadfence();
    st_release_s32(&S->ready, all ? 1 : 2);
  }
}

// ------------------------------------------------------------ window pilot
// Before the batch kernel, every tile's window start is set from a sample of
// the tile itself: one chunk from each of kPilotChunks equal strata of the
// tile's chunk range (every chunk of a smaller tile), the keys of their
// non-white pixels, and the key at the sample quantile q = p - delta, with
// p = pct / 100 and delta four standard deviations of the sample proportion,
// the variance taken from the sample's own between-chunk spread (a cluster
// sample: pixels of one chunk are not independent; see the design effect
// below), per stain.  The tile's own percentile lies at or above that key
// unless the sample is off by four standard deviations; a rank below the
// window start leaves the tile to the exact fallback, so the start changes
// the speed, never the result.  A stain without a hint keeps no window (the
// exact fallback); a sample with fewer than kPilotMinUnits tissue chunks
// keeps the hint's window.  Two 11-bit digits of the key (bits 31-21, then
// 20-10) are selected in shared memory; the start is the key with the low
// ten bits cleared, at or below the sample's key.
constexpr int kPilotChunks = 1024;
constexpr int kPilotMinUnits = 64;
constexpr int kPilotThreads = 512;
constexpr int kPilotBits = 11;
constexpr int kPilotBins = 1 << kPilotBits;
static_assert(kPilotChunks * kChunk * kChunk < (1 << 30), "a thread's pilot sums fit 32 bits");

struct PilotArgs {
  BatchTile* tiles;
  const Model* models;
  unsigned n_tiles;
  unsigned thr;   // white threshold
  double pct;
};

// The H-step of one pixel from an unreplicated copy of the projected table
// (channel-major, 256 entries each): the arithmetic of solve_one, so the same
// keys.
__device__ __forceinline__ void solve_table(const float2* proj, unsigned r, unsigned g,
                                             unsigned b, const Lasso& L, float& h1, float& h2) {
  const float2 eR = proj[r], eG = proj[256 + g], eB = proj[512 + b];
  const float D1 = add_sat(eR.x + eG.x, eB.x);
  const float D2 = add_sat(eR.y + eG.y, eB.y);
  const float t1 = mul_sat(L.kappa, fmaf(L.nrho1, D2, D1));
  const float t2 = mul_sat(L.kappa, fmaf(L.nrho2, D1, D2));
  h1 = fminf(D1, t1);
  h2 = fminf(D2, t2);
}

__device__ __forceinline__ unsigned pilot_hash(unsigned t, unsigned i) {
  unsigned h = t * 0x9E3779B1u + i * 0x85EBCA77u + 0x27D4EB2Fu;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return h;
}

// Block-wide sums of eight per-thread counts at once (one barrier round);
// every thread receives the totals.
__device__ __forceinline__ void block_sum8(u64 (&v)[8], u64 (*s_part)[8]) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], o);
  }
  __syncthreads();   // s_part is free
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) s_part[warp][i] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    u64 t = 0;
    for (unsigned w = 0; w < (blockDim.x >> 5); ++w) t += s_part[w][i];
    v[i] = t;
  }
}

// The pilot's shared memory (a static array of k_batch_pilot, carved from the
// dynamic shared memory of the persistent launch).
struct PilotSmem {
  unsigned hist[2][kPilotBins];
  float2 proj[kLutEntries];      // the tile's projected table
  u64 part[32][8];               // per-warp partial sums (up to 32 warps)
  u64 tmp[33];
  u64 before;
  u64 r[2];
  unsigned b1[2];
  int idx;
  int use;
};

// Window starts of the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (any
// block size up to 1024 threads).
__device__ void pilot_tiles(const PilotArgs& a, PilotSmem& sm) {
  unsigned (&s_hist)[2][kPilotBins] = sm.hist;
  float2 (&s_proj)[kLutEntries] = sm.proj;
  u64 (&s_part)[32][8] = sm.part;
  u64 (&s_tmp)[33] = sm.tmp;
  int& s_idx = sm.idx;
  u64& s_before = sm.before;
  unsigned (&s_b1)[2] = sm.b1;
  u64 (&s_r)[2] = sm.r;
  int& s_use = sm.use;
  for (unsigned t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    BatchTile* T = a.tiles + t;
    const Geometry g = T->g;
    const Model* m = a.models + T->model;
    const Lasso L = m->lasso;
    __syncthreads();   // the previous tile's table is no longer read
    for (int i = threadIdx.x; i < kLutEntries; i += blockDim.x) s_proj[i] = m->proj[i];
    __syncthreads();
    const u64 nch = g.nchunks;
    const unsigned ms = (unsigned)(nch < (u64)kPilotChunks ? nch : (u64)kPilotChunks);
    // every non-white pixel of the sample: f(key1, key2), then end() after
    // each sampled chunk
    auto visit = [&](auto&& f, auto&& end) -> unsigned {
      unsigned units = 0u;
      for (unsigned i = threadIdx.x; i < ms; i += blockDim.x) {
        u64 q = i;
        if (nch > (u64)kPilotChunks) {
          const u64 s0 = (u64)i * nch / kPilotChunks, s1 = (u64)(i + 1) * nch / kPilotChunks;
          q = s0 + pilot_hash(t, i) % (s1 - s0);
        }
        const ChunkPos p = chunk_pos(g, q);
        unsigned w[12];
        load_chunk<false>(g, p, w);
        bool any = false;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
          if (k >= p.n) break;
          const unsigned r = byte_at(w, 3 * k), gg = byte_at(w, 3 * k + 1), b = byte_at(w, 3 * k + 2);
          if (min(r, min(gg, b)) > a.thr) continue;   // white
          float h1, h2;
          solve_table(s_proj, r, gg, b, L, h1, h2);
          f(__float_as_uint(h1), __float_as_uint(h2));
          any = true;
        }
        end();
        units += any ? 1u : 0u;
      }
      return units;
    };
    auto none = [] {};
    for (int i = threadIdx.x; i < 2 * kPilotBins; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    // The margin delta = 4 sigma of the sample quantile, from the sample's own
    // between-chunk variance (pixels of one chunk are not independent): at
    // a provisional threshold t (the hint's key: the tile's percentile is
    // near its slide's), a_i = pixels of chunk i at or above t, m_i = its
    // non-white pixels, p^ = sum a / sum m, and the ratio estimator's
    // variance sum (a_i - p^ m_i)^2 / (u (u - 1) mbar^2) over p^ (1 - p^) /
    // sum m is the design effect d, clamped to [1, 16] (independent pixels ..
    // whole chunks as units); then sigma^2 = d p (1 - p) / sum m.  Without an
    // estimate (p^ of 0 or 1) the chunks are the units: sigma^2 = p (1 - p) /
    // u.  The chunk sums are taken in the same visit as the level-1
    // histograms: bits 31-21 of the keys (densities are >= 0: the sign bit
    // is 0).
    const unsigned t0 = T->hwin[0] ? T->hkey[0] : 0xFFFFFFFFu;
    const unsigned t1 = T->hwin[1] ? T->hkey[1] : 0xFFFFFFFFu;
    unsigned cm = 0u, ca0 = 0u, ca1 = 0u;   // the current chunk's counts
    // this thread's sums over its chunks (at most kPilotChunks / blockDim.x
    // chunks of 16 pixels: 32-bit sums are exact)
    unsigned sm = 0, smm = 0, sa0 = 0, saa0 = 0, sam0 = 0, sa1 = 0, saa1 = 0, sam1 = 0;
    const unsigned my_units = visit([&](unsigned k1, unsigned k2) {
      atomicAdd(&s_hist[0][k1 >> 21], 1u);
      atomicAdd(&s_hist[1][k2 >> 21], 1u);
      ++cm;
      ca0 += k1 >= t0 ? 1u : 0u;
      ca1 += k2 >= t1 ? 1u : 0u;
    }, [&] {
      sm += cm; smm += cm * cm;
      sa0 += ca0; saa0 += ca0 * ca0; sam0 += ca0 * cm;
      sa1 += ca1; saa1 += ca1 * ca1; sam1 += ca1 * cm;
      cm = ca0 = ca1 = 0u;
    });
    u64 units = 0;
    block_excl_scan((u64)my_units, s_tmp, &units);
    u64 nw = 0;
    {
      u64 part = 0;
      for (int i = threadIdx.x; i < kPilotBins; i += blockDim.x) part += s_hist[0][i];
      block_excl_scan(part, s_tmp, &nw);
    }
    u64 v[8] = {sm, smm, sa0, saa0, sam0, sa1, saa1, sam1};
    block_sum8(v, s_part);
    if (threadIdx.x == 0) {
      const double p = a.pct / 100.0;
      const double M = (double)v[0], U = (double)units;
      const u64 SA[2] = {v[2], v[5]}, SAA[2] = {v[3], v[6]}, SAM[2] = {v[4], v[7]};
      int use = units >= (u64)kPilotMinUnits && nw > 0;
      for (int j = 0; j < 2; ++j) {
        double var = p * (1.0 - p) / (U > 0.0 ? U : 1.0);   // chunks as units
        const double ph = M > 0.0 ? (double)SA[j] / M : 0.0;
        if (units >= 2 && ph > 0.0 && ph < 1.0) {
          const double mbar = M / U;
          const double ss = (double)SAA[j] - 2.0 * ph * (double)SAM[j] + ph * ph * (double)v[1];
          const double v = ss / (U * (U - 1.0) * mbar * mbar);
          double d = v / (ph * (1.0 - ph) / M);
          d = d < 1.0 ? 1.0 : (d > (double)kChunk ? (double)kChunk : d);
          var = d * p * (1.0 - p) / M;
        }
        const double q = p - 4.0 * sqrt(var);
        use = use && q > 0.0;
        s_r[j] = q > 0.0 && nw > 0 ? (u64)floor(q * (double)(nw - 1)) : 0;
      }
      s_use = use;
    }
    __syncthreads();
    if (s_use) {
      for (int j = 0; j < 2; ++j) {
        smem_find_rank(s_hist[j], kPilotBins, s_r[j], &s_idx, &s_before, s_tmp);
        if (threadIdx.x == 0) {
          s_b1[j] = (unsigned)max(s_idx, 0);
          s_r[j] -= s_idx >= 0 ? s_before : 0;
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < 2 * kPilotBins; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
      __syncthreads();
      // level 2: bits 20-10 of the keys in the level-1 bin
      const unsigned b10 = s_b1[0], b11 = s_b1[1];
      visit([&](unsigned k1, unsigned k2) {
        if ((k1 >> 21) == b10) atomicAdd(&s_hist[0][(k1 >> 10) & (kPilotBins - 1)], 1u);
        if ((k2 >> 21) == b11) atomicAdd(&s_hist[1][(k2 >> 10) & (kPilotBins - 1)], 1u);
      }, none);
      __syncthreads();
      for (int j = 0; j < 2; ++j) {
        smem_find_rank(s_hist[j], kPilotBins, s_r[j], &s_idx, &s_before, s_tmp);
        if (threadIdx.x == 0) {
          const unsigned lo = (s_b1[j] << 21) | ((unsigned)max(s_idx, 0) << 10);
          if (T->hwin[j] && lo > 0u) {
            T->lo[j] = lo;
            T->win[j] = 1u;
            below_consts(lo, &T->nk[j], &T->lk[j]);
          } else {
            T->lo[j] = T->hlo[j];
            T->win[j] = T->hwin[j];
            T->nk[j] = T->hnk[j];
            T->lk[j] = T->hlk[j];
          }
        }
        __syncthreads();
      }
    } else if (threadIdx.x == 0) {
      for (int j = 0; j < 2; ++j) {
        T->lo[j] = T->hlo[j];
        T->win[j] = T->hwin[j];
        T->nk[j] = T->hnk[j];
        T->lk[j] = T->hlk[j];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kPilotThreads, 2) k_batch_pilot(PilotArgs a) {
  __shared__ PilotSmem sm;
  pilot_tiles(a, sm);
}

// Pass 1 on one chunk with open-ended windows.  Per pixel: the non-white flag
// (0/1), [h~ < lo] per stain by saturated FMAs, accumulated with packed FMAs;
// the number of stains at or above their window start (0, 1 or 2) of each
// non-white pixel is packed base 4 into `mask` (pixel pair p at digit 7-p,
// even pixels in the low lane, odd pixels in the high lane).
__device__ __forceinline__ void open_window_chunk(const unsigned (&w)[12], const char* lut,
                                                  unsigned lr, f2 NR1, f2 NR2, float kappa,
                                                  unsigned wthr, float nk0, float lk0, float nk1,
                                                  float lk1, f2& c_nw, f2& c_b0, f2& c_b1,
                                                  f2& mask) {
  const f2 M1 = pk(-1.f, -1.f), FOUR = pk(4.f, 4.f), TWO = pk(2.f, 2.f);
  mask = pk(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < kChunk / 2; ++p) {
    const int kA = 2 * p, kB = 2 * p + 1;
    unsigned aRA, aGA, aBA, aRB, aGB, aBB;
    pixel_addr(w, kA, lr, aRA, aGA, aBA);
    pixel_addr(w, kB, lr, aRB, aGB, aBB);
    f2 H1, H2;
    solve_pair(lut, aRA, aGA, aBA, aRB, aGB, aBB, NR1, NR2, kappa, H1, H2);
    const bool nwA = min(min(aRA, aGA), aBA) < wthr;   // some channel <= threshold
    const bool nwB = min(min(aRB, aGB), aBB) < wthr;
    const f2 NW = pk(nwA ? 1.f : 0.f, nwB ? 1.f : 0.f);
    c_nw = add2(c_nw, NW);
    const float h1A = lo_of(H1), h1B = hi_of(H1), h2A = lo_of(H2), h2B = hi_of(H2);
    const f2 B0 = pk(fma_sat(h1A, nk0, lk0), fma_sat(h1B, nk0, lk0));
    const f2 B1 = pk(fma_sat(h2A, nk1, lk1), fma_sat(h2B, nk1, lk1));
    c_b0 = fma2(B0, NW, c_b0);
    c_b1 = fma2(B1, NW, c_b1);
    const f2 X = fma2(B0, M1, fma2(B1, M1, TWO));   // 2 - B0 - B1, exact
    mask = fma2(mask, FOUR, mul2(X, NW));
  }
}

// open_window_chunk for a row's last chunk with fewer than 16 pixels, pixel
// by pixel (the same tests; the padding bytes are not pixels): the counts,
// and the mask in the same base-4 layout for the hit queue.
__device__ __forceinline__ unsigned open_window_partial(const uint8_t* src, int n, const char* lut,
                                                        unsigned lr, const Lasso& L, unsigned wthr,
                                                        float nk0, float lk0, float nk1, float lk1,
                                                        f2& c_nw, f2& c_b0, f2& c_b1) {
  float nw = 0.f, b0 = 0.f, b1 = 0.f;
  unsigned mA = 0u, mB = 0u;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const unsigned aR = ((unsigned)__ldg(src + 3 * k) << 8) | lr;
    const unsigned aG = ((unsigned)__ldg(src + 3 * k + 1) << 8) | lr;
    const unsigned aB = ((unsigned)__ldg(src + 3 * k + 2) << 8) | lr;
    if (min(min(aR, aG), aB) >= wthr) continue;   // white
    float h1, h2;
    solve_one(lut, aR, aG, aB, L, h1, h2);
    const float B0 = fma_sat(h1, nk0, lk0), B1 = fma_sat(h2, nk1, lk1);
    nw += 1.f;
    b0 += B0;
    b1 += B1;
    const unsigned d = (unsigned)(2.f - B0 - B1) << (2 * (7 - (k >> 1)));
    if (k & 1) mB |= d; else mA |= d;
  }
  c_nw = add2(c_nw, pk(nw, 0.f));
  c_b0 = add2(c_b0, pk(b0, 0.f));
  c_b1 = add2(c_b1, pk(b1, 0.f));
  return mA | (mB << 16);
}

__device__ __forceinline__ ReconConst recon_const(const float* s_M, const float* l2i0) {
  ReconConst K;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    K.M1[c] = pk(s_M[c], s_M[c]);
    K.M2[c] = pk(s_M[3 + c], s_M[3 + c]);
    K.L2[c] = pk(l2i0[c], l2i0[c]);
  }
  return K;
}

// Contiguous image (one long row) whose source is 16-byte aligned: full
// chunks may be addressed by index with vector loads.
__device__ __forceinline__ bool flat_src(const FlatGeometry& g) { return g.vec_src; }
__device__ __forceinline__ bool flat_src(const Geometry& g) { return g.flat && g.vec_src; }

template <class G>
__device__ __forceinline__ G geometry_as(const Geometry& g);
template <>
__device__ __forceinline__ Geometry geometry_as<Geometry>(const Geometry& g) { return g; }
template <>
__device__ __forceinline__ FlatGeometry geometry_as<FlatGeometry>(const Geometry& g) {
#ifdef SPCN_CHECKED
  return FlatGeometry{g.src, g.dst, (u64)g.npx, g.vec_src, g.vec_dst, g.src_bytes, g.dst_bytes, g.err};
#else
  return FlatGeometry{g.src, g.dst, (u64)g.npx, g.vec_src, g.vec_dst};
#endif
}

// One pass-1 item: chunks [c0, c1) of a tile, by the whole block.
template <class G>
__device__ __forceinline__ unsigned batch_pass1(const BatchArgs& a, unsigned tile, u64 c0,
                                                u64 c1, const char* lut, unsigned lr,
                                                uint2* s_queue, unsigned* s_kb, unsigned* s_cnt,
                                                unsigned* s_piece) {
  const BatchTile* T = a.tiles + tile;
  BatchTileState* S = a.state + tile;
  const G g = geometry_as<G>(T->g);
  const Lasso L = a.models[T->model].lasso;
  const float nk0 = T->nk[0], lk0 = T->lk[0], nk1 = T->nk[1], lk1 = T->lk[1];
  unsigned* h1 = a.hist1 + (size_t)tile * 2 * kSelBins;
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  f2 c_nw = pk(0.f, 0.f), c_b0 = pk(0.f, 0.f), c_b1 = pk(0.f, 0.f);
  unsigned* kb0 = s_kb;
  unsigned* kb1 = s_kb + kKeyBuf;
  const unsigned lane = threadIdx.x & 31u;
  int qn = 0, kc0 = 0, kc1 = 0;   // warp-uniform
  // warps claim 32-chunk pieces of the item from a shared counter, so a warp
  // that spends time draining its queue takes fewer pieces and all warps
  // reach the end of the item together
  for (;;) {
    unsigned piece = 0u;
    if (lane == 0) piece = atomicAdd(s_piece, 1u);
    const u64 base = c0 + 32ull * __shfl_sync(0xFFFFFFFFu, piece, 0);
    if (base >= c1) break;
    const u64 q = base + lane;
    unsigned packed = 0u;
    if (q < c1) {
      const ChunkPos p = chunk_pos(g, q);
      unsigned w[12];
      load_chunk<false>(g, p, w);
      if (p.n == kChunk) {
        f2 mask;
        open_window_chunk(w, lut, lr, NR1, NR2, L.kappa, a.wthr, nk0, lk0, nk1, lk1, c_nw, c_b0,
                          c_b1, mask);
        packed = (unsigned)lo_of(mask) | ((unsigned)hi_of(mask) << 16);
      } else {
        if (SPCN_CHECK(p.src_off + 3 * (int64_t)p.n <= g.src_bytes, g.err))
        packed = open_window_partial(g.src + p.src_off, p.n, lut, lr, L, a.wthr, nk0, lk0, nk1,
                                     lk1, c_nw, c_b0, c_b1);
      }
    }
    const bool hit = packed != 0u;
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, hit);
    if (hit) s_queue[qn + __popc(ball & ((1u << lane) - 1u))] = make_uint2((unsigned)(q - c0), packed);
    qn += __popc(ball);
    if (qn >= 32) {
      __syncwarp();
      batch_drain(s_queue, qn, c0, g, lut, lr, L, kb0, kb1, kc0, kc1, T, S, h1);
      __syncwarp();
      qn = 0;
    }
  }
  __syncwarp();
  if (qn > 0) batch_drain(s_queue, qn, c0, g, lut, lr, L, kb0, kb1, kc0, kc1, T, S, h1);
  __syncwarp();
  {
    unsigned* h1 = a.hist1 + (size_t)tile * 2 * kSelBins;
    flush_keys(kb0, kc0, T->keys, T->list_cap, S->list_n, h1, T->lo[0]);
    flush_keys(kb1, kc1, T->keys + T->list_cap, T->list_cap, S->list_n + 1, h1 + kSelBins,
               T->lo[1]);
  }
  // per-thread counts are exact in FP32 (fewer than 2^24 pixels per thread),
  // per-warp sums fit 32 bits; one shared-memory round gives thread 0 the
  // block's counts
  unsigned v0 = (unsigned)lo_of(c_nw) + (unsigned)hi_of(c_nw);
  unsigned v1 = (unsigned)lo_of(c_b0) + (unsigned)hi_of(c_b0);
  unsigned v2 = (unsigned)lo_of(c_b1) + (unsigned)hi_of(c_b1);
  v0 = __reduce_add_sync(0xFFFFFFFFu, v0);
  v1 = __reduce_add_sync(0xFFFFFFFFu, v1);
  v2 = __reduce_add_sync(0xFFFFFFFFu, v2);
  if (lane == 0) {
    s_cnt[3 * (threadIdx.x >> 5)] = v0;
    s_cnt[3 * (threadIdx.x >> 5) + 1] = v1;
    s_cnt[3 * (threadIdx.x >> 5) + 2] = v2;
  }
  __threadfence();   // this thread's key stores before the completion ticket
  __syncthreads();
  unsigned ticket = 0u;
  if (threadIdx.x == 0) {
    u64 t_nw = 0, t_b0 = 0, t_b1 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t_nw += s_cnt[3 * w];
      t_b0 += s_cnt[3 * w + 1];
      t_b1 += s_cnt[3 * w + 2];
    }
    if (t_nw) atomicAdd(&S->sel.n_nw, t_nw);
    if (t_b0) atomicAdd(&S->sel.below[0], t_b0);
    if (t_b1) atomicAdd(&S->sel.below[1], t_b1);
    __threadfence();
    ticket = atomicAdd(&S->done1, 1u);   // read at the next loop top
  }
  return ticket;
}

// One pass-2 item: chunks [c0, c1) of a tile, by the whole block.  The
// block's table must be the tile's optical-density table.
template <class G>
__device__ __forceinline__ void batch_pass2(const BatchArgs& a, unsigned tile, u64 c0, u64 c1,
                                            const char* lut, const float* s_M) {
  const BatchTile* T = a.tiles + tile;
  const G g = geometry_as<G>(T->g);
  const Model* m = a.models + T->model;
  const Lasso L = m->lasso;
  const ProjConst P = proj_const(m);
  const ReconConst K = recon_const(s_M, a.l2i0);
  const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
  const unsigned lr = lane_reg_od();
  for_chunks<true, true>(g, c0 + threadIdx.x, c1, blockDim.x,
                         [&](const unsigned (&w)[12], const ChunkPos& p) {
                           unsigned o[12];
                           recon_chunk(w, lut, lr, P, NR1, NR2, L.kappa, K, o);
                           store_chunk(g, p, o);
                         });
}


template <class G>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  char* lut = s_dyn;
  char* work = s_dyn + kLutSmemBytes;
  const unsigned warp = threadIdx.x >> 5;
  uint2* s_queue = reinterpret_cast<uint2*>(work) + warp * kWarpQueue;
  unsigned* s_kb = reinterpret_cast<unsigned*>(work + kBatchQueueBytes) + warp * 2 * kKeyBuf;
  unsigned* s_hist = reinterpret_cast<unsigned*>(work);   // select / radix histograms (overlay)
  __shared__ u64 s_tmp[33];
  __shared__ unsigned s_cnt[3 * 32];
  __shared__ __align__(16) BatchItem s_items[2];   // current item and the prefetched next one
  __shared__ int s_go, s_sel_tile;
  __shared__ unsigned s_piece;
  __shared__ float s_M[6];
  // staged schedule (empty queue): the selects are done and counted the
  // tiles left to the fallback; none, nothing to do (the same in every block)
  if (a.n_items == 0 && __ldcg(&a.run->n_fallback) == 0u) return;
  const unsigned lr = lane_reg();
  int cur_table = -1;   // table in shared memory: 2 * model + (1: optical densities, 0: projected)
  // Thread 0 runs the queue one item ahead: the next item's descriptor is
  // copied into shared memory asynchronously (cp.async) and the ticket of the
  // one after it is in flight while the block works; the completion ticket of
  // a pass-1 item is read at the next loop top.
  unsigned t_next = 0u, pend_tile = ~0u, pend_ticket = 0u, pend_last = 0u;
  int cur = 0;
  if (threadIdx.x == 0) {
    const unsigned t1 = atomicAdd(&a.run->next, 1u);
    if (t1 < a.n_items) copy_item_async(&s_items[1], a.items + t1);
    else s_items[1].tile = ~0u;
    t_next = atomicAdd(&a.run->next, 1u);
  }
  for (;;) {
    cur ^= 1;
    if (threadIdx.x == 0) {
      s_sel_tile = (pend_tile != ~0u && pend_ticket == pend_last) ? (int)pend_tile : -1;
      pend_tile = ~0u;
      s_piece = 0u;
      cp_async_wait_all();
      BatchItem* nx = &s_items[cur ^ 1];   // read by nobody until the next loop top
      if (s_items[cur].tile != ~0u && t_next < a.n_items) {
        copy_item_async(nx, a.items + t_next);
        t_next = atomicAdd(&a.run->next, 1u);
      } else {
        nx->tile = ~0u;
      }
    }
    __syncthreads();
    if (s_sel_tile >= 0) {   // this block finished the tile's last pass-1 item
      __threadfence();
      batch_select(a, (unsigned)s_sel_tile, s_hist, s_tmp);
      __syncthreads();
    }
    const BatchItem item = s_items[cur];
    if (item.tile == ~0u) break;
    if (item.pass == 2) {
      if (threadIdx.x == 0) {
        BatchTileState* S = a.state + item.tile;
        const int st = wait_ready(&S->ready, &a.run->abort, &a.run->err, a.timeout_ns);
        if (st == 1)
          for (int i = 0; i < 6; ++i) s_M[i] = __ldcg(&S->M[i]);
        s_go = st;
      }
      __syncthreads();
      if (s_go < 0) break;     // the run was aborted
      if (s_go != 1) {         // tile left to the exact fallback
        __syncthreads();
        continue;
      }
    }
    const int want = 2 * (int)item.model + (item.pass == 2 ? 1 : 0);
    if (want != cur_table) {
      if (item.pass == 2) load_od_lut(a.models + item.model, lut);
      else load_lut(a.models + item.model, lut);
      cur_table = want;
    }
    if (item.pass == 1) {
      const unsigned tk = batch_pass1<G>(a, item.tile, item.c0, item.c1, lut, lr, s_queue, s_kb,
                                         s_cnt, &s_piece);
      if (threadIdx.x == 0) {
        pend_tile = item.tile;
        pend_ticket = tk;
        pend_last = item.n_items1 - 1u;
      }
    } else {
      batch_pass2<G>(a, item.tile, item.c0, item.c1, lut, s_M);
    }
    __syncthreads();   // the item is done: shared words and the table may be rewritten
  }
  // tiles whose ranks the windows missed: exact radix select over the whole
  // grid, then their pass 2 (tile order; the ready words are final here)
  if (!grid_barrier(&a.run->barrier, gridDim.x, &a.run->abort, &a.run->err, a.timeout_ns)) return;
  if (__ldcg(&a.run->n_fallback) == 0u) return;   // final after the barrier; the same everywhere
  unsigned target = gridDim.x;
  for (unsigned t = 0; t < a.n_tiles; ++t) {
    BatchTileState* S = a.state + t;
    if (__ldcg(&S->ready) != 2) continue;   // same value in every block
    if (blockIdx.x == 0 && threadIdx.x == 0) S->fallback = 1;
    const BatchTile* T = a.tiles + t;
    const unsigned model = T->model;
    __syncthreads();
    if (2 * (int)model != cur_table) {   // the select reads the projected table
      load_lut(a.models + model, lut);
      cur_table = 2 * (int)model;
    }
    const Lasso L = a.models[model].lasso;
    u64 rank[kTracks];
    int active[kTracks];
    for (int k = 0; k < kTracks; ++k) {
      rank[k] = __ldcg(&S->sel.rank[k]);
      active[k] = !__ldcg(&S->sel.resolved[k]);
    }
    const ImageSource src{T->g, a.thr};
    if (!radix_select<false>(src, lut, L, &S->sel, rank, active, a.rhist, s_hist, &S->sel.barrier,
                      &a.run->err, a.timeout_ns, a.tgt0, a.tgt1))
      return;
    target += gridDim.x;
    if (!grid_barrier(&a.run->barrier, target, &a.run->abort, &a.run->err, a.timeout_ns)) return;
    if (threadIdx.x == 0) {
      const double sc[2] = {__ldcg(&S->sel.scale[0]), __ldcg(&S->sel.scale[1])};
      for (int i = 0; i < 6; ++i) s_M[i] = recon_coef(a.Wt, sc, L.hscale, i);
    }
    __syncthreads();
    // the tile's pass 2 over the whole grid, from its optical-density table
    __syncthreads();
    load_od_lut(a.models + model, lut);
    cur_table = 2 * (int)model + 1;
    const ProjConst P = proj_const(a.models + model);
    const ReconConst K = recon_const(s_M, a.l2i0);
    const f2 NR1 = pk(L.nrho1, L.nrho1), NR2 = pk(L.nrho2, L.nrho2);
    const unsigned lro = lane_reg_od();
    const Geometry g = T->g;
    for_each_chunk<true, true>(g, [&](const unsigned (&w)[12], const ChunkPos& p) {
      unsigned o[12];
      recon_chunk(w, lut, lro, P, NR1, NR2, L.kappa, K, o);
      store_chunk(g, p, o);
    });
  }
}

// ------------------------------------------------------------ staged schedule
// SPCN_SCHED_STAGED runs the batch as separate launches, each with the whole
// shared memory and register budget for its own pass:
//   k_batch_pilot  window starts (above);
//   k_batch_p1     pass 1 of every tile with the single-image chunk handling:
//                  all-white chunks dropped, chunks provably below both
//                  window starts counted without densities, the others kept
//                  on a per-warp stack until a full warp of them runs the
//                  closed-form H-step, and every pixel at or above a window
//                  start queued, recomputed and its keys appended to the
//                  tile's lists (with the first-digit histograms);
//   k_batch_sel    one block per tile: batch_select over the lists;
//   k_batch_p2     pass 2 of every tile whose percentile is known;
//   k_batch        with an empty queue: only the exact fallback of the tiles
//                  whose ranks missed their window.
// Blocks claim items (chunk ranges of one tile; the tiles of one table are
// adjacent in the list) from a ticket.  All warps of a block work on the same
// item, so the current tile's constants live in shared memory and a table is
// loaded only when the model changes.  A warp's stack and hit queue hold
// chunks of one tile: they are emptied when the block moves to another tile.
constexpr size_t kStagedQueueBytes = sizeof(uint2) * kWarpQueue * kWarps;
constexpr size_t kStagedStackBytes =
    (3 * sizeof(uint4) + sizeof(unsigned)) * kChunkStack * kWarps;
constexpr int kStagedKeyBuf = 96;   // keys per stain buffered per warp (flushed above 64)
constexpr size_t kStagedKeyBytes = sizeof(unsigned) * 2 * kStagedKeyBuf * kWarps;
constexpr size_t kStagedSmem =
    kLutSmemBytes + kStagedQueueBytes + kStagedStackBytes + kStagedKeyBytes;
constexpr size_t kSelectSmem = sizeof(unsigned) * 2 * kSelBins;

// The current tile of a k_batch_p1 block.
struct StagedTile {
  WindowConst C;      // [h~ < lo] tests of the tile's window starts; the upper
                      // tests are constant 1 (the windows are open above)
  unsigned* list0;    // key lists (stain 1 at list0 + cap)
  unsigned* list1;
  u64* list_n;        // keys appended per stain
  unsigned* hist;     // first-digit histograms (stain 1 at hist + kSelBins)
  SelectState* sel;   // the tile's counts
  u64 cap;
};

// The warp's buffered keys appended to the tile's lists (flush_keys: one
// atomic reservation per stain) and the buffers emptied.  Called by the whole
// warp; kc0 and kc1 are warp-uniform.
__device__ __forceinline__ void staged_flush_keys(unsigned* kb, int& kc0, int& kc1,
                                                  const StagedTile& t) {
  __syncwarp();
  flush_keys(kb, kc0, t.list0, t.cap, t.list_n, t.hist, t.C.lo0);
  flush_keys(kb + kStagedKeyBuf, kc1, t.list1, t.cap, t.list_n + 1, t.hist + kSelBins, t.C.lo1);
  __syncwarp();
  kc0 = kc1 = 0;
}

// Keys of up to 32 queued pixels (lane e takes entry e < count: the tile's
// chunk index and the pixel in the chunk).  The pixel is read again (still in
// L2) and its densities recomputed with solve_one, so its keys are those of
// every other pass; keys at or above a window start go to the warp's key
// buffers (kb: stain 0, kb + kStagedKeyBuf: stain 1), flushed to the lists
// once more than kStagedKeyBuf - 32 wait.  Called by the whole warp.
template <class G>
__device__ __forceinline__ void staged_drain(const uint2* queue, int count, const G& g,
                                             const char* lut, unsigned lr, const Lasso& L,
                                             const StagedTile& t, unsigned* kb, int& kc0,
                                             int& kc1) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  unsigned k0 = 0u, k1 = 0u;
  bool in0 = false, in1 = false;
  if ((int)lane < count) {
    const uint2 ent = queue[lane];
    const ChunkPos p = chunk_pos(g, (u64)ent.x);
    const int k = (int)ent.y;
    if (SPCN_CHECK(k < p.n && p.src_off >= 0 && p.src_off + 3 * (int64_t)k + 3 <= g.src_bytes,
                   g.err)) {
      const uint8_t* src = g.src + p.src_off + 3 * k;
      const unsigned r = __ldg(src), gg = __ldg(src + 1), b = __ldg(src + 2);
      float h1, h2;
      solve_one(lut, (r << 8) | lr, (gg << 8) | lr, (b << 8) | lr, L, h1, h2);
      k0 = __float_as_uint(h1);
      k1 = __float_as_uint(h2);
      in0 = k0 >= t.C.lo0;
      in1 = k1 >= t.C.lo1;
    }
  }
  const unsigned b0 = __ballot_sync(0xFFFFFFFFu, in0), b1 = __ballot_sync(0xFFFFFFFFu, in1);
  if (in0) kb[kc0 + __popc(b0 & lt)] = k0;
  if (in1) kb[kStagedKeyBuf + kc1 + __popc(b1 & lt)] = k1;
  kc0 += __popc(b0);
  kc1 += __popc(b1);
  if (kc0 > kStagedKeyBuf - 32 || kc1 > kStagedKeyBuf - 32) staged_flush_keys(kb, kc0, kc1, t);
}

// Queue the flagged pixels of the warp's chunks: bit 2 (7 - p) + h of d marks
// pixel 2 p + h of the lane's chunk qi.  Every 32 waiting entries are drained
// in one step of the warp.  Called by the whole warp; qn is warp-uniform.
template <class G>
__device__ __forceinline__ void staged_queue(unsigned d, unsigned qi, uint2* s_queue, int& qn,
                                             const G& g, const char* lut, unsigned lr,
                                             const Lasso& L, const StagedTile& t, unsigned* kb,
                                             int& kc0, int& kc1) {
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
      staged_drain(s_queue, 32, g, lut, lr, L, t, kb, kc0, kc1);
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

// A row's last chunk when it holds fewer than 16 pixels, pixel by pixel: the
// counts (the padding bytes are not pixels) and the flags of its pixels at
// or above a window start, in the layout of staged_queue.
__device__ __forceinline__ unsigned staged_partial(const uint8_t* src, int n, const char* lut,
                                                   unsigned lr, const Lasso& L,
                                                   const WindowConst& C, f2& c_nw, f2& c_b0,
                                                   f2& c_b1) {
  float nw = 0.f, b0 = 0.f, b1 = 0.f;
  unsigned d = 0u;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const unsigned aR = ((unsigned)__ldg(src + 3 * k) << 8) | lr;
    const unsigned aG = ((unsigned)__ldg(src + 3 * k + 1) << 8) | lr;
    const unsigned aB = ((unsigned)__ldg(src + 3 * k + 2) << 8) | lr;
    if (min(min(aR, aG), aB) >= C.wthr) continue;   // white
    float h1, h2;
    solve_one(lut, aR, aG, aB, L, h1, h2);
    const float B0 = fma_sat(h1, C.nk0, C.lk0), B1 = fma_sat(h2, C.nk1, C.lk1);
    nw += 1.f;
    b0 += B0;
    b1 += B1;
    if (B0 + B1 < 2.f) d |= 1u << (2 * (7 - (k >> 1)) + (k & 1));
  }
  c_nw = add2(c_nw, pk(nw, 0.f));
  c_b0 = add2(c_b0, pk(b0, 0.f));
  c_b1 = add2(c_b1, pk(b1, 0.f));
  return d;
}

// A warp's counts added to the tile's totals, then zeroed.  Per-thread counts
// are exact in FP32 (one item holds fewer than 2^24 pixels per thread); a
// thread's below counts can be negative (a stacked chunk's white pixels are
// taken off by the lane that classified it and counted by the lane that runs
// its H-step), and the 32-bit warp sums, sign-extended, add up modulo 2^64 to
// the tile's exact totals.
__device__ __forceinline__ void staged_counts(SelectState* sel, f2& c_nw, f2& c_b0, f2& c_b1) {
  const int v0 = __reduce_add_sync(0xFFFFFFFFu, (int)lo_of(c_nw) + (int)hi_of(c_nw));
  const int v1 = __reduce_add_sync(0xFFFFFFFFu, (int)lo_of(c_b0) + (int)hi_of(c_b0));
  const int v2 = __reduce_add_sync(0xFFFFFFFFu, (int)lo_of(c_b1) + (int)hi_of(c_b1));
  if ((threadIdx.x & 31u) == 0u) {
    if (v0) atomicAdd(&sel->n_nw, (u64)(long long)v0);
    if (v1) atomicAdd(&sel->below[0], (u64)(long long)v1);
    if (v2) atomicAdd(&sel->below[1], (u64)(long long)v2);
  }
  c_nw = c_b0 = c_b1 = pk(0.f, 0.f);
}

// Pass 1 of every tile (staged schedule).  One block per SM; items from the
// run's first ticket.
template <class G>
__device__ __forceinline__ void p1_phase(const BatchArgs& a, char* s_dyn) {
  char* lut = s_dyn;
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  uint2* s_queue = reinterpret_cast<uint2*>(s_dyn + kLutSmemBytes) + warp * kWarpQueue;
  char* stk = s_dyn + kLutSmemBytes + kStagedQueueBytes;
  uint4* s_stk = reinterpret_cast<uint4*>(stk) + warp * (3 * kChunkStack);
  unsigned* s_stq =
      reinterpret_cast<unsigned*>(stk + sizeof(uint4) * 3 * kChunkStack * kWarps) +
      warp * kChunkStack;
  unsigned* s_kb = reinterpret_cast<unsigned*>(stk + kStagedStackBytes) + warp * 2 * kStagedKeyBuf;
  __shared__ __align__(16) BatchItem s_items[2];   // current item and the prefetched next one
  __shared__ unsigned s_piece;
  __shared__ StagedTile s_t;
  __shared__ G s_g;
  __shared__ Lasso s_L;
  const unsigned lr = lane_reg();
  const WhiteBytes wb = white_bytes(a.thr);
  int cur_tile = -1, cur_model = -1;
  bool wbelow = false;   // every white pixel of the tile lies below both window starts
  int qn = 0;            // entries in this warp's hit queue (warp-uniform)
  int ns = 0;            // chunks on this warp's stack (warp-uniform)
  int kc0 = 0, kc1 = 0;  // keys in this warp's buffers (warp-uniform)
  f2 c_nw = pk(0.f, 0.f), c_b0 = c_nw, c_b1 = c_nw;
  // the window arithmetic of a warp of tissue chunks (lanes with have =
  // false take no part), then the hit queue
  auto lasso = [&](const unsigned (&w)[12], unsigned qi, bool have) {
    unsigned d = 0u;
    if (have) {
      const f2 NR1 = pk(s_L.nrho1, s_L.nrho1), NR2 = pk(s_L.nrho2, s_L.nrho2);
      f2 mask;
      if (wbelow)
        window_chunk<false, true>(w, lut, lr, NR1, NR2, s_L.kappa, s_t.C, c_nw, c_b0, c_b1, mask);
      else
        window_chunk<false, false>(w, lut, lr, NR1, NR2, s_L.kappa, s_t.C, c_nw, c_b0, c_b1,
                                   mask);
      const unsigned m0 = (unsigned)lo_of(mask), m1 = (unsigned)hi_of(mask);
      d = ((m0 | (m0 >> 1)) & 0x5555u) | (((m1 | (m1 >> 1)) & 0x5555u) << 1);
    }
    staged_queue(d, qi, s_queue, qn, s_g, lut, lr, s_L, s_t, s_kb, kc0, kc1);
  };
  // counts of a full, not all-white chunk; true when it needs the H-step
  // (not provably below both window starts)
  auto classify = [&](const unsigned (&w)[12]) -> bool {
    unsigned rg, bb;
    const float nw = chunk_nonwhite_min(w, wb, &rg, &bb);
    const bool below = below_bound(rg, bb, lut, lr, s_t.C);
    if (below || wbelow) {
      const f2 nb = pk(below ? nw : nw - (float)kChunk, 0.f);
      c_nw = add2(c_nw, pk(nw, 0.f));
      c_b0 = add2(c_b0, nb);
      c_b1 = add2(c_b1, nb);
    }
    return !below;
  };
  // tissue chunks wait on the stack until a full warp of them is ready
  auto warp_step = [&](bool tissue, unsigned (&w)[12], unsigned qi) {
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, tissue);
    const int cnt = __popc(ball);
    __syncwarp();   // the stack's previous reads and writes are done
    if (ns + cnt < 32) {
      if (tissue) stack_put(s_stk, s_stq, ns + __popc(ball & lt), w, qi);
      ns += cnt;
      return;
    }
    if (!tissue) stack_get(s_stk, s_stq, ns - 1 - __popc(~ball & lt), w, qi);
    ns -= 32 - cnt;
    lasso(w, qi, true);
  };
  // the rest of the warp's stack and queue, and its counts, before the block
  // moves to another tile
  auto flush_tile = [&]() {
    __syncwarp();
    if (ns > 0) {
      const bool have = lane < (unsigned)ns;
      unsigned w[12];
      unsigned qi = 0u;
      if (have) stack_get(s_stk, s_stq, (int)lane, w, qi);
      lasso(w, qi, have);
      ns = 0;
    }
    if (qn > 0) {
      __syncwarp();
      staged_drain(s_queue, qn, s_g, lut, lr, s_L, s_t, s_kb, kc0, kc1);
      qn = 0;
    }
    staged_flush_keys(s_kb, kc0, kc1, s_t);
    staged_counts(s_t.sel, c_nw, c_b0, c_b1);
  };
  // thread 0 walks the block's segments, copying the next descriptor into
  // shared memory one segment ahead (cp.async)
  unsigned i_next = 0u, i_end = 0u;
  int cur = 0;
  if (threadIdx.x == 0) {
    i_next = a.p1_first[blockIdx.x];
    i_end = a.p1_first[blockIdx.x + 1];
    if (i_next < i_end) copy_item_async(&s_items[1], a.p1_items + i_next++);
    else s_items[1].tile = ~0u;
  }
  for (;;) {
    cur ^= 1;
    if (threadIdx.x == 0) {
      cp_async_wait_all();
      BatchItem* nx = &s_items[cur ^ 1];   // read by nobody until the next loop top
      if (s_items[cur].tile != ~0u && i_next < i_end) copy_item_async(nx, a.p1_items + i_next++);
      else nx->tile = ~0u;
      s_piece = 0u;
    }
    __syncthreads();
    const unsigned tile = s_items[cur].tile;
    const u64 c0 = s_items[cur].c0, c1 = s_items[cur].c1;
    const unsigned model = s_items[cur].model;
    if ((int)tile != cur_tile && cur_tile >= 0) flush_tile();
    if (tile == ~0u) break;
    if ((int)tile != cur_tile) {
      __syncthreads();   // every warp is done with the previous tile's table and constants
      if ((int)model != cur_model) {
        load_lut(a.models + model, lut);   // ends with a block barrier
        cur_model = (int)model;
      }
      if (threadIdx.x == 0) {
        const BatchTile* T = a.tiles + tile;
        BatchTileState* S = a.state + tile;
        StagedTile st;
        st.C = WindowConst{nullptr, a.wthr, T->win[0] ? T->lo[0] : 0xFFFFFFFFu,
                           T->win[1] ? T->lo[1] : 0xFFFFFFFFu, 0u, 0u, T->nk[0], T->lk[0],
                           T->nk[1], T->lk[1], 0.f, 1.f, 0.f, 1.f};
        st.list0 = T->keys;
        st.list1 = T->keys + T->list_cap;
        st.list_n = S->list_n;
        st.hist = a.hist1 + (size_t)tile * 2 * kSelBins;
        st.sel = &S->sel;
        st.cap = T->list_cap;
        s_t = st;
        s_g = geometry_as<G>(T->g);
        s_L = a.models[model].lasso;
      }
      __syncthreads();
      cur_tile = (int)tile;
      wbelow = whites_below(a.thr, lut, lr, s_t.C);
    }
    // chunks below vfull are full chunks of a contiguous tile whose source
    // is 16-byte aligned (0: the general traversal for every chunk)
    const u64 vfull = flat_src(s_g) ? (u64)s_g.npx / kChunk : 0ull;
    // the item's chunks, 32 per warp step, in pieces claimed from a shared
    // counter (a warp that spends time on its stack or queue takes fewer)
    for (;;) {
      unsigned piece = 0u;
      if (lane == 0) piece = atomicAdd(&s_piece, 1u);
      const u64 base = c0 + 32ull * __shfl_sync(0xFFFFFFFFu, piece, 0);
      if (base >= c1) break;
      const u64 q = base + lane;
      unsigned w[12];
      bool tissue = false;
      unsigned dpart = 0u;
      if (q < c1 && q < vfull) {
        // full chunk of a contiguous, 16-byte aligned tile: plain vector loads
        if (SPCN_CHECK((int64_t)(q + 1) * (3 * kChunk) <= s_g.src_bytes, s_g.err)) {
          const uint4* v = reinterpret_cast<const uint4*>(s_g.src) + 3 * q;
          const uint4 x = __ldg(v), y = __ldg(v + 1), z = __ldg(v + 2);
          w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
          w[4] = y.x; w[5] = y.y; w[6] = y.z; w[7] = y.w;
          w[8] = z.x; w[9] = z.y; w[10] = z.z; w[11] = z.w;
          tissue = !chunk_white(w, a.wm, a.we) && classify(w);
        }
      } else if (q < c1) {
        const ChunkPos p = chunk_pos(s_g, q);
        load_chunk<false>(s_g, p, w);
        if (p.n == kChunk) {
          tissue = !chunk_white(w, a.wm, a.we) && classify(w);
        } else if (SPCN_CHECK(p.src_off >= 0 && p.src_off + 3 * (int64_t)p.n <= s_g.src_bytes,
                              s_g.err)) {
          dpart = staged_partial(s_g.src + p.src_off, p.n, lut, lr, s_L, s_t.C, c_nw, c_b0, c_b1);
        }
      }
      warp_step(tissue, w, (unsigned)q);
      if (__any_sync(0xFFFFFFFFu, dpart != 0u))
        staged_queue(dpart, (unsigned)q, s_queue, qn, s_g, lut, lr, s_L, s_t, s_kb, kc0, kc1);
    }
    staged_counts(s_t.sel, c_nw, c_b0, c_b1);
    __syncthreads();   // the item is done: s_items and s_piece may be rewritten
  }
}

template <class G>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_p1(BatchArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  p1_phase<G>(a, s_dyn);
}

// The percentiles of every tile from its key lists (staged schedule).
__global__ void __launch_bounds__(kBatchThreads) k_batch_sel(BatchArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ u64 s_tmp[33];
  for (unsigned t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    batch_select(a, t, reinterpret_cast<unsigned*>(s_dyn), s_tmp);
    __syncthreads();
  }
}

// ------------------------------------------------------------ grid-wide select
// The staged schedule's per-tile select in three launches, so that a large
// tile's lists are read by the whole grid rather than by one block:
//   k_sel_first  one block per tile: the ranks, and for each track the bin of
//                the pass-1 first-digit histogram that holds its rank (tiles
//                without tissue, or with no rank in the lists, are finished
//                here); the tile's second-digit histograms zeroed;
//   k_sel_count  the whole grid: every list in segments of kSelSeg keys,
//                each key of a track's bin counted in that track's
//                second-digit histogram (tracks of one stain that share the
//                bin share the histogram);
//   k_sel_final  one block per tile: the second digits, the percentiles and
//                the pass-2 coefficients, exactly as batch_select.
constexpr int kSelThreads = 512;
constexpr int kSelSeg = 4096;             // keys per segment of k_sel_count
static_assert(kSelSeg % (4 * kSelThreads) == 0, "whole vectors per thread");
constexpr int kGridSelMaxTiles = 1024;    // second-digit histograms: 64 KB per tile

__device__ __forceinline__ void finish_no_tissue(const BatchArgs& a, unsigned tile) {
  const BatchTile* T = a.tiles + tile;
  BatchTileState* S = a.state + tile;
  SelectState* s = &S->sel;
  S->status = SPCN_ERR_NO_TISSUE;
  for (int t = 0; t < kTracks; ++t) { s->key[t] = 0; s->resolved[t] = 1; }
  s->p99[0] = s->p99[1] = 0.0;
  s->scale[0] = s->scale[1] = 1.0;
  s->t = 0.0;
  s->all_resolved = 1;
  const float hs = a.models[T->model].lasso.hscale;
  for (int i = 0; i < 6; ++i) S->M[i] = recon_coef(a.Wt, s->scale, hs, i);
  __threadfence();
  st_release_s32(&S->ready, 1);
}

// Shared memory of the per-tile select steps (static arrays of k_sel_first
// and k_sel_final, carved from the dynamic shared memory of the persistent
// launch).
struct SelSmem {
  unsigned hist[kSelBins];
  u64 tmp[33];
  u64 before;
  u64 rr[kTracks];
  int bin[kTracks];
  int res[kTracks];
  int idx;
};

__device__ void sel_first_tiles(const BatchArgs& a, SelSmem& sm) {
  unsigned (&s_hist)[kSelBins] = sm.hist;
  u64 (&s_tmp)[33] = sm.tmp;
  int& s_idx = sm.idx;
  u64& s_before = sm.before;
  int (&s_bin)[kTracks] = sm.bin;
  u64 (&s_rr)[kTracks] = sm.rr;
  for (unsigned tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const BatchTile* T = a.tiles + tile;
    BatchTileState* S = a.state + tile;
    SelectState* s = &S->sel;
    const u64 n = __ldcg(&s->n_nw);
    if (n == 0) {   // uniform across the block
      if (threadIdx.x == 0) finish_no_tissue(a, tile);
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      set_ranks(s, n, a.pct);
      for (int j = 0; j < 2; ++j) { s->lo[j] = T->lo[j]; s->nb[j] = 0u; }
      for (int t = 0; t < kTracks; ++t) { s_bin[t] = -1; s_rr[t] = s->rank[t]; }
    }
    __syncthreads();
    for (int j = 0; j < 2; ++j) {
      const u64 cnt = __ldcg(&S->list_n[j]);
      const u64 below = __ldcg(&s->below[j]);
      bool in[2];
      for (int u = 0; u < 2; ++u) {
        const u64 r = s_rr[2 * j + u];
        in[u] = T->win[j] && cnt <= T->list_cap && r >= below && r - below < cnt;
      }
      if (!in[0] && !in[1]) continue;   // uniform across the block
      const unsigned* h1 = a.hist1 + ((size_t)tile * 2 + j) * kSelBins;
      for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) s_hist[i] = __ldcg(h1 + i);
      __syncthreads();
      for (int u = 0; u < 2; ++u) {
        if (!in[u]) continue;
        smem_find_rank(s_hist, kSelBins, s_rr[2 * j + u] - below, &s_idx, &s_before, s_tmp);
        if (threadIdx.x == 0 && s_idx >= 0 && s_idx < kSelBins - 1) {
          s_bin[2 * j + u] = s_idx;
          s_rr[2 * j + u] = s_rr[2 * j + u] - below - s_before;
        }
        __syncthreads();
      }
    }
    // zero the histograms the count will fill (a stain's second track shares
    // the first one's when both lie in the same bin)
    for (int t = 0; t < kTracks; ++t) {
      const bool own = s_bin[t] >= 0 && !((t & 1) && s_bin[t] == s_bin[t - 1]);
      if (!own) continue;   // uniform
      unsigned* h2 = a.hist2 + ((size_t)tile * kTracks + t) * kSelBins;
      for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) h2[i] = 0u;
    }
    if (threadIdx.x == 0) {
      int any = 0;
      for (int t = 0; t < kTracks; ++t) {
        S->sbin[t] = s_bin[t];
        S->srank[t] = s_rr[t];
        any |= s_bin[t] >= 0;
        s->resolved[t] = 0;
      }
      if (!any) {   // nothing in the lists: the exact fallback
        s->all_resolved = 0;
        atomicAdd(&a.run->n_fallback, 1u);
        __threadfence();
        st_release_s32(&S->ready, 2);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_first(BatchArgs a) {
  __shared__ SelSmem sm;
  sel_first_tiles(a, sm);
}

// Pair metadata of k_sel_count, one per (tile, stain).
struct SelPair {
  unsigned lo;
  int b0, b1;      // first-digit bins of the stain's two tracks (-1: none)
  unsigned n;      // listed keys (0: nothing to count)
};

__device__ __forceinline__ unsigned sel_segments(unsigned n) {
  return (n + kSelSeg - 1) / kSelSeg;
}

// Every list in segments of kSelSeg keys, numbered over all pairs (a block
// scan gives each pair's first segment); block b takes segments b, b + G, ...
// and finds a segment's pair by binary search.
__device__ void sel_count_segments(const BatchArgs& a, char* s_dyn, u64* s_tmp) {
  const unsigned np = 2 * a.n_tiles;
  SelPair* s_pair = reinterpret_cast<SelPair*>(s_dyn);
  unsigned* s_seg = reinterpret_cast<unsigned*>(s_pair + np);   // np + 1 entries
  const unsigned per = (np + blockDim.x - 1) / blockDim.x;
  const unsigned p0 = min(np, threadIdx.x * per), p1 = min(np, p0 + per);
  unsigned local = 0;
  for (unsigned p = p0; p < p1; ++p) {
    const unsigned tile = p >> 1, j = p & 1u;
    const BatchTileState* S = a.state + tile;
    SelPair sp;
    sp.lo = a.tiles[tile].lo[j];
    sp.b0 = __ldcg(&S->sbin[2 * j]);
    sp.b1 = __ldcg(&S->sbin[2 * j + 1]);
    const u64 cnt = __ldcg(&S->list_n[j]);
    sp.n = (__ldcg(&S->ready) == 0 && (sp.b0 >= 0 || sp.b1 >= 0)) ? (unsigned)cnt : 0u;
    s_pair[p] = sp;
    local += sel_segments(sp.n);
  }
  u64 total = 0;
  unsigned run = (unsigned)block_excl_scan((u64)local, s_tmp, &total);
  for (unsigned p = p0; p < p1; ++p) {
    s_seg[p] = run;
    run += sel_segments(s_pair[p].n);
  }
  if (threadIdx.x == 0) s_seg[np] = (unsigned)total;
  __syncthreads();
  for (unsigned gs = blockIdx.x; gs < (unsigned)total; gs += gridDim.x) {
    // the pair: the last p with s_seg[p] <= gs (it holds segments)
    unsigned lo = 0u, hi = np;   // s_seg[lo] <= gs < s_seg[hi]
    while (hi - lo > 1u) {
      const unsigned mid = (lo + hi) >> 1;
      if (s_seg[mid] <= gs) lo = mid; else hi = mid;
    }
    const unsigned p = lo, k = gs - s_seg[p];
    const SelPair sp = s_pair[p];
    const unsigned tile = p >> 1, j = p & 1u;
    const unsigned* list = a.tiles[tile].keys + (u64)j * a.tiles[tile].list_cap;
    unsigned* h0 = a.hist2 + ((size_t)tile * kTracks + 2 * j) * kSelBins;
    unsigned* h1 = (sp.b1 >= 0 && sp.b1 != sp.b0) ? h0 + kSelBins : h0;
    auto count = [&](unsigned key) {
      const unsigned d = key - sp.lo;
      const int hb = (int)min(d >> kSelBits, (unsigned)(kSelBins - 1));
      const unsigned low = d & (kSelBins - 1);
      if (hb == sp.b0) red_add_u32(h0 + low, 1u);
      else if (hb == sp.b1) red_add_u32(h1 + low, 1u);
    };
    // the segment's keys as 16-byte vectors (lists and segments start on
    // 16-byte boundaries), every load issued before the counting; a last
    // partial vector key by key
    const unsigned i0 = k * kSelSeg, i1 = min(sp.n, i0 + kSelSeg);
    const uint4* v = reinterpret_cast<const uint4*>(list + i0);
    const unsigned nv = (i1 - i0) / 4;
    constexpr int kVec = kSelSeg / 4 / kSelThreads;   // vectors per thread
    uint4 x[kVec];
#pragma unroll
    for (int r = 0; r < kVec; ++r) {
      const unsigned vi = threadIdx.x + (unsigned)r * blockDim.x;
      x[r] = vi < nv ? __ldcg(v + vi) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int r = 0; r < kVec; ++r) {
      if (threadIdx.x + (unsigned)r * blockDim.x < nv) {
        count(x[r].x); count(x[r].y); count(x[r].z); count(x[r].w);
      }
    }
    for (unsigned i = i0 + 4 * nv + threadIdx.x; i < i1; i += blockDim.x) count(__ldcg(list + i));
  }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_count(BatchArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ u64 s_tmp[33];
  sel_count_segments(a, s_dyn, s_tmp);
}

__device__ void sel_final_tiles(const BatchArgs& a, SelSmem& sm) {
  unsigned (&s_hist)[kSelBins] = sm.hist;
  u64 (&s_tmp)[33] = sm.tmp;
  int& s_idx = sm.idx;
  u64& s_before = sm.before;
  int (&s_res)[kTracks] = sm.res;
  for (unsigned tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const BatchTile* T = a.tiles + tile;
    BatchTileState* S = a.state + tile;
    SelectState* s = &S->sel;
    if (__ldcg(&S->ready) != 0) continue;   // finished by k_sel_first (uniform)
    if (threadIdx.x < kTracks) s_res[threadIdx.x] = 0;
    for (int t = 0; t < kTracks; ++t) {
      const int bin = __ldcg(&S->sbin[t]);
      if (bin < 0) continue;   // uniform
      const int src = ((t & 1) && bin == __ldcg(&S->sbin[t - 1])) ? t - 1 : t;
      const unsigned* h2 = a.hist2 + ((size_t)tile * kTracks + src) * kSelBins;
      __syncthreads();
      for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) s_hist[i] = __ldcg(h2 + i);
      __syncthreads();
      smem_find_rank(s_hist, kSelBins, __ldcg(&S->srank[t]), &s_idx, &s_before, s_tmp);
      if (threadIdx.x == 0 && s_idx >= 0) {
        s->key[t] = T->lo[t >> 1] + ((unsigned)bin << kSelBits) + (unsigned)s_idx;
        s_res[t] = 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int t = 0; t < kTracks; ++t) { s->resolved[t] = s_res[t]; all &= s_res[t]; }
      if (all) {
        const float hs = a.models[T->model].lasso.hscale;
        finish_percentiles(s, a.tgt0, a.tgt1, hs);
        for (int i = 0; i < 6; ++i) S->M[i] = recon_coef(a.Wt, s->scale, hs, i);
      }
      s->all_resolved = all;
      if (!all) atomicAdd(&a.run->n_fallback, 1u);
      __threadfence();
      st_release_s32(&S->ready, all ? 1 : 2);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_final(BatchArgs a) {
  __shared__ SelSmem sm;
  sel_final_tiles(a, sm);
}

// Pass 2 of every tile whose percentile the lists gave (staged schedule).
// The work per chunk is the same everywhere, so the chunks of all tiles (the
// tiles in table order) are split into equal contiguous shares, one per
// block, each a short list of segments (chunk ranges of one tile) built when
// the batch is created: a block crosses few tile boundaries, loads a table
// when the model changes and streams its share without waits between items.  For batches of
// at most kP2PreloadTiles tiles every tile's coefficients are read into
// shared memory once.
struct P2Tile {
  float M[6];
  int go;          // 1: the percentile is known (else the exact fallback finishes the tile)
};
constexpr int kP2PreloadTiles = 2048;
constexpr size_t kP2Smem = kLutSmemBytes + sizeof(P2Tile) * kP2PreloadTiles;

template <class G>
__device__ __forceinline__ void p2_phase(const BatchArgs& a, char* s_dyn) {
  char* lut = s_dyn;
  P2Tile* s_tiles = reinterpret_cast<P2Tile*>(s_dyn + kLutSmemBytes);
  __shared__ __align__(16) BatchItem s_items[2];   // current segment and the prefetched next one
  __shared__ P2Tile s_one;                          // the current tile's, without preloading
  const bool pre = a.n_tiles <= (unsigned)kP2PreloadTiles;
  int cur_model = -1, cur = 0;
  // thread 0 walks the block's segments, copying the next descriptor into
  // shared memory one segment ahead
  unsigned i_next = 0u, i_end = 0u;
  if (threadIdx.x == 0) {
    i_next = a.p2_first[blockIdx.x];
    i_end = a.p2_first[blockIdx.x + 1];
    if (i_next < i_end) copy_item_async(&s_items[1], a.p2_items + i_next++);
    else s_items[1].tile = ~0u;
  }
  if (pre) {
    for (unsigned t = threadIdx.x; t < a.n_tiles; t += blockDim.x) {
      const BatchTileState* S = a.state + t;
      P2Tile pt;
      pt.go = __ldcg(&S->ready) == 1;
#pragma unroll
      for (int i = 0; i < 6; ++i) pt.M[i] = pt.go ? __ldcg(&S->M[i]) : 0.f;
      s_tiles[t] = pt;
    }
  }
  for (;;) {
    cur ^= 1;
    if (threadIdx.x == 0) {
      cp_async_wait_all();
      BatchItem* nx = &s_items[cur ^ 1];   // read by nobody until the next loop top
      const unsigned tile = s_items[cur].tile;
      if (tile != ~0u && i_next < i_end) copy_item_async(nx, a.p2_items + i_next++);
      else nx->tile = ~0u;
      if (!pre && tile != ~0u) {
        const BatchTileState* S = a.state + tile;
        s_one.go = __ldcg(&S->ready) == 1;
        for (int i = 0; i < 6; ++i) s_one.M[i] = s_one.go ? __ldcg(&S->M[i]) : 0.f;
      }
    }
    __syncthreads();
    const BatchItem item = s_items[cur];
    if (item.tile == ~0u) break;
    const P2Tile* pt = pre ? s_tiles + item.tile : &s_one;
    if (pt->go) {
      if ((int)item.model != cur_model) {
        load_od_lut(a.models + item.model, lut);   // ends with a block barrier
        cur_model = (int)item.model;
      }
      batch_pass2<G>(a, item.tile, item.c0, item.c1, lut, pt->M);
    }
    __syncthreads();   // the segment is done: shared words and the table may be rewritten
  }
}

template <class G>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_p2(BatchArgs a) {
  extern __shared__ __align__(16) char s_dyn[];
  p2_phase<G>(a, s_dyn);
}

// ------------------------------------------------------------ persistent schedule
// SPCN_SCHED_PERSISTENT: the staged schedule's steps as phases of ONE
// cooperative persistent launch (one block per SM), separated by grid
// barriers instead of kernel boundaries: window starts, pass 1, the three
// select steps, pass 2.  Each phase reuses the block's dynamic shared memory
// (the pass-1 layout is the largest).  Data written in one phase is read in
// the next after the barrier's acquire.  The exact fallback of tiles whose
// ranks missed their window stays a separate cooperative launch that returns
// at once when no tile needs it.
template <class G>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_persist(BatchArgs a, PilotArgs pa) {
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ u64 s_tmp[33];
  unsigned target = 0;
  auto sync_grid = [&]() -> bool {
    target += gridDim.x;
    return grid_barrier(&a.run->barrier2, target, &a.run->abort, &a.run->err, a.timeout_ns);
  };
  pilot_tiles(pa, *reinterpret_cast<PilotSmem*>(s_dyn));
  if (!sync_grid()) return;
  p1_phase<G>(a, s_dyn);
  if (!sync_grid()) return;
  sel_first_tiles(a, *reinterpret_cast<SelSmem*>(s_dyn));
  if (!sync_grid()) return;
  sel_count_segments(a, s_dyn, s_tmp);
  if (!sync_grid()) return;
  sel_final_tiles(a, *reinterpret_cast<SelSmem*>(s_dyn));
  if (!sync_grid()) return;
  p2_phase<G>(a, s_dyn);
}

// ------------------------------------------------------------ host side
struct Batch {
  Context* c = nullptr;
  int n = 0;
  std::vector<BatchTile> tiles;
  std::vector<int> tile_status;
  int n_models = 0;
  Model* models = nullptr;
  BatchTile* d_tiles = nullptr;
  BatchItem* d_items = nullptr;
  size_t items_cap = 0;
  unsigned n_items = 0;
  char* d_state = nullptr;       // BatchRunState, then n BatchTileState
  size_t state_bytes = 0;
  unsigned* keys = nullptr;
  unsigned* hist2 = nullptr;     // grid-wide select (batches of at most kGridSelMaxTiles)
  BatchItem* p1_items = nullptr; // staged pass 1: each block's segments
  unsigned* p1_first = nullptr;
  BatchItem* p2_items = nullptr; // staged pass 2: each block's segments
  unsigned* p2_first = nullptr;
  u64* rhist = nullptr;
  int grid = 0;
  int grid_p1 = 0, grid_p2 = 0, grid_sel = 0;   // staged schedule
  bool persist_ok = false;       // the persistent schedule can run (see configure_persist)
  u64 max_chunks = 0;            // chunks of the largest tile
  bool flat = false;             // every tile contiguous: launch the flat instantiation
  BatchArgs args{};
  spcn_batch_config cfg{};
};

constexpr size_t kRunStateBytes = (sizeof(BatchRunState) + 255) & ~size_t(255);

template <class G>
static int configure_batch_kernel(Context* c, int* grid) {
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_batch<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kBatchSmem));
  int occ = 0;
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<G>, kBatchThreads,
                                                              kBatchSmem));
  if (occ < 1) return SPCN_ERR_CUDA;
  *grid = c->num_sms * occ;
  return SPCN_OK;
}

template <class G>
static int configure_staged_kernels(Context* c, int* grid_p1, int* grid_p2) {
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_batch_p1<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kStagedSmem));
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_batch_p2<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kP2Smem));
  int o1 = 0, o2 = 0;
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_batch_p1<G>, kBatchThreads,
                                                              kStagedSmem));
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_batch_p2<G>, kBatchThreads,
                                                              kP2Smem));
  if (o1 < 1 || o2 < 1) return SPCN_ERR_CUDA;
  *grid_p1 = c->num_sms * o1;
  *grid_p2 = c->num_sms * o2;
  return SPCN_OK;
}

// The persistent launch holds the pass-1 layout (the largest of its phases'
// shared memory) with one block per SM; its pass 1 and pass 2 take the
// static shares built for grid_p1 and grid_p2 blocks, so both must equal its
// grid, and its select is the grid-wide one (batches with hist2).
template <class G>
static int configure_persist(Context* c, Batch* b) {
  b->persist_ok = false;
  SPCN_CUDA_TRY(cudaFuncSetAttribute(k_batch_persist<G>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedSmem));
  int occ = 0;
  SPCN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_persist<G>,
                                                              kBatchThreads, kStagedSmem));
  const size_t sel_count_smem = (sizeof(SelPair) + sizeof(unsigned)) * 2 * (size_t)b->n + 4;
  const size_t p2_smem =
      kLutSmemBytes + (b->n <= kP2PreloadTiles ? sizeof(P2Tile) * (size_t)b->n : 0);
  b->persist_ok = occ >= 1 && b->grid_p1 == c->num_sms && b->grid_p2 == c->num_sms &&
                  b->hist2 != nullptr && sel_count_smem <= kStagedSmem && p2_smem <= kStagedSmem &&
                  sizeof(PilotSmem) <= kStagedSmem && sizeof(SelSmem) <= kStagedSmem &&
                  b->max_chunks < (1ull << 32);
  return SPCN_OK;
}

static bool config_ok(const spcn_batch_config* cfg) {
  if (!cfg) return false;
  if (cfg->item_chunks < kPassThreads || cfg->item_chunks % kPassThreads != 0) return false;
  if (cfg->schedule != SPCN_SCHED_PHASED && cfg->schedule != SPCN_SCHED_INTERLEAVED &&
      cfg->schedule != SPCN_SCHED_STAGED && cfg->schedule != SPCN_SCHED_PERSISTENT)
    return false;
  if (cfg->schedule == SPCN_SCHED_INTERLEAVED && cfg->group_px < 1) return false;
  return true;
}

// Tiles grouped by table (tables in the order of their largest tile), largest
// first within a table.
static std::vector<int> table_order(const Batch* b) {
  std::vector<int> order(b->n);
  for (int t = 0; t < b->n; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->tiles[x].g.npx > b->tiles[y].g.npx;
  });
  std::vector<int> rank(b->n_models, -1), order2 = order;
  int r = 0;
  for (int t : order)
    if (rank[b->tiles[t].model] < 0) rank[b->tiles[t].model] = r++;
  std::stable_sort(order2.begin(), order2.end(), [&](int x, int y) {
    return rank[b->tiles[x].model] < rank[b->tiles[y].model];
  });
  return order2;
}

// Work queue of a schedule.  Every pass-1 item of a tile precedes the tile's
// pass-2 items (the kernel's waits rely on it).
static void build_items(const Batch* b, const spcn_batch_config& cfg, std::vector<BatchItem>* out,
                        std::vector<unsigned>* n_items1) {
  const u64 S = (u64)cfg.item_chunks;
  out->clear();
  n_items1->assign(b->n, 0u);
  // the staged passes take static shares (build_shares), not queue items
  if (cfg.schedule == SPCN_SCHED_STAGED || cfg.schedule == SPCN_SCHED_PERSISTENT) return;
  // largest tiles first: their list selects end early, and the small tiles
  // even out the end of each pass
  std::vector<int> order(b->n);
  for (int t = 0; t < b->n; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->tiles[x].g.npx > b->tiles[y].g.npx;
  });
  auto emit = [&](int t, unsigned pass) {
    const u64 nch = b->tiles[t].g.nchunks;
    const unsigned n1 = (unsigned)((nch + S - 1) / S);
    for (u64 c0 = 0; c0 < nch; c0 += S)
      out->push_back({(unsigned)t, pass, b->tiles[t].model, n1, c0, std::min(nch, c0 + S)});
    if (pass == 1) (*n_items1)[t] = n1;
  };
  if (cfg.schedule == SPCN_SCHED_PHASED) {
    // pass 2 needs no particular order: tiles sharing a table go together
    // (fewer table reloads), largest first within a table
    const std::vector<int> order2 = table_order(b);
    for (int t : order) emit(t, 1);
    for (int t : order2) emit(t, 2);
    return;
  }
  // groups of consecutive tiles (in size order) holding about group_px pixels
  std::vector<std::pair<int, int>> groups;
  int start = 0;
  int64_t px = 0;
  for (int k = 0; k < b->n; ++k) {
    px += b->tiles[order[k]].g.npx;
    if (px >= cfg.group_px || k == b->n - 1) {
      groups.push_back({start, k + 1});
      start = k + 1;
      px = 0;
    }
  }
  for (size_t k = 0; k <= groups.size(); ++k) {
    if (k < groups.size())
      for (int i = groups[k].first; i < groups[k].second; ++i) emit(order[i], 1);
    if (k >= 1)
      for (int i = groups[k - 1].first; i < groups[k - 1].second; ++i) emit(order[i], 2);
  }
}

static int apply_config(Batch* b, const spcn_batch_config& cfg) {
  // the staged pass 1 queues 32-bit chunk indices of a tile
  if (cfg.schedule == SPCN_SCHED_STAGED && b->max_chunks >= (1ull << 32)) return SPCN_ERR_INVALID_ARG;
  if (cfg.schedule == SPCN_SCHED_PERSISTENT && !b->persist_ok) return SPCN_ERR_INVALID_ARG;
  std::vector<BatchItem> items;
  std::vector<unsigned> n1;
  build_items(b, cfg, &items, &n1);
  if (items.size() > 0xFFFFFFF0ull) return SPCN_ERR_INVALID_ARG;
  if (items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    SPCN_CUDA_TRY(cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem)));
    b->items_cap = items.size();
  }
  for (int t = 0; t < b->n; ++t) b->tiles[t].n_items1 = n1[t];
  if (!items.empty())
    SPCN_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem),
                             cudaMemcpyHostToDevice));
  SPCN_CUDA_TRY(cudaMemcpy(b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(BatchTile),
                           cudaMemcpyHostToDevice));
  // a pageable copy may return before it lands: finish it before any launch
  SPCN_CUDA_TRY(cudaDeviceSynchronize());
  b->n_items = (unsigned)items.size();
  b->args.items = b->d_items;
  b->args.n_items = b->n_items;
  b->cfg = cfg;
  b->cfg.ms = 0.f;
  return SPCN_OK;
}

static void batch_free(Batch* b) {
  void* ptrs[] = {b->models, b->d_tiles, b->d_items, b->d_state, b->keys, b->hist2,
                  b->p1_items, b->p1_first, b->p2_items, b->p2_first, b->rhist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

static int batch_launch(Batch* b, cudaStream_t st) {
  Context* c = b->c;
  SPCN_CUDA_TRY(cudaMemsetAsync(b->d_state, 0, b->state_bytes, st));
  const bool persist = b->cfg.schedule == SPCN_SCHED_PERSISTENT;
  PilotArgs pa;
  pa.tiles = b->d_tiles;
  pa.models = b->models;
  pa.n_tiles = (unsigned)b->n;
  pa.thr = b->args.thr;
  pa.pct = b->args.pct;
  if (!persist) {   // the persistent launch sets the window starts itself
    const int pg = std::min(b->n, 4 * c->num_sms);
    k_batch_pilot<<<pg, kPilotThreads, 0, st>>>(pa);
    SPCN_LAUNCH_CHECK(c);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SPCN_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  const bool staged = b->cfg.schedule == SPCN_SCHED_STAGED;
  // staged and persistent: the fused kernel runs with an empty queue (only
  // the exact fallback of tiles whose ranks missed their window)
  BatchArgs fa = b->args;
  if (staged || persist) fa.n_items = 0;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)b->grid);
  lc.blockDim = dim3(kBatchThreads);
  lc.dynamicSmemBytes = kBatchSmem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  int launched = 0;
  // contiguous tiles only: the flat traversal (fewer registers per loop)
  auto launch = [&]() -> cudaError_t {
    if (persist) {
      cudaLaunchConfig_t pc = lc;
      pc.gridDim = dim3((unsigned)c->num_sms);
      pc.dynamicSmemBytes = kStagedSmem;
      const cudaError_t e0 =
          b->flat ? cudaLaunchKernelEx(&pc, k_batch_persist<FlatGeometry>, b->args, pa)
                  : cudaLaunchKernelEx(&pc, k_batch_persist<Geometry>, b->args, pa);
      if (e0 != cudaSuccess) return e0;
      ++launched;
    }
    if (staged) {
      if (b->flat)
        k_batch_p1<FlatGeometry><<<b->grid_p1, kBatchThreads, kStagedSmem, st>>>(b->args);
      else
        k_batch_p1<Geometry><<<b->grid_p1, kBatchThreads, kStagedSmem, st>>>(b->args);
      ++launched;
      if (b->hist2) {
        k_sel_first<<<b->grid_sel, kSelThreads, 0, st>>>(b->args);
        k_sel_count<<<2 * c->num_sms, kSelThreads,
                      (sizeof(SelPair) + sizeof(unsigned)) * 2 * b->n + sizeof(unsigned), st>>>(
            b->args);
        k_sel_final<<<b->grid_sel, kSelThreads, 0, st>>>(b->args);
        launched += 3;
      } else {
        k_batch_sel<<<b->grid_sel, kBatchThreads, kSelectSmem, st>>>(b->args);
        ++launched;
      }
      const size_t p2_smem =
          kLutSmemBytes + (b->n <= kP2PreloadTiles ? sizeof(P2Tile) * (size_t)b->n : 0);
      if (b->flat)
        k_batch_p2<FlatGeometry><<<b->grid_p2, kBatchThreads, p2_smem, st>>>(b->args);
      else
        k_batch_p2<Geometry><<<b->grid_p2, kBatchThreads, p2_smem, st>>>(b->args);
      ++launched;
      const cudaError_t e0 = cudaGetLastError();
      if (e0 != cudaSuccess) return e0;
    }
    ++launched;
    return b->flat ? cudaLaunchKernelEx(&lc, k_batch<FlatGeometry>, fa)
                   : cudaLaunchKernelEx(&lc, k_batch<Geometry>, fa);
  };
  cudaError_t e;
  if (cap == cudaStreamCaptureStatusNone) {
    TimedLaunch tl(c, SPCN_KERNEL_BATCH, st);
    e = launch();
  } else {
    e = launch();
  }
  c->launches += launched;
  if (e != cudaSuccess) return SPCN_ERR_CUDA;
  return SPCN_OK;
}

// The staged passes' static schedule: the chunks of all tiles (in table
// order) in equal contiguous shares, one per block of a grid of `grid`
// blocks, each cut at tile boundaries into segments; block b's segments are
// (*items)[(*first)[b] .. (*first)[b + 1]).  A block crosses few tile and
// table boundaries and takes no tickets.
static int build_shares(Batch* b, int grid, unsigned pass, BatchItem** items, unsigned** first) {
  const std::vector<int> ord = table_order(b);
  u64 total = 0;
  for (int t : ord) total += b->tiles[t].g.nchunks;
  std::vector<BatchItem> segs;
  std::vector<unsigned> fst(grid + 1);
  size_t k = 0;
  u64 tile0 = 0;   // first chunk of tile ord[k] in the order
  for (int blk = 0; blk < grid; ++blk) {
    fst[blk] = (unsigned)segs.size();
    u64 c = total * (u64)blk / (u64)grid;
    const u64 e = total * (u64)(blk + 1) / (u64)grid;
    while (c < e) {
      while (tile0 + b->tiles[ord[k]].g.nchunks <= c) tile0 += b->tiles[ord[k++]].g.nchunks;
      const BatchTile& T = b->tiles[ord[k]];
      const u64 stop = std::min(e, tile0 + T.g.nchunks);
      segs.push_back({(unsigned)ord[k], pass, T.model, 0u, c - tile0, stop - tile0});
      c = stop;
    }
  }
  fst[grid] = (unsigned)segs.size();
  if (cudaMalloc(items, sizeof(BatchItem) * std::max<size_t>(1, segs.size())) != cudaSuccess ||
      cudaMalloc(first, sizeof(unsigned) * fst.size()) != cudaSuccess)
    return SPCN_ERR_OOM;
  if ((!segs.empty() && cudaMemcpy(*items, segs.data(), sizeof(BatchItem) * segs.size(),
                                   cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(*first, fst.data(), sizeof(unsigned) * fst.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return SPCN_ERR_CUDA;
  return SPCN_OK;
}

static int batch_create(Context* c, int n, const spcn_image* tiles, const spcn_stats* tile_stats,
                        const spcn_stats* tgt, const spcn_params* params, uint8_t* const* outs,
                        const int64_t* out_pitches, Batch** out) {
  Batch* b = new (std::nothrow) Batch();
  if (!b) return SPCN_ERR_OOM;
  b->c = c;
  b->n = n;
  b->tiles.resize(n);
  // one table per distinct (W, i0): tiles of one slide share it
  std::vector<int> rep;   // first tile of each table
  u64 keys_total = 0;
  for (int t = 0; t < n; ++t) {
    BatchTile& T = b->tiles[t];
    memset(&T, 0, sizeof(T));
    T.g = make_geometry(&tiles[t], outs[t], out_pitches[t], c->err);
    int m = -1;
    for (size_t k = 0; k < rep.size() && m < 0; ++k)
      if (memcmp(tile_stats[rep[k]].W, tile_stats[t].W, sizeof(float) * 6) == 0 &&
          memcmp(tile_stats[rep[k]].i0, tile_stats[t].i0, sizeof(float) * 3) == 0)
        m = (int)k;
    if (m < 0) {
      m = (int)rep.size();
      rep.push_back(t);
    }
    T.model = (unsigned)m;
    const int hexp = host_table_hexp(tile_stats[t].W, tile_stats[t].i0, params->lambda);
    const double hs = ldexp(1.0, -hexp);
    for (int j = 0; j < 2; ++j) {
      const double h = tile_stats[t].p99[j] * hs * kOpenLow;
      float f = (float)h;
      unsigned key = 0u;
      memcpy(&key, &f, 4);
      const float fh = (float)(tile_stats[t].p99[j] * hs);
      memcpy(&T.hkey[j], &fh, 4);
      if (h > 0x1p-100 && std::isfinite(h) && key > 0u) {
        T.win[j] = 1u;
        T.lo[j] = key;
        below_consts(key, &T.nk[j], &T.lk[j]);
      } else {   // no window: [h~ < lo] is 1 for every pixel, nothing is listed
        T.win[j] = 0u;
        T.lo[j] = 0u;
        T.nk[j] = 0.f;
        T.lk[j] = 1.f;
      }
      T.hlo[j] = T.lo[j];
      T.hwin[j] = T.win[j];
      T.hnk[j] = T.nk[j];
      T.hlk[j] = T.lk[j];
    }
    // room for 1/8 of the pixels per stain (a window from 0.75 P99 holds a
    // few percent; an overflowing list sends the tile to the exact fallback)
    T.list_cap = ((u64)T.g.npx / 8 + 1024 + 3) & ~u64(3);
    T.keys = reinterpret_cast<unsigned*>((uintptr_t)keys_total);   // offset until allocated
    keys_total += 2 * T.list_cap;
  }
  b->n_models = (int)rep.size();
  int rc = SPCN_OK;
  auto fail = [&](int code) { batch_free(b); return code; };
  if (cudaMalloc(&b->models, sizeof(Model) * rep.size()) != cudaSuccess) return fail(SPCN_ERR_OOM);
  if (cudaMalloc(&b->d_tiles, sizeof(BatchTile) * n) != cudaSuccess) return fail(SPCN_ERR_OOM);
  b->state_bytes = kRunStateBytes + sizeof(BatchTileState) * (size_t)n +
                   sizeof(unsigned) * 2 * kSelBins * (size_t)n;
  if (cudaMalloc(&b->d_state, b->state_bytes) != cudaSuccess) return fail(SPCN_ERR_OOM);
  if (cudaMalloc(&b->keys, sizeof(unsigned) * keys_total) != cudaSuccess) return fail(SPCN_ERR_OOM);
  for (BatchTile& T : b->tiles) T.keys = b->keys + reinterpret_cast<uintptr_t>(T.keys);
  if (cudaMalloc(&b->rhist, sizeof(u64) * 3 * kTracks * kRadixBins) != cudaSuccess)
    return fail(SPCN_ERR_OOM);
  if (n <= kGridSelMaxTiles &&
      cudaMalloc(&b->hist2, sizeof(unsigned) * kTracks * kSelBins * (size_t)n) != cudaSuccess)
    return fail(SPCN_ERR_OOM);
  for (size_t k = 0; k < rep.size(); ++k) {
    rc = launch_build_model(c, b->models + k, tile_stats[rep[k]].W, tile_stats[rep[k]].i0,
                            params->lambda, nullptr, nullptr);
    if (rc) return fail(rc);
  }
  b->flat = true;
  for (const BatchTile& T : b->tiles) {
    b->flat = b->flat && T.g.flat;
    b->max_chunks = std::max(b->max_chunks, (u64)T.g.nchunks);
  }
  rc = b->flat ? configure_batch_kernel<FlatGeometry>(c, &b->grid)
               : configure_batch_kernel<Geometry>(c, &b->grid);
  if (rc) return fail(rc);
  rc = b->flat ? configure_staged_kernels<FlatGeometry>(c, &b->grid_p1, &b->grid_p2)
               : configure_staged_kernels<Geometry>(c, &b->grid_p1, &b->grid_p2);
  if (rc) return fail(rc);
  b->grid_sel = std::min(n, 4 * c->num_sms);
  rc = build_shares(b, b->grid_p1, 1u, &b->p1_items, &b->p1_first);
  if (rc == SPCN_OK) rc = build_shares(b, b->grid_p2, 2u, &b->p2_items, &b->p2_first);
  if (rc == SPCN_OK)
    rc = b->flat ? configure_persist<FlatGeometry>(c, b) : configure_persist<Geometry>(c, b);
  if (rc) return fail(rc);
  BatchArgs& a = b->args;
  a.tiles = b->d_tiles;
  a.state = reinterpret_cast<BatchTileState*>(b->d_state + kRunStateBytes);
  a.hist1 = reinterpret_cast<unsigned*>(b->d_state + kRunStateBytes +
                                        sizeof(BatchTileState) * (size_t)n);
  a.hist2 = b->hist2;
  a.p1_items = b->p1_items;
  a.p1_first = b->p1_first;
  a.p2_items = b->p2_items;
  a.p2_first = b->p2_first;
  a.run = reinterpret_cast<BatchRunState*>(b->d_state);
  a.models = b->models;
  a.rhist = b->rhist;
  a.n_tiles = (unsigned)n;
  a.wthr = ((unsigned)params->white_thresh + 1u) << 8;
  a.thr = (unsigned)params->white_thresh;
  white_test_consts(params->white_thresh, &a.wm, &a.we);
  a.pct = (double)params->stain_pct;
  a.tgt0 = tgt->p99[0];
  a.tgt1 = tgt->p99[1];
  for (int i = 0; i < 6; ++i) a.Wt[i] = tgt->W[i];
  for (int i = 0; i < 3; ++i) a.l2i0[i] = (float)log2((double)tgt->i0[i]);
  a.timeout_ns = c->timeout_ns;
  // default schedule: the staged launches (fastest on the benchmark's
  // 256-tile batch), else the fused one
  spcn_batch_config cfg{};
  const bool staged_ok = b->max_chunks < (1ull << 32);
  cfg.item_chunks = (staged_ok ? 32 : 16) * kPassThreads;
  cfg.schedule = staged_ok ? SPCN_SCHED_STAGED : SPCN_SCHED_PHASED;
  cfg.group_px = 0;
  rc = apply_config(b, cfg);
  if (rc) return fail(rc);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(SPCN_ERR_CUDA);
  *out = b;
  return SPCN_OK;
}

static int batch_results(Batch* b, double* p99_out, int32_t* status_out, int32_t* fallback_out,
                         cudaStream_t st) {
  const size_t bytes = kRunStateBytes + sizeof(BatchTileState) * (size_t)b->n;
  std::vector<char> h(bytes);
  SPCN_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d_state, bytes, cudaMemcpyDeviceToHost, st));
  SPCN_CUDA_TRY(cudaStreamSynchronize(st));
  const BatchRunState* run = reinterpret_cast<const BatchRunState*>(h.data());
  const BatchTileState* ts = reinterpret_cast<const BatchTileState*>(h.data() + kRunStateBytes);
  for (int t = 0; t < b->n; ++t) {
    if (p99_out) {
      p99_out[2 * t] = ts[t].sel.p99[0];
      p99_out[2 * t + 1] = ts[t].sel.p99[1];
    }
    if (status_out) status_out[t] = ts[t].status;
    if (fallback_out) fallback_out[t] = ts[t].fallback;
  }
  return run->err;
}

}  // namespace spcn

using namespace spcn;

extern "C" {

int spcn_batch_create(void* ctx, int32_t n, const spcn_image* tiles, const spcn_stats* tile_stats,
                      const spcn_stats* tgt_st, const spcn_params* params, uint8_t* const* outs,
                      const int64_t* out_pitches, void** batch) {
  if (!ctx || n < 1 || n > (1 << 20) || !tiles || !tile_stats || !tgt_st || !outs ||
      !out_pitches || !batch || !params_ok(params))
    return SPCN_ERR_INVALID_ARG;
  // pass 1 always runs, with the lasso densities
  if (params->flags & (SPCN_FLAG_P99_SAMPLED | SPCN_FLAG_H_PINV)) return SPCN_ERR_INVALID_ARG;
  *batch = nullptr;
  int rc = stats_ok(tgt_st);
  if (rc) return rc;
  for (int t = 0; t < n; ++t) {
    const spcn_image* s = &tiles[t];
    if (!image_ok(s) || !outs[t] || out_pitches[t] < 3ll * s->width) return SPCN_ERR_INVALID_ARG;
    rc = stats_ok(&tile_stats[t]);
    if (rc) return rc;
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(s->data);
    const uintptr_t s1 = s0 + (uintptr_t)((s->height - 1) * s->pitch_bytes + 3ll * s->width);
    const uintptr_t d0 = reinterpret_cast<uintptr_t>(outs[t]);
    const uintptr_t d1 = d0 + (uintptr_t)((s->height - 1) * out_pitches[t] + 3ll * s->width);
    if (d0 < s1 && s0 < d1) return SPCN_ERR_INVALID_ARG;
  }
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  Batch* b = nullptr;
  const spcn_stats to = output_target(tgt_st, params);
  rc = batch_create(c, n, tiles, tile_stats, &to, params, outs, out_pitches, &b);
  if (rc) return rc;
  *batch = b;
  return SPCN_OK;
}

int spcn_batch_run(void* batch, void* stream) {
  if (!batch) return SPCN_ERR_INVALID_ARG;
  Batch* b = static_cast<Batch*>(batch);
  DeviceGuard guard(b->c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  return batch_launch(b, static_cast<cudaStream_t>(stream));
}

int spcn_batch_results(void* batch, double* p99_out, int32_t* status_out, int32_t* fallback_out,
                       void* stream) {
  if (!batch) return SPCN_ERR_INVALID_ARG;
  Batch* b = static_cast<Batch*>(batch);
  DeviceGuard guard(b->c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  return batch_results(b, p99_out, status_out, fallback_out, static_cast<cudaStream_t>(stream));
}

int spcn_batch_get_config(void* batch, spcn_batch_config* cfg) {
  if (!batch || !cfg) return SPCN_ERR_INVALID_ARG;
  *cfg = static_cast<Batch*>(batch)->cfg;
  return SPCN_OK;
}

int spcn_batch_set_config(void* batch, const spcn_batch_config* cfg) {
  if (!batch || !config_ok(cfg)) return SPCN_ERR_INVALID_ARG;
  Batch* b = static_cast<Batch*>(batch);
  DeviceGuard guard(b->c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SPCN_ERR_CUDA;   // no run may read the old queue
  return apply_config(b, *cfg);
}

int spcn_batch_tune(void* batch, int32_t reps, spcn_batch_config* trials, int32_t max_trials,
                    int32_t* n_trials, void* stream) {
  if (!batch || reps < 1 || (trials && max_trials < 0)) return SPCN_ERR_INVALID_ARG;
  Batch* b = static_cast<Batch*>(batch);
  DeviceGuard guard(b->c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // candidates: item sizes (2K-64K chunks) x (phased, interleaved groups of
  // 16 Mpx), sizes above the largest tile's chunk count skipped, and the
  // staged schedule (static shares: the item size does not change it)
  u64 max_chunks = 0;
  for (const BatchTile& T : b->tiles) max_chunks = std::max(max_chunks, (u64)T.g.nchunks);
  std::vector<spcn_batch_config> cand;
  for (int k : {2, 4, 8, 16, 32, 64}) {
    if (k > 2 && (u64)k * kPassThreads > 2 * max_chunks) break;
    spcn_batch_config c0{};
    c0.item_chunks = k * kPassThreads;
    c0.schedule = SPCN_SCHED_PHASED;
    cand.push_back(c0);
    spcn_batch_config c1 = c0;
    c1.schedule = SPCN_SCHED_INTERLEAVED;
    c1.group_px = 16ll << 20;
    cand.push_back(c1);
  }
  if (max_chunks < (1ull << 32)) {
    spcn_batch_config c2{};
    c2.item_chunks = 32 * kPassThreads;
    c2.schedule = SPCN_SCHED_STAGED;
    cand.push_back(c2);
  }
  if (b->persist_ok) {
    spcn_batch_config c3{};
    c3.item_chunks = 32 * kPassThreads;
    c3.schedule = SPCN_SCHED_PERSISTENT;
    cand.push_back(c3);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPCN_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SPCN_ERR_CUDA; }
  int rc = SPCN_OK;
  int best = -1;
  float best_ms = 0.f;
  int written = 0;
  const bool timing = b->c->timing;
  b->c->timing = false;   // the tuner's own runs are not reported as kernel time
  for (size_t k = 0; k < cand.size() && rc == SPCN_OK; ++k) {
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
    rc = apply_config(b, cand[k]);
    if (rc) break;
    rc = batch_launch(b, st);   // untimed run
    for (int r = 0; r < reps && rc == SPCN_OK; ++r) {
      if (r == 0 && cudaEventRecord(e0, st) != cudaSuccess) rc = SPCN_ERR_CUDA;
      if (rc == SPCN_OK) rc = batch_launch(b, st);
    }
    if (rc) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = SPCN_ERR_CUDA;
      break;
    }
    int err = 0;
    std::vector<char> h(kRunStateBytes);
    if (cudaMemcpy(h.data(), b->d_state, kRunStateBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = SPCN_ERR_CUDA;
      break;
    }
    err = reinterpret_cast<const BatchRunState*>(h.data())->err;
    if (err) { rc = err; break; }
    cand[k].ms = ms / (float)reps;
    if (trials && written < max_trials) trials[written++] = cand[k];
    if (best < 0 || cand[k].ms < best_ms) { best = (int)k; best_ms = cand[k].ms; }
  }
  b->c->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_trials) *n_trials = written;
  if (rc) return rc;
  rc = apply_config(b, cand[best]);
  b->cfg.ms = best_ms;
  return rc;
}

int spcn_batch_destroy(void* batch) {
  if (!batch) return SPCN_OK;
  Batch* b = static_cast<Batch*>(batch);
  DeviceGuard guard(b->c->device);
  cudaDeviceSynchronize();
  batch_free(b);
  return SPCN_OK;
}

int spcn_normalize_batched(void* ctx, int32_t n, const spcn_image* tiles,
                           const spcn_stats* tile_stats, const spcn_stats* tgt_st,
                           const spcn_params* params, uint8_t* const* outs,
                           const int64_t* out_pitches, double* p99_out, int32_t* status_out,
                           void* stream) {
  void* b = nullptr;
  int rc = spcn_batch_create(ctx, n, tiles, tile_stats, tgt_st, params, outs, out_pitches, &b);
  if (rc) return rc;
  rc = spcn_batch_run(b, stream);
  if (rc == SPCN_OK) rc = spcn_batch_results(b, p99_out, status_out, nullptr, stream);
  spcn_batch_destroy(b);
  return rc;
}

}  // extern "C"
