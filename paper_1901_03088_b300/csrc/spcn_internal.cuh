// Internal declarations of the SPCN CUDA library (sm_103a).
//
// Layout of the per-pixel path (see the public header for the paper's steps):
//   k_build_model   Eq. 1 table: v_c(i) = log(i0_c / max(i,1)) in FP64, and
//                   the W-projected, lambda-folded table used by every pixel
//                   pass; the closed-form coefficients of the Eq. 2 H-step.
//   k_pass_window   pass 1: H of every pixel, non-white count, and an exact
//                   per-key histogram of a window around the expected P99
//                   (keys = FP32 bit patterns); the last block selects the
//                   percentile ranks inside the window.
//   k_select_image  exact radix select over the image for ranks the window
//                   missed (returns at once when nothing is missing).
//   k_pass_recon    pass 2: H again, Eq. 3 scaling, Eq. 4, rounding, store.
//   k_pass_density  H written planar.
//   basis kernels   sampling, stable compaction, i0, sparse NMF, sample P99.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spcn.h"

namespace spcn {

typedef unsigned long long u64;

constexpr int kLutRep = 16;          // copies per table entry: lane l reads copy l%16
constexpr int kLutEntries = 3 * 256;
constexpr int kChunk = 16;           // pixels per thread step (48 bytes)
constexpr int kWinBits = 20;
constexpr int kWinBins = 1 << kWinBits;   // exact key bins per stain in the window
constexpr int kWinGroupBits = 10;
constexpr int kWinGroup = 1 << kWinGroupBits;
constexpr int kWinGroups = kWinBins >> kWinGroupBits;
constexpr int kRadixBins = 2048;
constexpr int kTracks = 4;           // (stain 0, rank k), (0, k+1), (1, k), (1, k+1)
constexpr int kPassThreads = 512;
constexpr int kAcc = 12;             // sparse-NMF reduced sums
constexpr double kWindowDelta = 0.04;   // relative half-width of the P99 window

// Closed form of the two-atom non-negative lasso for one basis:
//   d = W'v - lambda (folded into the projected table),
//   t1 = a11 d1 + a12 max(d2,0),  t2 = a22 d2 + a21 max(d1,0),
//   h1 = max(0, min(u1 d1, t1)),  h2 = max(0, min(u2 d2, t2)),
// with a11 = G22/det, a12 = a21 = -G12/det, a22 = G11/det, u_j = 1/G_jj.
// Equal to the KKT active-set solution whenever G12 = w1.w2 >= 0, which
// holds for non-negative bases.
struct Lasso {
  float a11, a12, a21, a22, u1, u2;
};

// Per-image model in device memory.
struct Model {
  float2 proj[kLutEntries];   // (W[c,0] v_c(i), W[c,1] v_c(i)) - (lambda,lambda) for c == 0
  float od[kLutEntries];      // v_c(i)
  Lasso lasso;
  float W[6];                 // column-major 3x2
  float i0[3];
  int status;
};

// Device-side selection record of one percentile computation.
struct SelectState {
  u64 n_nw;                   // non-white pixels
  u64 below[2];               // non-white pixels whose key < lo[j]
  u64 rank[kTracks];          // wanted 0-based ranks
  unsigned lo[2];             // window: keys lo .. lo+nb-1
  unsigned nb[2];
  unsigned key[kTracks];      // selected keys
  int resolved[kTracks];
  int all_resolved;
  unsigned done_ctas;         // last-block ticket of pass 1
  unsigned barrier;           // grid barrier counter
  int abort;                  // set when a grid-wide wait gave up (this launch only)
  double t;                   // interpolation weight of the type-7 percentile
  double p99[2];
  double scale[2];            // tgt_p99 / p99 (1 where p99 == 0)
};

// Pixel traversal of one image (and optionally an output of the same size).
struct Geometry {
  const uint8_t* src;
  uint8_t* dst;
  int64_t src_pitch, dst_pitch;
  int64_t width, height;
  int64_t npx;
  u64 nchunks;
  u64 cpr;          // chunks per row (row mode)
  u64 magic;        // ceil(2^64 / cpr) for cpr >= 2
  int flat;         // 1: rows are contiguous in both src and dst -> one long row
  int vec_src;      // 16-byte vector loads allowed on full chunks
  int vec_dst;      // 16-byte vector stores allowed on full chunks
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void record_error(int* err, int code) {
  atomicCAS(err, 0, code);
}

// Grid-wide barrier for cooperative launches.  `target` is the arrival count
// that releases this barrier (k * expected blocks for the k-th barrier).
// `abort` is a per-launch word, zeroed before the launch.  The wait gives up
// after timeout_ns, or as soon as another block gave up; it then sets
// *abort, records SPCN_ERR_TIMEOUT in the context's error word and returns
// false, and the caller returns.
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned target, int* abort,
                                             int* err, long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    unsigned long long t0 = global_timer_ns();
    int ok = 1;
    while (ld_acquire(counter) < target) {
      if (*(volatile int*)abort != 0) { ok = 0; break; }
      if ((long long)(global_timer_ns() - t0) > timeout_ns) {
        atomicExch(abort, 1);
        record_error(err, SPCN_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// floor(q / cpr) exactly for q * cpr < 2^64 (multiply-high by ceil(2^64/cpr)).
__device__ __forceinline__ u64 div_chunks(u64 q, u64 cpr, u64 magic) {
  return cpr == 1 ? q : __umul64hi(q, magic);
}

// Byte k of a 48-byte chunk held in 12 words.
template <int I>
__device__ __forceinline__ unsigned chunk_byte(const unsigned (&w)[12]) {
  return (w[I >> 2] >> ((I & 3) * 8)) & 0xFFu;
}

// The Eq. 2 H-step of one pixel from its 8-bit channels.  `lut` points at
// this lane's copy of the projected table.  Every pixel pass uses exactly
// this arithmetic, so their densities agree bit for bit.
__device__ __forceinline__ void solve_pixel(const float2* __restrict__ lut, unsigned r,
                                            unsigned g, unsigned b, const Lasso& L,
                                            float& h1, float& h2) {
  const float2 e0 = lut[r * kLutRep];
  const float2 e1 = lut[(256u + g) * kLutRep];
  const float2 e2 = lut[(512u + b) * kLutRep];
  const float d1 = (e0.x + e1.x) + e2.x;
  const float d2 = (e0.y + e1.y) + e2.y;
  const float t1 = fmaf(L.a12, fmaxf(d2, 0.f), L.a11 * d1);
  const float t2 = fmaf(L.a21, fmaxf(d1, 0.f), L.a22 * d2);
  const float m1 = fminf(L.u1 * d1, t1);
  const float m2 = fminf(L.u2 * d2, t2);
  // max with 0 on the bit pattern: negative values and -0 become +0
  h1 = __int_as_float(max(__float_as_int(m1), 0));
  h2 = __int_as_float(max(__float_as_int(m2), 0));
}

// Copy the projected table of `m` into shared memory, replicated kLutRep
// times (entry e, copy r at s[e * kLutRep + r]); returns this lane's base.
__device__ __forceinline__ const float2* load_lut(const Model* __restrict__ m, float2* s) {
  for (int i = threadIdx.x; i < kLutEntries * kLutRep; i += blockDim.x)
    s[i] = m->proj[i / kLutRep];
  __syncthreads();
  return s + (threadIdx.x & (kLutRep - 1));
}

// Inclusive warp scan of 64-bit counts.
__device__ __forceinline__ u64 warp_incl_scan(u64 v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

__device__ __forceinline__ u64 warp_sum(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  s_tmp: >= 32 entries.
__device__ __forceinline__ u64 block_sum(u64 v, u64* s_tmp) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_tmp[w] = v;
  __syncthreads();
  u64 t = 0;
  for (int i = 0; i < nw; ++i) t += s_tmp[i];
  return t;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and sets *total.  s_tmp: >= 33 entries.
__device__ __forceinline__ u64 block_excl_scan(u64 v, u64* s_tmp, u64* total) {
  const u64 incl = warp_incl_scan(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 31) s_tmp[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 run = 0;
    for (int i = 0; i < nw; ++i) { u64 x = s_tmp[i]; s_tmp[i] = run; run += x; }
    s_tmp[32] = run;
  }
  __syncthreads();
  *total = s_tmp[32];
  return s_tmp[w] + incl - v;
}

// Find the first index i in cnt[0..n) whose inclusive prefix sum exceeds r.
// Sets *s_idx (-1 if the total is <= r) and *s_before (prefix before i).
// Whole block must call.  s_tmp: >= 33 entries.
__device__ __forceinline__ void block_find_rank(const u64* cnt, int n, u64 r, int* s_idx,
                                                u64* s_before, u64* s_tmp) {
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int beg = threadIdx.x * per;
  const int end = min(n, beg + per);
  u64 local = 0;
  for (int i = beg; i < end; ++i) local += __ldcg(cnt + i);
  u64 total;
  const u64 excl = block_excl_scan(local, s_tmp, &total);
  if (threadIdx.x == 0) *s_idx = -1;
  __syncthreads();
  if (local > 0 && excl <= r && r < excl + local) {
    u64 c = excl;
    for (int i = beg; i < end; ++i) {
      const u64 x = __ldcg(cnt + i);
      if (r < c + x) { *s_idx = i; *s_before = c; break; }
      c += x;
    }
  }
  __syncthreads();
}

// Type-7 percentile value from the order statistics a (rank k) and b (rank
// k+1): a + t (b - a), computed without fused multiply-add so that a host
// evaluation of the same expression gives the same double.
__device__ __forceinline__ double interp_type7(float a, float b, double t) {
  const double da = (double)a, db = (double)b;
  return __dadd_rn(da, __dmul_rn(t, __dsub_rn(db, da)));
}

// Set ranks and interpolation weight of the type-7 percentile for n values.
__device__ __forceinline__ void type7_ranks(u64 n, double pct, u64* k_out, u64* k1_out,
                                            double* t_out) {
  const double pos = (double)(n - 1) * (pct / 100.0);
  u64 k = (u64)floor(pos);
  if (k > n - 1) k = n - 1;
  *k_out = k;
  *k1_out = (k + 1 <= n - 1) ? k + 1 : k;
  *t_out = pos - (double)k;
}

__device__ __forceinline__ void set_ranks(SelectState* s, u64 n, double pct) {
  u64 k, k1;
  double t;
  type7_ranks(n, pct, &k, &k1, &t);
  s->t = t;
  s->rank[0] = k; s->rank[1] = k1; s->rank[2] = k; s->rank[3] = k1;
}

// Percentiles and scale factors once all four keys are known.
__device__ __forceinline__ void finish_percentiles(SelectState* s, double tgt0, double tgt1) {
  const double tg[2] = {tgt0, tgt1};
  for (int j = 0; j < 2; ++j) {
    const double p = interp_type7(__uint_as_float(s->key[2 * j]),
                                  __uint_as_float(s->key[2 * j + 1]), s->t);
    s->p99[j] = p;
    s->scale[j] = (p != 0.0) ? tg[j] / p : 1.0;
  }
}

// ---------------------------------------------------------------- host side
struct Context;

// Launchers (defined in the .cu files); all return spcn_status.
int launch_build_model(Context* c, Model* m, const float* W, const float* i0, float lambda,
                       const Model* from_device, cudaStream_t st);
int launch_percentile_passes(Context* c, const Geometry& g, const Model* m, int white_thresh,
                             double pct, const double* hint, const double* tgt_p99,
                             cudaStream_t st);
int launch_recon(Context* c, const Geometry& g, const Model* m, const float* Wt,
                 const float* i0t, cudaStream_t st);
int launch_density(Context* c, const Geometry& g, const Model* m, float* H, int64_t stride,
                   cudaStream_t st);
int run_estimate_basis(Context* c, const spcn_image* img, const spcn_params* p, spcn_stats* out,
                       cudaStream_t st);
int launch_debug_barrier(Context* c, int extra, long long timeout_ns, cudaStream_t st);

}  // namespace spcn
