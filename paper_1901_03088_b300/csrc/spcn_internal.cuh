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

// Shared-memory table of Eq. 1 projected on the basis: one 256-byte row per
// 8-bit intensity, holding 16 copies (one per lane of a half-warp, so 64-bit
// loads never conflict) of the red and green entries; a second 64 KB region
// holds the blue entries.  The byte offset of (channel, intensity i) for lane
// l is i*256 + (l%16)*8 + {0, 128, 65536}: one byte permute builds it from
// the packed pixel bytes.
constexpr int kLutRep = 16;
constexpr int kLutEntries = 3 * 256;
constexpr int kLutRowBytes = 256;
constexpr int kLutOffG = 128;
constexpr int kLutOffB = 256 * kLutRowBytes;
constexpr int kLutSmemBytes = 2 * 256 * kLutRowBytes;
constexpr int kChunk = 16;           // pixels per thread step (48 bytes)
constexpr int kWinBits = 20;
constexpr int kWinBins = 1 << kWinBits;   // exact key bins per stain in the window
constexpr int kWinGroupBits = 10;
constexpr int kWinGroup = 1 << kWinGroupBits;
constexpr int kWinGroups = kWinBins >> kWinGroupBits;
constexpr int kRadixBins = 2048;
constexpr int kTracks = 4;           // (stain 0, rank k), (0, k+1), (1, k), (1, k+1)
constexpr int kPassThreads = 1024;     // one block per SM (the table fills 128 KB)
constexpr int kHexpAuto = -1000000;
constexpr int kAcc = 12;             // sparse-NMF reduced sums
constexpr double kWindowDelta = 0.04;   // relative half-width of the P99 window

// Closed form of the two-atom non-negative lasso (Eq. 2's H-step) used by
// every pixel pass.  With G = W'W, d_j = (w_j.v - lambda)/G_jj, rho_j =
// G12/G_jj and kappa = G11 G22 / det G, the minimiser over h >= 0 is
//   h_j = max(0, min(d_j, kappa (d_j - rho_j max(d_other, 0))))
// whenever G12 >= 0 (non-negative bases); with D_j = max(0, d_j) this is
//   h_j = min(D_j, max(0, kappa (D_j - rho_j D_other))).
// The table stores s*d_j contributions (lambda and 1/G_jj folded in, s =
// 2^-hexp chosen so that |s d_j| <= 1/2), so both max(0, .) become the
// hardware saturate modifier; h_j = 2^hexp * h~_j exactly.
struct Lasso {
  float nrho1, nrho2;   // -rho_1, -rho_2
  float kappa;
  float hscale;         // 2^hexp
  int hexp;
  int pinv;             // the table holds pseudo-inverse rows (SPCN_FLAG_H_PINV)
};

// Per-image model in device memory.
struct Model {
  float2 proj[kLutEntries];   // s ((W[c,0] v_c(i) - [c==0] lambda)/G11, (W[c,1] v_c(i) - [c==0] lambda)/G22)
  float od[kLutEntries];      // v_c(i) = log(i0_c / max(i,1))
  Lasso lasso;
  float pa[6];                // s W[c,j] / G_jj, index 3 j + c (pass 2 projects OD with FMAs)
  float pb[2];                // -s lambda / G_jj
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
  unsigned barrier2;          // grid barrier counter of the window-miss recovery
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
#ifdef SPCN_CHECKED
  int64_t src_bytes, dst_bytes;   // extent of each buffer: (height - 1) pitch + 3 width
  int* err;         // the context's error word, where failed device checks are recorded
#endif
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

// Bounds-checked build (-DSPCN_CHECKED, library libspcn_checked.so): device
// checks of every buffer index and extent that the kernels derive; a failed
// check records SPCN_ERR_INVALID_ARG in the context's error word (returned by
// the next synchronising call) and the access is skipped, with no trap.  In
// the normal build each check is the constant true and compiles away.
#ifdef SPCN_CHECKED
__device__ __forceinline__ bool check_or_record(bool ok, int* err) {
  if (!ok && err) record_error(err, SPCN_ERR_INVALID_ARG);
  return ok;
}
#define SPCN_CHECK(cond, err) (::spcn::check_or_record((cond), (err)))
#else
#define SPCN_CHECK(cond, err) (true)
#endif

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
    const unsigned long long t0 = global_timer_ns();
    int ok = 1;
    // back-to-back acquire polls (the acquire orders this block's later
    // reads); the abort word and the clock every 16th poll
    for (unsigned polls = 1; ld_acquire(counter) < target; ++polls) {
      if ((polls & 15u) != 0u) continue;
      if (*(volatile int*)abort != 0) { ok = 0; break; }
      if ((long long)(global_timer_ns() - t0) > timeout_ns) {
        atomicExch(abort, 1);
        record_error(err, SPCN_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// floor(q / cpr) exactly for q * cpr < 2^64 (multiply-high by ceil(2^64/cpr)).
__device__ __forceinline__ u64 div_chunks(u64 q, u64 cpr, u64 magic) {
  return cpr == 1 ? q : __umul64hi(q, magic);
}

// ---------------------------------------------------------------- f32x2
typedef unsigned long long f2;   // two packed FP32 lanes (lo, hi)

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo_of(f2 v) {
  float a;
  asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(v));
  return a;
}
__device__ __forceinline__ float hi_of(f2 v) {
  float b;
  asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(v));
  return b;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float add_sat(float a, float b) {
  float d;
  asm("add.rn.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float mul_sat(float a, float b) {
  float d;
  asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
  float d;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// ---------------------------------------------------------------- H-step
// Table byte offset of the intensity held in byte `s` (0..3) of `word` for
// this lane: lanereg = (lane % 16) * 8 supplies byte 0, the intensity byte
// lands in byte 1 (x256), bytes 2-3 are zero.
__device__ __forceinline__ unsigned lut_addr(unsigned word, unsigned lanereg, int s) {
  return __byte_perm(word, lanereg, 0x7604u | ((unsigned)s << 4));
}

__device__ __forceinline__ float2 lut_ld(const char* lut, unsigned off) {
  return *reinterpret_cast<const float2*>(lut + off);
}

// Scaled H-step of one pixel from its three table offsets.  Every pixel pass
// (and solve_pair below, lane by lane) uses exactly this arithmetic, so all
// passes produce the same densities bit for bit.  PINV: the table holds the
// rows of pinv(W) times the optical density (§2.1), and the densities are the
// plain sums (signed, no sparsity).
template <bool PINV = false>
__device__ __forceinline__ void solve_one(const char* lut, unsigned aR, unsigned aG, unsigned aB,
                                          const Lasso& L, float& h1, float& h2) {
  const float2 eR = lut_ld(lut, aR), eG = lut_ld(lut, aG + kLutOffG), eB = lut_ld(lut, aB + kLutOffB);
  if (PINV) {
    h1 = (eR.x + eG.x) + eB.x;
    h2 = (eR.y + eG.y) + eB.y;
    return;
  }
  const float D1 = add_sat(eR.x + eG.x, eB.x);
  const float D2 = add_sat(eR.y + eG.y, eB.y);
  const float t1 = mul_sat(L.kappa, fmaf(L.nrho1, D2, D1));
  const float t2 = mul_sat(L.kappa, fmaf(L.nrho2, D1, D2));
  h1 = fminf(D1, t1);
  h2 = fminf(D2, t2);
}

// The same for two pixels at once, packed lanes: (A, B) -> H1 = (h1_A, h1_B),
// H2 = (h2_A, h2_B).
template <bool PINV = false>
__device__ __forceinline__ void solve_pair(const char* lut, unsigned aRA, unsigned aGA,
                                           unsigned aBA, unsigned aRB, unsigned aGB, unsigned aBB,
                                           f2 NR1, f2 NR2, float kappa, f2& H1, f2& H2) {
  const float2 eRA = lut_ld(lut, aRA), eGA = lut_ld(lut, aGA + kLutOffG),
               eBA = lut_ld(lut, aBA + kLutOffB);
  const float2 eRB = lut_ld(lut, aRB), eGB = lut_ld(lut, aGB + kLutOffG),
               eBB = lut_ld(lut, aBB + kLutOffB);
  const f2 SA = add2(pk(eRA.x, eRA.y), pk(eGA.x, eGA.y));
  const f2 SB = add2(pk(eRB.x, eRB.y), pk(eGB.x, eGB.y));
  if (PINV) {
    H1 = pk(lo_of(SA) + eBA.x, lo_of(SB) + eBB.x);
    H2 = pk(hi_of(SA) + eBA.y, hi_of(SB) + eBB.y);
    return;
  }
  const float D1A = add_sat(lo_of(SA), eBA.x), D2A = add_sat(hi_of(SA), eBA.y);
  const float D1B = add_sat(lo_of(SB), eBB.x), D2B = add_sat(hi_of(SB), eBB.y);
  const f2 P1 = pk(D1A, D1B), P2 = pk(D2A, D2B);
  const f2 Q1 = fma2(NR1, P2, P1);
  const f2 Q2 = fma2(NR2, P1, P2);
  const float t1A = mul_sat(kappa, lo_of(Q1)), t1B = mul_sat(kappa, hi_of(Q1));
  const float t2A = mul_sat(kappa, lo_of(Q2)), t2B = mul_sat(kappa, hi_of(Q2));
  H1 = pk(fminf(D1A, t1A), fminf(D1B, t1B));
  H2 = pk(fminf(D2A, t2A), fminf(D2B, t2B));
}

// Order-preserving map of FP32 bit patterns to unsigned keys for signed
// densities (pseudo-inverse): negative values reversed below the positive
// ones.  The non-negative densities of the lasso use the raw bits.
__device__ __forceinline__ unsigned signed_key(unsigned b) {
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned signed_key_inv(unsigned k) {
  return (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
}

// Copy the projected table of `m` into the shared-memory layout above.
__device__ __forceinline__ void load_lut(const Model* __restrict__ m, char* s) {
  float2* f = reinterpret_cast<float2*>(s);
  // region 0: rows of [R x16][G x16]; region 1: rows of [B x16][unused x16]
  for (int i = threadIdx.x; i < 2 * 256 * 32; i += blockDim.x) {
    const int region = i >> 13, row = (i >> 5) & 255, half = (i >> 4) & 1;
    const int c = region == 0 ? half : 2;
    f[i] = (region == 1 && half == 1) ? make_float2(0.f, 0.f) : m->proj[c * 256 + row];
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned lane_reg() { return (threadIdx.x & 15u) << 3; }

// Optical-density table for pass 2: the same 256-byte rows, but 4-byte
// entries v_c(i) with one copy per lane of the warp (32 copies: a 4-byte
// load by 32 lanes is one conflict-free wavefront, half the wavefronts of
// the projected table's 8-byte loads).  Row i of the first 64 KB holds R
// then G, the second 64 KB holds B; lane l's entry is at i*256 + 4 l.
__device__ __forceinline__ void load_od_lut(const Model* __restrict__ m, char* s) {
  float* f = reinterpret_cast<float*>(s);
  for (int i = threadIdx.x; i < 2 * 256 * 64; i += blockDim.x) {
    const int region = i >> 14, row = (i >> 6) & 255, half = (i >> 5) & 1;
    const int c = region == 0 ? half : 2;
    f[i] = (region == 1 && half == 1) ? 0.f : m->od[c * 256 + row];
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned lane_reg_od() { return (threadIdx.x & 31u) << 2; }

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

// block_find_rank for the four tracks at once: a quarter of the block per
// track (blockDim.x a multiple of 128), histogram cnt[t] of n bins and rank
// r[t] for the tracks with act[t] set.  Each thread's bins (at most
// kFindPer of them are kept in registers for the search; more are read
// again) are loaded once, all in flight together.  s_idx[t] = -1 if the
// track's total is <= r[t].  Whole block must call.
constexpr int kFindPer = 8;
__device__ __forceinline__ void block_find_rank4(const u64* const (&cnt)[4], int n,
                                                 const u64 (&r)[4], const int (&act)[4],
                                                 int* s_idx, u64* s_before, u64* s_wsum) {
  const int group = (int)blockDim.x >> 2;
  const int t = (int)threadIdx.x / group, sub = (int)threadIdx.x % group;
  const int per = (n + group - 1) / group;
  const int beg = min(n, sub * per), end = min(n, beg + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this thread's track, by selects (an array indexed at run time would live
  // in local memory)
  const u64* ct = t == 0 ? cnt[0] : (t == 1 ? cnt[1] : (t == 2 ? cnt[2] : cnt[3]));
  const u64 rt = t == 0 ? r[0] : (t == 1 ? r[1] : (t == 2 ? r[2] : r[3]));
  const int at = t == 0 ? act[0] : (t == 1 ? act[1] : (t == 2 ? act[2] : act[3]));
  u64 v[kFindPer];
  u64 local = 0;
#pragma unroll
  for (int k = 0; k < kFindPer; ++k) {
    v[k] = (at && beg + k < end) ? __ldcg(ct + beg + k) : 0ull;
    local += v[k];
  }
  if (at)
    for (int i = beg + kFindPer; i < end; ++i) local += __ldcg(ct + i);
  const u64 incl = warp_incl_scan(local);
  if (sub == 0) s_idx[t] = -1;
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  u64 excl = incl - local;
  for (int w = t * (group >> 5); w < warp; ++w) excl += s_wsum[w];
  if (at && local > 0 && excl <= rt && rt < excl + local) {
    u64 c = excl;
    int found = -1;
    u64 bef = 0;
#pragma unroll
    for (int k = 0; k < kFindPer; ++k) {
      if (found < 0 && rt < c + v[k]) { found = beg + k; bef = c; }
      c += v[k];
    }
    for (int i = beg + kFindPer; found < 0 && i < end; ++i) {
      const u64 x = __ldcg(ct + i);
      if (rt < c + x) { found = i; bef = c; }
      c += x;
    }
    s_idx[t] = found;
    s_before[t] = bef;
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

// Percentiles and scale factors once all four keys are known.  Keys are the
// bit patterns of the scaled densities h~; h = hscale * h~ exactly.
__device__ __forceinline__ void finish_percentiles(SelectState* s, double tgt0, double tgt1,
                                                   float hscale) {
  const double tg[2] = {tgt0, tgt1};
  for (int j = 0; j < 2; ++j) {
    const double p = interp_type7(__fmul_rn(__uint_as_float(s->key[2 * j]), hscale),
                                  __fmul_rn(__uint_as_float(s->key[2 * j + 1]), hscale), s->t);
    s->p99[j] = p;
    s->scale[j] = (p != 0.0) ? tg[j] / p : 1.0;
  }
}

// ---------------------------------------------------------------- host side
struct Context;

// Launchers (defined in the .cu files); all return spcn_status.
// pinv: the pseudo-inverse variant of the densities (SPCN_FLAG_H_PINV); the
// model must have been built with the same choice.
int launch_build_model(Context* c, Model* m, const float* W, const float* i0, float lambda,
                       const Model* from_device, cudaStream_t st, bool pinv = false);
int launch_percentile_passes(Context* c, const Geometry& g, const Model* m, int white_thresh,
                             double pct, const double* hint, int hexp, const double* tgt_p99,
                             cudaStream_t st, bool pinv = false);
int host_table_hexp(const float* W, const float* i0, float lambda);
int launch_recon(Context* c, const Geometry& g, const Model* m, const float* Wt,
                 const float* i0t, cudaStream_t st, bool pinv = false);
int launch_density(Context* c, const Geometry& g, const Model* m, float* H, int64_t stride,
                   cudaStream_t st, bool pinv = false);
// hint_only: the sample percentile is needed only as a search hint (a
// regular sub-sample is then selected instead of the whole sample)
int launch_estimate_basis(Context* c, const spcn_image* img, const spcn_params* p,
                          cudaStream_t st, bool hint_only = false);
int finish_estimate_basis(Context* c, spcn_stats* out, cudaStream_t st);
int run_estimate_basis(Context* c, const spcn_image* img, const spcn_params* p, spcn_stats* out,
                       cudaStream_t st);
int launch_debug_barrier(Context* c, int extra, long long timeout_ns, cudaStream_t st);
int launch_f32(Context* c, bool backward, const float* x, const float* gy, int batch, int64_t hw,
               const spcn_stats* src, const spcn_stats* tgt, const float* wt, float lambda,
               float* y, float* gx, float* gwt, cudaStream_t st);

}  // namespace spcn
