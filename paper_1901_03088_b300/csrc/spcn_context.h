// Host-side context of the SPCN library: the device scratch it owns and the
// launch configuration measured once per device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spcn_internal.cuh"

namespace spcn {

// Device-side state of one basis estimation.
struct BasisState {
  u64 m;              // sample size
  u64 n_nw, n_br;     // non-white / bright sample pixels
  int n_acc;          // accepted patches
  int iters;
  int status;
  int pad;
  double objective;
  double W[6];        // final basis in FP64 (ordered)
  SelectState sel;    // percentile of the sampled non-white densities
  unsigned i0_hist[3 * 256];
  unsigned i0_ticket;
};

struct Context {
  int device = 0;
  int num_sms = 0;
  int* err = nullptr;              // first error recorded on the device
  Model* model = nullptr;          // image / source model
  Model* model_b = nullptr;        // basis-estimation model
  SelectState* sel = nullptr;      // full-image percentile record
  u64* coarse = nullptr;           // [2][kWinGroups]
  u64* fine = nullptr;             // [2][kWinBins]
  u64* rhist = nullptr;            // [3][kTracks][kRadixBins]
  u64* rhist_b = nullptr;          // same, for the sample percentile
  double* partials = nullptr;      // [2][max grid][kAcc]
  BasisState* bs = nullptr;
  void* wdev = nullptr;            // P99 window computed on the device (struct Window)
  u64* fallbacks = nullptr;        // whole-image percentile launches that missed pass 1's window
  unsigned* f32_ticket = nullptr;  // last-block ticket of the float backward (0 between launches)
  // grown on demand
  uint32_t* sample = nullptr;      // packed RGB of the sample
  uint32_t* nw = nullptr;          // non-white sample pixels (stable order)
  uint32_t* br = nullptr;          // bright sample pixels (stable order)
  size_t sample_cap = 0;
  unsigned* blk = nullptr;         // per-block counts for the compaction [2][nblk]
  u64* blk_off = nullptr;          // exclusive offsets [2][nblk]
  size_t blk_cap = 0;
  int* cand = nullptr;             // patch candidates: counts, then accepted origins
  int cand_cap = 0;
  // buffers point into memory the context does not own (the allocation-free
  // entry point): a request beyond their capacity is refused, never regrown
  bool fixed_scratch = false;
  int64_t launches = 0;
  // blocks per SM at the launch configuration of each kernel
  int occ_window = 0, occ_recon = 0, occ_density = 0, occ_select = 0;
  int occ_snmf = 0, occ_radix_list = 0, occ_debug = 0;
  int occ_f32_fwd = 0, occ_f32_bwd = 0;
  long long timeout_ns = 2000000000LL;   // grid-barrier give-up time
  // optional CUDA-event timing of the pixel kernels
  struct Timed { int kernel; cudaEvent_t a, b; };
  bool timing = false;
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
  double kernel_ms[SPCN_KERNEL_COUNT] = {};
  int64_t kernel_n[SPCN_KERNEL_COUNT] = {};
};

// Brackets one launch with events when the context's timing is on.
struct TimedLaunch {
  Context* c;
  int kernel;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(Context* ctx, int k, cudaStream_t s);
  ~TimedLaunch();
};
int drain_timing(Context* c);

// Selects the context's device for the duration of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Argument checks shared by the entry points (spcn_api.cu).
bool image_ok(const spcn_image* img);
bool params_ok(const spcn_params* p);
// SPCN_OK, INVALID_ARG or DEGENERATE_BASIS; signed_p99: the percentiles may
// be negative (pseudo-inverse densities)
int stats_ok(const spcn_stats* s, bool signed_p99 = false);
spcn_stats output_target(const spcn_stats* t, const spcn_params* p);   // Eq. 4's target record
Geometry make_geometry(const spcn_image* img, uint8_t* out, int64_t out_pitch, int* err);

int ensure_sample_capacity(Context* c, size_t n);
int ensure_candidate_capacity(Context* c, int n);

#define SPCN_CUDA_TRY(expr)                         \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) {                        \
      return e_ == cudaErrorMemoryAllocation ? SPCN_ERR_OOM : SPCN_ERR_CUDA; \
    }                                               \
  } while (0)

#define SPCN_LAUNCH_CHECK(ctx)                      \
  do {                                              \
    (ctx)->launches++;                              \
    cudaError_t e_ = cudaGetLastError();            \
    if (e_ != cudaSuccess) return SPCN_ERR_CUDA;    \
  } while (0)

// Shared-memory sizes of the pixel kernels.
constexpr int kChunkStack = 32;   // per-warp stack of tissue chunks in pass 1 (at most 31 used)
constexpr size_t kWindowSmem = kLutSmemBytes + sizeof(unsigned) * 2 * kWinGroups +
                               sizeof(uint2) * 2 * kPassThreads +   // per-warp hit queues (64 each)
                               (3 * sizeof(uint4) + sizeof(unsigned)) * kChunkStack * (kPassThreads / 32);
constexpr size_t kRadixSmem = kLutSmemBytes + sizeof(unsigned) * kTracks * kRadixBins;
// the density pass stages one plane of a warp's 512 pixels (2 KB per warp)
constexpr size_t kDensitySmem = kLutSmemBytes + 2048 * (kPassThreads / 32);

// Constants of the conservative all-white test of a full chunk (pass 1):
// (AND of its words & wm) == we.
void white_test_consts(int T, unsigned* wm, unsigned* we);

int configure_pixel_kernels(Context* c);
int configure_basis_kernels(Context* c);
int configure_grad_kernels(Context* c);

}  // namespace spcn
