// Basis estimation without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns every byte of the GPU through its own pool, plugin
// or driver-style hosts that forbid cudaMalloc (it can synchronise the whole
// device and stall other work), and latency-critical pipelines that must not
// touch the allocator once they are running.  They cannot create an
// spcn_context, which allocates its scratch.  spcn_estimate_basis_noalloc
// serves them: it runs the same kernels as spcn_estimate_basis, with every
// scratch buffer carved out of one fixed array compiled into this library
// (g_noalloc_scratch below, about 6.8 MB, held by every GPU that loads the
// library until the process exits).  The caller passes only the image and
// receives the statistics record.
#include <mutex>

#include "spcn_context.h"
#include "spcn_internal.cuh"

namespace spcn {

// Capacity of the static scratch.
constexpr u64 kNoAllocMaxSample = 1ull << 19;   // sample pixels (3 lists of 4 bytes each)
constexpr int kNoAllocMaxPatches = 4096;        // patches kept (5 ints of candidates each)
constexpr int kNoAllocMaxSnmfGrid = 1024;       // blocks of the sparse-NMF launch
constexpr int kNoAllocMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of each buffer inside the static array.
constexpr size_t kOffErr = 0;
constexpr size_t kOffModel = kOffErr + align256(sizeof(int));
constexpr size_t kOffBasis = kOffModel + align256(sizeof(Model));
constexpr size_t kOffSel = kOffBasis + align256(sizeof(BasisState));
constexpr size_t kOffRhist = kOffSel + align256(sizeof(SelectState));
constexpr size_t kOffPartials = kOffRhist + align256(sizeof(u64) * 3 * kTracks * kRadixBins);
constexpr size_t kOffCand = kOffPartials + align256(sizeof(double) * 2 * kNoAllocMaxSnmfGrid * kAcc);
constexpr u64 kNoAllocMaxBlk = (kNoAllocMaxSample + 4095) / 4096;
constexpr size_t kOffBlk = kOffCand + align256(sizeof(int) * 5 * kNoAllocMaxPatches);
constexpr size_t kOffBlkOff = kOffBlk + align256(sizeof(unsigned) * 2 * kNoAllocMaxBlk);
constexpr size_t kOffSample = kOffBlkOff + align256(sizeof(u64) * 2 * kNoAllocMaxBlk);
constexpr size_t kOffNw = kOffSample + align256(sizeof(uint32_t) * kNoAllocMaxSample);
constexpr size_t kOffBr = kOffNw + align256(sizeof(uint32_t) * kNoAllocMaxSample);
constexpr size_t kNoAllocScratchBytes = kOffBr + align256(sizeof(uint32_t) * kNoAllocMaxSample);

// The scratch itself.  In host code this name is only a stand-in; the device
// address comes from cudaGetSymbolAddress during the per-device set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Per-device view of the scratch (host memory, no heap allocation).
static Context g_noalloc_ctx[kNoAllocMaxDevices];
static bool g_noalloc_ready[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Set-up for the current device, done once: resolve the scratch's device
// address, point every buffer of a context view into it, and read the launch
// configuration (function attributes and occupancy; nothing is allocated).
static int noalloc_setup(int dev, Context** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SPCN_ERR_INVALID_ARG;
  Context* c = &g_noalloc_ctx[dev];
  if (!g_noalloc_ready[dev]) {
    unsigned char* base = nullptr;
    if (cudaGetSymbolAddress((void**)&base, g_noalloc_scratch) != cudaSuccess || !base)
      return SPCN_ERR_CUDA;
    c->device = dev;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return SPCN_ERR_CUDA;
    c->err = reinterpret_cast<int*>(base + kOffErr);
    c->model_b = reinterpret_cast<Model*>(base + kOffModel);
    c->bs = reinterpret_cast<BasisState*>(base + kOffBasis);
    c->sel = reinterpret_cast<SelectState*>(base + kOffSel);
    c->rhist_b = reinterpret_cast<u64*>(base + kOffRhist);
    c->partials = reinterpret_cast<double*>(base + kOffPartials);
    c->cand = reinterpret_cast<int*>(base + kOffCand);
    c->cand_cap = 5 * kNoAllocMaxPatches;
    c->blk = reinterpret_cast<unsigned*>(base + kOffBlk);
    c->blk_off = reinterpret_cast<u64*>(base + kOffBlkOff);
    c->blk_cap = kNoAllocMaxBlk;
    c->sample = reinterpret_cast<uint32_t*>(base + kOffSample);
    c->nw = reinterpret_cast<uint32_t*>(base + kOffNw);
    c->br = reinterpret_cast<uint32_t*>(base + kOffBr);
    c->sample_cap = kNoAllocMaxSample;
    c->fixed_scratch = true;
    int rc = configure_pixel_kernels(c);
    if (rc) return rc;
    rc = configure_basis_kernels(c);
    if (rc) return rc;
    if (c->num_sms * c->occ_snmf > kNoAllocMaxSnmfGrid) c->occ_snmf = kNoAllocMaxSnmfGrid / c->num_sms;
    if (c->occ_snmf < 1) return SPCN_ERR_CUDA;
    if (cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess) return SPCN_ERR_CUDA;
    g_noalloc_ready[dev] = true;
  }
  *out = c;
  return SPCN_OK;
}

}  // namespace spcn

using namespace spcn;

extern "C" int spcn_estimate_basis_noalloc(const spcn_image* img, const spcn_params* params,
                                           spcn_stats* out, void* stream) {
  // the arguments are checked before any size is derived from them
  if (!out || !image_ok(img) || !params_ok(params)) return SPCN_ERR_INVALID_ARG;
  // the sample must fit the static scratch (a first, early answer: the
  // capacity checks inside the estimation refuse anything larger as well,
  // because this context's buffers are marked fixed)
  const u64 N = (u64)img->width * (u64)img->height;
  u64 need = 0;
  if (params->sample_mode == SPCN_SAMPLE_ALL) {
    need = N;
  } else if (params->sample_mode == SPCN_SAMPLE_HASH) {
    need = (u64)((double)params->sample_rate * (double)N + 0.5);
  } else {
    if (params->n_patches > kNoAllocMaxPatches) return SPCN_ERR_SCRATCH_LIMIT;
    need = (u64)params->n_patches * (u64)params->patch_size * (u64)params->patch_size;
  }
  if (need > kNoAllocMaxSample) return SPCN_ERR_SCRATCH_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPCN_ERR_CUDA;
  Context* c = nullptr;
  const int rc = noalloc_setup(dev, &c);
  if (rc) return rc;
  return spcn_estimate_basis(c, img, params, out, stream);
}
