// C-ABI entry points of the SPCN library (declared in include/spcn.h):
// argument validation, the context and its scratch, and the order of the
// kernel launches of each call.
#include <math.h>
#include <string.h>

#include <cmath>
#include <new>

#include "spcn_context.h"
#include "spcn_internal.cuh"
#include "spcn_pixel.cuh"

namespace spcn {

int ensure_sample_capacity(Context* c, size_t n) {
  if (n == 0) n = 1;
  const size_t nblk = (n + 4095) / 4096;
  if (c->fixed_scratch && (n > c->sample_cap || nblk > c->blk_cap)) return SPCN_ERR_SCRATCH_LIMIT;
  if (n > c->sample_cap) {
    cudaFree(c->sample);
    cudaFree(c->nw);
    cudaFree(c->br);
    c->sample = c->nw = c->br = nullptr;
    c->sample_cap = 0;
    SPCN_CUDA_TRY(cudaMalloc(&c->sample, n * sizeof(uint32_t)));
    SPCN_CUDA_TRY(cudaMalloc(&c->nw, n * sizeof(uint32_t)));
    SPCN_CUDA_TRY(cudaMalloc(&c->br, n * sizeof(uint32_t)));
    c->sample_cap = n;
  }
  if (nblk > c->blk_cap) {
    cudaFree(c->blk);
    cudaFree(c->blk_off);
    c->blk = nullptr;
    c->blk_off = nullptr;
    c->blk_cap = 0;
    SPCN_CUDA_TRY(cudaMalloc(&c->blk, 2 * nblk * sizeof(unsigned)));
    SPCN_CUDA_TRY(cudaMalloc(&c->blk_off, 2 * nblk * sizeof(u64)));
    c->blk_cap = nblk;
  }
  return SPCN_OK;
}

int ensure_candidate_capacity(Context* c, int n) {
  if (c->fixed_scratch && n > c->cand_cap) return SPCN_ERR_SCRATCH_LIMIT;
  if (n > c->cand_cap) {
    cudaFree(c->cand);
    c->cand = nullptr;
    c->cand_cap = 0;
    SPCN_CUDA_TRY(cudaMalloc(&c->cand, (size_t)n * sizeof(int)));
    c->cand_cap = n;
  }
  return SPCN_OK;
}

TimedLaunch::TimedLaunch(Context* ctx, int k, cudaStream_t s) : c(ctx), kernel(k), st(s) {
  if (!c->timing) return;
  for (cudaEvent_t* e : {&a, &b}) {
    if (!c->pool.empty()) { *e = c->pool.back(); c->pool.pop_back(); }
    else if (cudaEventCreate(e) != cudaSuccess) *e = nullptr;
  }
  if (a && b) cudaEventRecord(a, st);
}

TimedLaunch::~TimedLaunch() {
  if (!c->timing) return;
  if (a && b) {
    cudaEventRecord(b, st);
    c->pending.push_back({kernel, a, b});
  } else {
    if (a) c->pool.push_back(a);
    if (b) c->pool.push_back(b);
  }
}

int drain_timing(Context* c) {
  int rc = SPCN_OK;
  for (auto& t : c->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess)
      rc = SPCN_ERR_CUDA;
    else {
      c->kernel_ms[t.kernel] += ms;
      c->kernel_n[t.kernel] += 1;
    }
    c->pool.push_back(t.a);
    c->pool.push_back(t.b);
  }
  c->pending.clear();
  return rc;
}

static void free_all(Context* c) {
  drain_timing(c);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  c->pool.clear();
  void* ptrs[] = {c->err, c->model, c->model_b, c->sel, c->coarse, c->fine, c->rhist,
                  c->rhist_b, c->partials, c->bs, c->wdev, c->sample, c->nw, c->br, c->blk,
                  c->blk_off, c->cand, c->fallbacks, c->f32_ticket};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// ---------------------------------------------------------------- validation
bool image_ok(const spcn_image* img) {
  if (!img || !img->data || img->width < 1 || img->height < 1) return false;
  if (img->pitch_bytes < 3ll * img->width) return false;
  const long long npx = (long long)img->width * img->height;
  if (npx >= (1ll << 36)) return false;
  // chunk indices are kept in 32 bits (pitched images: 16-pixel chunks per row)
  const long long chunks = (long long)img->height * ((img->width + 15) / 16);
  return chunks < (1ll << 32);
}

bool params_ok(const spcn_params* p) {
  if (!p) return false;
  if (!(p->lambda >= 0.f) || !std::isfinite(p->lambda)) return false;
  if (p->white_thresh < 0 || p->white_thresh > 255) return false;
  if (!(p->i0_pct >= 0.f && p->i0_pct <= 100.f)) return false;
  if (!(p->stain_pct >= 0.f && p->stain_pct <= 100.f)) return false;
  if (p->i0_max_samples < 1) return false;
  if (p->sample_mode < SPCN_SAMPLE_ALL || p->sample_mode > SPCN_SAMPLE_PATCHES) return false;
  if (p->sample_mode == SPCN_SAMPLE_HASH && !(p->sample_rate > 0.f && p->sample_rate <= 1.f))
    return false;
  if (p->sample_mode == SPCN_SAMPLE_PATCHES &&
      (p->n_patches < 1 || p->n_patches > 100000 || p->patch_size < 1 || p->patch_size > 4096))
    return false;
  if (p->max_iter < 1 || p->max_iter > 1000000) return false;
  if (!(p->tol >= 0.f) || !std::isfinite(p->tol)) return false;
  const uint32_t known = SPCN_FLAG_I0_255 | SPCN_FLAG_ORDER_BLUE | SPCN_FLAG_P99_SAMPLED |
                         SPCN_FLAG_P99_PATCH_MEDIAN | SPCN_FLAG_H_PINV | SPCN_FLAG_I0_OUT_255;
  if (p->flags & ~known) return false;
  if ((p->flags & SPCN_FLAG_P99_PATCH_MEDIAN) &&
      (p->sample_mode != SPCN_SAMPLE_PATCHES || p->n_patches > 4096))
    return false;
  return true;
}

// The target record as Eq. 4 uses it: with SPCN_FLAG_I0_OUT_255 the output
// white is 255 in every channel instead of the target's i0.
spcn_stats output_target(const spcn_stats* t, const spcn_params* p) {
  spcn_stats o = *t;
  if (p->flags & SPCN_FLAG_I0_OUT_255)
    for (int c = 0; c < 3; ++c) o.i0[c] = 255.f;
  return o;
}

// A usable basis and i0: finite, W >= 0, columns not parallel, i0 in [1,255].
int stats_ok(const spcn_stats* s, bool signed_p99) {
  if (!s) return SPCN_ERR_INVALID_ARG;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(s->W[i]) || s->W[i] < 0.f) return SPCN_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!(s->i0[i] >= 1.f && s->i0[i] <= 255.f)) return SPCN_ERR_INVALID_ARG;
  for (int i = 0; i < 2; ++i)
    if (!std::isfinite(s->p99[i]) || (!signed_p99 && s->p99[i] < 0.0)) return SPCN_ERR_INVALID_ARG;
  double g11 = 0, g22 = 0, g12 = 0;
  for (int c = 0; c < 3; ++c) {
    g11 += (double)s->W[c] * s->W[c];
    g22 += (double)s->W[3 + c] * s->W[3 + c];
    g12 += (double)s->W[c] * s->W[3 + c];
  }
  if (!(g11 * g22 - g12 * g12 > 1e-12)) return SPCN_ERR_DEGENERATE_BASIS;
  return SPCN_OK;
}

Geometry make_geometry(const spcn_image* img, uint8_t* out, int64_t out_pitch, int* err) {
  Geometry g;
  memset(&g, 0, sizeof(g));
  g.src = img->data;
  g.dst = out;
  g.src_pitch = img->pitch_bytes;
  g.dst_pitch = out ? out_pitch : 0;
  g.width = img->width;
  g.height = img->height;
#ifdef SPCN_CHECKED
  g.src_bytes = (int64_t)(img->height - 1) * img->pitch_bytes + 3ll * img->width;
  g.dst_bytes = out ? (int64_t)(img->height - 1) * out_pitch + 3ll * img->width : 0;
  g.err = err;
#else
  (void)err;
#endif
  g.npx = (int64_t)img->width * img->height;
  const int64_t row = 3ll * img->width;
  const bool contiguous = img->pitch_bytes == row && (!out || out_pitch == row);
  const uintptr_t sa = reinterpret_cast<uintptr_t>(img->data);
  const uintptr_t da = reinterpret_cast<uintptr_t>(out);
  if (contiguous) {
    g.flat = 1;
    g.nchunks = ((u64)g.npx + kChunk - 1) / kChunk;
    g.cpr = g.nchunks;
    g.magic = 0;
    g.vec_src = (sa & 15u) == 0;
    g.vec_dst = out ? ((da & 15u) == 0) : 0;
  } else {
    g.flat = 0;
    g.cpr = ((u64)img->width + kChunk - 1) / kChunk;
    g.nchunks = g.cpr * (u64)img->height;
    g.magic = g.cpr >= 2 ? (~0ull / g.cpr) + 1ull : 0ull;
    g.vec_src = (sa & 15u) == 0 && (img->pitch_bytes & 15) == 0;
    g.vec_dst = out ? ((da & 15u) == 0 && (out_pitch & 15) == 0) : 0;
  }
  return g;
}

static int read_error(Context* c, cudaStream_t st, int* out) {
  int h = 0;
  SPCN_CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPCN_CUDA_TRY(cudaStreamSynchronize(st));
  if (h != 0) SPCN_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), st));
  *out = h;
  return SPCN_OK;
}

}  // namespace spcn

using namespace spcn;

extern "C" {

void spcn_params_default(spcn_params* p) {
  if (!p) return;
  p->lambda = 0.1f;
  p->white_thresh = 220;
  p->i0_pct = 80.f;
  p->stain_pct = 99.f;
  p->i0_max_samples = 100000;
  p->sample_mode = SPCN_SAMPLE_HASH;
  p->sample_rate = 0.01f;
  p->n_patches = 200;
  p->patch_size = 256;
  p->max_iter = 200;
  p->tol = 1e-6f;
  p->flags = 0u;
  p->seed = 0ull;
}

const char* spcn_strerror(int status) {
  switch (status) {
    case SPCN_OK: return "ok";
    case SPCN_ERR_INVALID_ARG: return "invalid argument";
    case SPCN_ERR_CUDA: return "CUDA runtime error";
    case SPCN_ERR_OOM: return "out of device memory";
    case SPCN_ERR_NO_TISSUE: return "no non-white (tissue) pixel";
    case SPCN_ERR_DEGENERATE_BASIS: return "degenerate stain basis";
    case SPCN_ERR_TIMEOUT: return "grid-wide wait timed out";
    case SPCN_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

int spcn_context_create(void** out, int device) {
  if (!out) return SPCN_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return SPCN_ERR_CUDA;
  if (device < 0 || device >= ndev) return SPCN_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  Context* c = new (std::nothrow) Context();
  if (!c) return SPCN_ERR_OOM;
  c->device = device;
  int rc = SPCN_OK;
  do {
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) !=
        cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop) { rc = SPCN_ERR_CUDA; break; }
#define ALLOC(ptr, bytes)                                                        \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) { rc = SPCN_ERR_OOM; break; }
    ALLOC(c->err, sizeof(int));
    ALLOC(c->model, sizeof(Model));
    ALLOC(c->model_b, sizeof(Model));
    ALLOC(c->sel, sizeof(SelectState));
    ALLOC(c->coarse, sizeof(u64) * 2 * kWinGroups);
    ALLOC(c->fine, sizeof(u64) * 2 * (size_t)kWinBins);
    ALLOC(c->rhist, sizeof(u64) * 3 * kTracks * kRadixBins);
    ALLOC(c->rhist_b, sizeof(u64) * 3 * kTracks * kRadixBins);
    ALLOC(c->partials, sizeof(double) * 2 * 4096 * kAcc);
    ALLOC(c->bs, sizeof(BasisState));
    ALLOC(c->wdev, sizeof(Window));
    ALLOC(c->fallbacks, sizeof(u64));
    ALLOC(c->f32_ticket, sizeof(unsigned));
#undef ALLOC
    if (cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
    if (cudaMemset(c->fallbacks, 0, sizeof(u64)) != cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
    if (cudaMemset(c->f32_ticket, 0, sizeof(unsigned)) != cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
    rc = configure_pixel_kernels(c);
    if (rc) break;
    rc = configure_basis_kernels(c);
    if (rc) break;
    rc = configure_grad_kernels(c);
    if (rc) break;
    if (cudaDeviceSynchronize() != cudaSuccess) { rc = SPCN_ERR_CUDA; break; }
  } while (0);
  if (rc != SPCN_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return SPCN_OK;
}

int spcn_context_destroy(void* ctx) {
  if (!ctx) return SPCN_OK;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  cudaDeviceSynchronize();
  free_all(c);
  delete c;
  return SPCN_OK;
}

int64_t spcn_launch_count(void* ctx) {
  return ctx ? static_cast<Context*>(ctx)->launches : 0;
}

int spcn_exact_fallbacks(void* ctx, int64_t* count) {
  if (!ctx || !count) return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  u64 n = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&n, c->fallbacks, sizeof(u64), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SPCN_ERR_CUDA;
  *count = (int64_t)n;
  return SPCN_OK;
}

int spcn_estimate_basis(void* ctx, const spcn_image* img, const spcn_params* params,
                        spcn_stats* out, void* stream) {
  if (!ctx || !image_ok(img) || !params_ok(params) || !out) return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  const int rc = run_estimate_basis(c, img, params, out, static_cast<cudaStream_t>(stream));
  out->status = rc;
  return rc;
}

int spcn_stain_percentile(void* ctx, const spcn_image* img, const spcn_stats* st,
                          const spcn_params* params, double* p99_out, void* stream) {
  if (!ctx || !image_ok(img) || !params_ok(params) || !p99_out) return SPCN_ERR_INVALID_ARG;
  int rc = stats_ok(st, (params->flags & SPCN_FLAG_H_PINV) != 0);
  if (rc) return rc;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry g = make_geometry(img, nullptr, 0, c->err);
  const bool pinv = (params->flags & SPCN_FLAG_H_PINV) != 0;
  rc = launch_build_model(c, c->model, st->W, st->i0, params->lambda, nullptr, s, pinv);
  if (rc) return rc;
  const double ones[2] = {1.0, 1.0};
  rc = launch_percentile_passes(c, g, c->model, params->white_thresh, (double)params->stain_pct,
                                st->p99, host_table_hexp(st->W, st->i0, params->lambda), ones, s,
                                pinv);
  if (rc) return rc;
  double p[2];
  SPCN_CUDA_TRY(cudaMemcpyAsync(p, c->sel->p99, sizeof(p), cudaMemcpyDeviceToHost, s));
  int err = 0;
  rc = read_error(c, s, &err);
  if (rc) return rc;
  p99_out[0] = p[0];
  p99_out[1] = p[1];
  return err;
}

int spcn_stain_densities(void* ctx, const spcn_image* img, const spcn_stats* st,
                         const spcn_params* params, float* H, int64_t h_stride, void* stream) {
  if (!ctx || !image_ok(img) || !params_ok(params) || !H) return SPCN_ERR_INVALID_ARG;
  if (h_stride < (int64_t)img->width * img->height) return SPCN_ERR_INVALID_ARG;
  int rc = stats_ok(st, true);   // the percentiles are not used here
  if (rc) return rc;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry g = make_geometry(img, nullptr, 0, c->err);
  const bool pinv = (params->flags & SPCN_FLAG_H_PINV) != 0;
  rc = launch_build_model(c, c->model, st->W, st->i0, params->lambda, nullptr, s, pinv);
  if (rc) return rc;
  return launch_density(c, g, c->model, H, h_stride, s, pinv);
}

int spcn_normalize(void* ctx, const spcn_image* src, const spcn_stats* src_st,
                   const spcn_stats* tgt_st, const spcn_params* params, uint8_t* out,
                   int64_t out_pitch, double* src_p99_out, void* stream) {
  if (!ctx || !image_ok(src) || !params_ok(params) || !out) return SPCN_ERR_INVALID_ARG;
  if (out_pitch < 3ll * src->width) return SPCN_ERR_INVALID_ARG;
  const bool signed_p99 = (params->flags & SPCN_FLAG_H_PINV) != 0;
  int rc = stats_ok(src_st, signed_p99);
  if (rc) return rc;
  rc = stats_ok(tgt_st, signed_p99);
  if (rc) return rc;
  if (params->flags & SPCN_FLAG_P99_SAMPLED)   // signed only for the pseudo-inverse
    for (int j = 0; j < 2; ++j)
      if (!std::isfinite(src_st->p99[j]) ||
          (!(params->flags & SPCN_FLAG_H_PINV) && !(src_st->p99[j] >= 0.0)))
        return SPCN_ERR_INVALID_ARG;
  // out must not overlap the source rows
  {
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(src->data);
    const uintptr_t s1 = s0 + (uintptr_t)((src->height - 1) * src->pitch_bytes + 3ll * src->width);
    const uintptr_t d0 = reinterpret_cast<uintptr_t>(out);
    const uintptr_t d1 = d0 + (uintptr_t)((src->height - 1) * out_pitch + 3ll * src->width);
    if (d0 < s1 && s0 < d1) return SPCN_ERR_INVALID_ARG;
  }
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry g = make_geometry(src, out, out_pitch, c->err);
  const bool pinv = (params->flags & SPCN_FLAG_H_PINV) != 0;
  rc = launch_build_model(c, c->model, src_st->W, src_st->i0, params->lambda, nullptr, s, pinv);
  if (rc) return rc;
  if (params->flags & SPCN_FLAG_P99_SAMPLED)   // the given percentile, no pass 1
    rc = launch_scale_given(c, src_st->p99, tgt_st->p99, s);
  else
    rc = launch_percentile_passes(c, g, c->model, params->white_thresh, (double)params->stain_pct,
                                  src_st->p99,
                                  host_table_hexp(src_st->W, src_st->i0, params->lambda),
                                  tgt_st->p99, s, pinv);
  if (rc) return rc;
  const spcn_stats to = output_target(tgt_st, params);
  rc = launch_recon(c, g, c->model, to.W, to.i0, s, pinv);
  if (rc) return rc;
  if (src_p99_out) {
    double p[2];
    SPCN_CUDA_TRY(cudaMemcpyAsync(p, c->sel->p99, sizeof(p), cudaMemcpyDeviceToHost, s));
    int err = 0;
    rc = read_error(c, s, &err);
    if (rc) return rc;
    src_p99_out[0] = p[0];
    src_p99_out[1] = p[1];
    return err;
  }
  return SPCN_OK;
}

int spcn_kernel_timing(void* ctx, int enable) {
  if (!ctx) return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  const int rc = drain_timing(c);
  for (int k = 0; k < SPCN_KERNEL_COUNT; ++k) { c->kernel_ms[k] = 0.0; c->kernel_n[k] = 0; }
  c->timing = enable != 0;
  return rc;
}

int spcn_kernel_times(void* ctx, int kernel, double* total_ms, int64_t* launches) {
  if (!ctx || kernel < 0 || kernel >= SPCN_KERNEL_COUNT || !total_ms || !launches)
    return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  const int rc = drain_timing(c);
  *total_ms = c->kernel_ms[kernel];
  *launches = c->kernel_n[kernel];
  return rc;
}

int spcn_normalize_f32(void* ctx, const float* x, int32_t batch, int32_t height, int32_t width,
                       const spcn_stats* src_stats, const spcn_stats* tgt_stats, const float* wt,
                       const spcn_params* params, float* y, void* stream) {
  if (!ctx || !x || !y || !wt || !src_stats || batch < 1 || height < 1 || width < 1 ||
      !params_ok(params) || (params->flags & SPCN_FLAG_H_PINV))
    return SPCN_ERR_INVALID_ARG;
  int rc = stats_ok(tgt_stats);
  if (rc) return rc;
  for (int b = 0; b < batch; ++b) {
    rc = stats_ok(&src_stats[b]);
    if (rc) return rc;
  }
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  const spcn_stats to = output_target(tgt_stats, params);
  return launch_f32(c, false, x, nullptr, batch, (int64_t)height * width, src_stats, &to, wt,
                    params->lambda, y, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

int spcn_normalize_f32_backward(void* ctx, const float* x, const float* gy, int32_t batch,
                                int32_t height, int32_t width, const spcn_stats* src_stats,
                                const spcn_stats* tgt_stats, const float* wt,
                                const spcn_params* params, float* gx, float* gwt, void* stream) {
  if (!ctx || !x || !gy || !gx || !gwt || !wt || !src_stats || batch < 1 || height < 1 ||
      width < 1 || !params_ok(params) || (params->flags & SPCN_FLAG_H_PINV))
    return SPCN_ERR_INVALID_ARG;
  int rc = stats_ok(tgt_stats);
  if (rc) return rc;
  for (int b = 0; b < batch; ++b) {
    rc = stats_ok(&src_stats[b]);
    if (rc) return rc;
  }
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  const spcn_stats to = output_target(tgt_stats, params);
  return launch_f32(c, true, x, gy, batch, (int64_t)height * width, src_stats, &to, wt,
                    params->lambda, nullptr, gx, gwt, static_cast<cudaStream_t>(stream));
}

int spcn_normalize_estimated(void* ctx, const spcn_image* src, const spcn_stats* tgt_st,
                             const spcn_params* params, uint8_t* out, int64_t out_pitch,
                             spcn_stats* src_st_out, void* stream) {
  if (!ctx || !image_ok(src) || !params_ok(params) || !out) return SPCN_ERR_INVALID_ARG;
  if (out_pitch < 3ll * src->width) return SPCN_ERR_INVALID_ARG;
  int rc = stats_ok(tgt_st, (params->flags & SPCN_FLAG_H_PINV) != 0);
  if (rc) return rc;
  {
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(src->data);
    const uintptr_t s1 = s0 + (uintptr_t)((src->height - 1) * src->pitch_bytes + 3ll * src->width);
    const uintptr_t d0 = reinterpret_cast<uintptr_t>(out);
    const uintptr_t d1 = d0 + (uintptr_t)((src->height - 1) * out_pitch + 3ll * src->width);
    if (d0 < s1 && s0 < d1) return SPCN_ERR_INVALID_ARG;
  }
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // basis estimation, left on the device; unless the sample percentile is
  // the one Eq. 3 uses, it only places pass 1's window
  rc = launch_estimate_basis(c, src, params, s, !(params->flags & SPCN_FLAG_P99_SAMPLED));
  if (rc) return rc;
  // the basis estimation's final table (estimated basis and i0, this lambda)
  // is the source table; the window comes from the sample P99
  const Model* m = c->model_b;
  const Geometry g = make_geometry(src, out, out_pitch, c->err);
  const bool pinv = (params->flags & SPCN_FLAG_H_PINV) != 0;
  if (params->flags & SPCN_FLAG_P99_SAMPLED) {   // the sample percentile, no pass 1
    rc = launch_scale_from_basis(c, m, &c->bs->sel, &c->bs->status, tgt_st->p99, s);
    if (rc) return rc;
  } else {
    Window* wdev = static_cast<Window*>(c->wdev);
    rc = launch_window_from_basis(c, m, c->model_b, &c->bs->sel, &c->bs->status, wdev, s);
    if (rc) return rc;
    rc = launch_percentile_passes_dev(c, g, m, params->white_thresh, (double)params->stain_pct,
                                      wdev, tgt_st->p99, s, pinv);
    if (rc) return rc;
  }
  const spcn_stats to = output_target(tgt_st, params);
  rc = launch_recon(c, g, m, to.W, to.i0, s, pinv);
  if (rc) return rc;
  if (src_st_out) {
    memset(src_st_out, 0, sizeof(*src_st_out));
    rc = finish_estimate_basis(c, src_st_out, s);   // waits; basis status
    double p[2];
    SPCN_CUDA_TRY(cudaMemcpyAsync(p, c->sel->p99, sizeof(p), cudaMemcpyDeviceToHost, s));
    int err = 0;
    const int rc2 = read_error(c, s, &err);
    if (rc2) return rc2;
    src_st_out->p99[0] = p[0];   // the percentile the scale used (exact unless sampled)
    src_st_out->p99[1] = p[1];
    src_st_out->status = rc ? rc : err;
    return rc ? rc : err;
  }
  return SPCN_OK;
}

int spcn_stain_densities_estimated(void* ctx, const spcn_image* img, const spcn_params* params,
                                   float* H, int64_t h_stride, spcn_stats* st_out,
                                   void* stream) {
  if (!ctx || !image_ok(img) || !params_ok(params) || !H) return SPCN_ERR_INVALID_ARG;
  if (h_stride < (int64_t)img->width * img->height) return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = launch_estimate_basis(c, img, params, s);
  if (rc) return rc;
  // the basis estimation's final table is the density table
  rc = launch_check_basis(c, c->model_b, &c->bs->status, s);
  if (rc) return rc;
  const Geometry g = make_geometry(img, nullptr, 0, c->err);
  rc = launch_density(c, g, c->model_b, H, h_stride, s, (params->flags & SPCN_FLAG_H_PINV) != 0);
  if (rc) return rc;
  if (st_out) {
    memset(st_out, 0, sizeof(*st_out));
    rc = finish_estimate_basis(c, st_out, s);   // waits; clears the error word it reports
    if (rc) return rc;
    int err = 0;
    rc = read_error(c, s, &err);
    if (rc) return rc;
    st_out->status = err;
    return err;
  }
  return SPCN_OK;
}

int spcn_synchronize(void* ctx, void* stream) {
  if (!ctx) return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  int err = 0;
  const int rc = read_error(c, static_cast<cudaStream_t>(stream), &err);
  return rc ? rc : err;
}

int spcn_debug_barrier_timeout(void* ctx, int32_t extra_arrivals, int64_t timeout_ns,
                               void* stream) {
  if (!ctx || extra_arrivals < 0 || timeout_ns <= 0 || timeout_ns > 10000000000ll)
    return SPCN_ERR_INVALID_ARG;
  Context* c = static_cast<Context*>(ctx);
  DeviceGuard guard(c->device);
  if (!guard.ok) return SPCN_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = launch_debug_barrier(c, extra_arrivals, (long long)timeout_ns, s);
  if (rc) return rc;
  int err = 0;
  const int rc2 = read_error(c, s, &err);
  return rc2 ? rc2 : err;
}

}  // extern "C"
