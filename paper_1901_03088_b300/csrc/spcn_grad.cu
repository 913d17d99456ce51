// Differentiable form of the normalisation (Eq. 1-4) on float images, for use
// inside training pipelines: images are FP32 intensities in [0, 255], planar
// (batch, 3, H, W).  The forward computes y = i0_t exp(-W_t (s * h(x))), with
// h the Eq. 2 lasso of the source basis; the backward recomputes h (nothing
// is stored between the two) and returns dL/dx and dL/dW_t through the
// active-set solution of the lasso, the log of Eq. 1 and the exp of Eq. 4.
// The percentile scale s, the source basis and both i0 are constants.
#include <math.h>

#include <cmath>

#include "spcn_context.h"
#include "spcn_internal.cuh"

namespace spcn {

constexpr int kF32MaxBatch = 192;   // images per launch (their constants travel as kernel parameters)
constexpr int kF32Threads = 256;

// Per-image constants of the source side.
struct F32Img {
  float wd[6];      // ln2 * W_s[c,j] / G_jj, column-major: wd[3j + c]
  float ws[6];      // W_s, column-major
  float lam[2];     // lambda / G_jj
  float l2i0[3];    // log2 i0_s
  float nrho1, nrho2, kappa;
  float ginv[3];    // G^-1 entries (00, 01, 11)
  float ig11, ig22; // 1 / G_jj
  float s[2];       // Eq. 3 scale
};

struct F32Args {
  const float* x;
  const float* gy;
  float* y;
  float* gx;
  const float* wt;        // target basis, device, column-major (6)
  double* partials;       // [grid][6] dL/dW_t block sums (backward)
  double* acc;            // FP64 running sum of a batch that takes several launches
  float* gwt;             // dL/dW_t (written by the last launch)
  unsigned* ticket;       // last-block ticket (returns to 0 after every launch)
  int first, last;        // this launch is the first / last of its batch
  int* err;               // the context's error word (bounds-checked build)
  int64_t hw;             // pixels per image
  int batch;              // images in this launch
  float l2i0t[3];         // log2 i0_t
  F32Img img[kF32MaxBatch];
};

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx_g(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-image constants held in registers for the pixel loop.
struct F32Reg {
  float wd0, wd1, wd2, wd3, wd4, wd5, lam0, lam1, l20, l21, l22;
  float nrho1, nrho2, kappa, s0, s1;
};

__device__ __forceinline__ F32Reg f32_reg(const F32Img& I) {
  F32Reg r;
  r.wd0 = I.wd[0]; r.wd1 = I.wd[1]; r.wd2 = I.wd[2];
  r.wd3 = I.wd[3]; r.wd4 = I.wd[4]; r.wd5 = I.wd[5];
  r.lam0 = I.lam[0]; r.lam1 = I.lam[1];
  r.l20 = I.l2i0[0]; r.l21 = I.l2i0[1]; r.l22 = I.l2i0[2];
  r.nrho1 = I.nrho1; r.nrho2 = I.nrho2; r.kappa = I.kappa;
  r.s0 = I.s[0]; r.s1 = I.s[1];
  return r;
}

// Densities of one pixel from its intensities (closed form of the lasso).
__device__ __forceinline__ void f32_solve(const F32Reg& R, float x0, float x1, float x2,
                                          float& h1, float& h2) {
  const float v0 = R.l20 - lg2_approx(fmaxf(x0, 1.f));   // log2(i0/x); ln2 is folded into wd
  const float v1 = R.l21 - lg2_approx(fmaxf(x1, 1.f));
  const float v2 = R.l22 - lg2_approx(fmaxf(x2, 1.f));
  const float d1 = fmaf(R.wd2, v2, fmaf(R.wd1, v1, fmaf(R.wd0, v0, -R.lam0)));
  const float d2 = fmaf(R.wd5, v2, fmaf(R.wd4, v1, fmaf(R.wd3, v0, -R.lam1)));
  const float D1 = fmaxf(d1, 0.f), D2 = fmaxf(d2, 0.f);
  h1 = fminf(D1, fmaxf(0.f, R.kappa * fmaf(R.nrho1, D2, D1)));
  h2 = fminf(D2, fmaxf(0.f, R.kappa * fmaf(R.nrho2, D1, D2)));
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }
__device__ __forceinline__ float& comp(float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Four consecutive pixels per thread (16-byte accesses per plane) when the
// image size and pointers allow it, one pixel per step otherwise.
__global__ void __launch_bounds__(kF32Threads) k_f32_forward(F32Args a) {
  const int b = blockIdx.y;
  if (!SPCN_CHECK(b < a.batch && b < kF32MaxBatch, a.err)) return;
  const F32Reg R = f32_reg(a.img[b]);
  float wt[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) wt[k] = __ldg(a.wt + k);
  const float l2t0 = a.l2i0t[0], l2t1 = a.l2i0t[1], l2t2 = a.l2i0t[2];
  const float* xb = a.x + (int64_t)b * 3 * a.hw;
  float* yb = a.y + (int64_t)b * 3 * a.hw;
  const bool vec = (a.hw & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.y)) & 15) == 0;
  const int64_t n4 = vec ? a.hw >> 2 : 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
    float4 X0 = ld4(xb + 4 * q), X1 = ld4(xb + a.hw + 4 * q), X2 = ld4(xb + 2 * a.hw + 4 * q);
    float4 Y0, Y1, Y2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float h1, h2;
      f32_solve(R, comp(X0, k), comp(X1, k), comp(X2, k), h1, h2);
      const float sh1 = R.s0 * h1, sh2 = R.s1 * h2;
      comp(Y0, k) = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[0], sh1, wt[3] * sh2), l2t0));
      comp(Y1, k) = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[1], sh1, wt[4] * sh2), l2t1));
      comp(Y2, k) = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[2], sh1, wt[5] * sh2), l2t2));
    }
    st4(yb + 4 * q, Y0);
    st4(yb + a.hw + 4 * q, Y1);
    st4(yb + 2 * a.hw + 4 * q, Y2);
  }
  for (int64_t p = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.hw;
       p += (int64_t)gridDim.x * blockDim.x) {
    float h1, h2;
    f32_solve(R, xb[p], xb[a.hw + p], xb[2 * a.hw + p], h1, h2);
    const float sh1 = R.s0 * h1, sh2 = R.s1 * h2;
    yb[p] = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[0], sh1, wt[3] * sh2), l2t0));
    yb[a.hw + p] = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[1], sh1, wt[4] * sh2), l2t1));
    yb[2 * a.hw + p] = ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[2], sh1, wt[5] * sh2), l2t2));
  }
}

struct F32Back {
  float g00, g01, g11;   // G^-1
  float ig11, ig22;
  float ws0, ws1, ws2, ws3, ws4, ws5;
};

// One pixel of the backward: accumulates dL/dW_t into gw, returns dL/dx.
__device__ __forceinline__ void f32_back_px(const F32Reg& R, const F32Back& B, const float (&wt)[6],
                                            float l2t0, float l2t1, float l2t2, float x0, float x1,
                                            float x2, float g0, float g1, float g2, float (&gw)[6],
                                            float& gx0, float& gx1, float& gx2) {
  float h1, h2;
  f32_solve(R, x0, x1, x2, h1, h2);
  const float sh1 = R.s0 * h1, sh2 = R.s1 * h2;
  // Eq. 4 again (y is not stored), then dL/dV'_c = -g_c y_c
  const float gv0 = -g0 * ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[0], sh1, wt[3] * sh2), l2t0));
  const float gv1 = -g1 * ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[1], sh1, wt[4] * sh2), l2t1));
  const float gv2 = -g2 * ex2_approx_g(fmaf(-1.4426950408889634f, fmaf(wt[2], sh1, wt[5] * sh2), l2t2));
  gw[0] = fmaf(gv0, sh1, gw[0]);
  gw[1] = fmaf(gv1, sh1, gw[1]);
  gw[2] = fmaf(gv2, sh1, gw[2]);
  gw[3] = fmaf(gv0, sh2, gw[3]);
  gw[4] = fmaf(gv1, sh2, gw[4]);
  gw[5] = fmaf(gv2, sh2, gw[5]);
  const float gh1 = R.s0 * fmaf(wt[2], gv2, fmaf(wt[1], gv1, wt[0] * gv0));
  const float gh2 = R.s1 * fmaf(wt[5], gv2, fmaf(wt[4], gv1, wt[3] * gv0));
  // through the active-set solution of the lasso (branch-free)
  const bool a1 = h1 > 0.f, a2 = h2 > 0.f;
  const float gb1 = fmaf(B.g00, gh1, B.g01 * gh2), gb2 = fmaf(B.g01, gh1, B.g11 * gh2);
  const float gc1 = (a1 && a2) ? gb1 : (a1 ? gh1 * B.ig11 : 0.f);
  const float gc2 = (a1 && a2) ? gb2 : (a2 ? gh2 * B.ig22 : 0.f);
  // dL/dv_c, then Eq. 1: dv_c/dx_c = -1/x_c above the clamp
  gx0 = x0 > 1.f ? __fdividef(-fmaf(B.ws0, gc1, B.ws3 * gc2), x0) : 0.f;
  gx1 = x1 > 1.f ? __fdividef(-fmaf(B.ws1, gc1, B.ws4 * gc2), x1) : 0.f;
  gx2 = x2 > 1.f ? __fdividef(-fmaf(B.ws2, gc1, B.ws5 * gc2), x2) : 0.f;
}

__device__ __forceinline__ float2 ld2(const float* p) { return __ldcs(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st2(float* p, float2 v) { __stcs(reinterpret_cast<float2*>(p), v); }

// One wave of blocks (blockIdx.y = image, so the image's constants are
// uniform), each looping over its image two pixels at a time (8-byte accesses
// per plane, the next pair's loads in flight while the current pair is
// computed) when the size and pointers allow it, one pixel otherwise.  The
// dL/dW_t block sums go to `partials`; the block that finishes last (a
// ticket that returns to zero) adds them in block order with a fixed tree,
// so reruns are bit-identical, and writes gwt or the running sum.
constexpr int kF32BwdBlocksPerSm = 4;   // 64 registers: room for the prefetched pair
__global__ void __launch_bounds__(kF32Threads, kF32BwdBlocksPerSm) k_f32_backward(F32Args a) {
  __shared__ double s_red[kF32Threads / 32][6];
  __shared__ int s_last;
  const int b = blockIdx.y;
  if (!SPCN_CHECK(b < a.batch && b < kF32MaxBatch, a.err)) return;
  const F32Img& I = a.img[b];
  const F32Reg R = f32_reg(I);
  F32Back B;
  B.g00 = I.ginv[0]; B.g01 = I.ginv[1]; B.g11 = I.ginv[2];
  B.ig11 = I.ig11; B.ig22 = I.ig22;
  B.ws0 = I.ws[0]; B.ws1 = I.ws[1]; B.ws2 = I.ws[2];
  B.ws3 = I.ws[3]; B.ws4 = I.ws[4]; B.ws5 = I.ws[5];
  float wt[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) wt[k] = __ldg(a.wt + k);
  const float l2t0 = a.l2i0t[0], l2t1 = a.l2i0t[1], l2t2 = a.l2i0t[2];
  float gw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int64_t base = (int64_t)b * 3 * a.hw;
  const float* xb = a.x + base;
  const float* gb = a.gy + base;
  float* gxb = a.gx + base;
  const bool vec = (a.hw & 1) == 0 &&
                   ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.gy) |
                     reinterpret_cast<uintptr_t>(a.gx)) & 7) == 0;
  const int64_t n2 = vec ? a.hw >> 1 : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the next pair's six loads are issued before the current pair is computed
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float2 nX0, nX1, nX2, nG0, nG1, nG2;
  if (q < n2) {
    nX0 = ld2(xb + 2 * q); nX1 = ld2(xb + a.hw + 2 * q); nX2 = ld2(xb + 2 * a.hw + 2 * q);
    nG0 = ld2(gb + 2 * q); nG1 = ld2(gb + a.hw + 2 * q); nG2 = ld2(gb + 2 * a.hw + 2 * q);
  }
  for (; q < n2; q += stride) {
    const float2 X0 = nX0, X1 = nX1, X2 = nX2, G0 = nG0, G1 = nG1, G2 = nG2;
    const int64_t qn = q + stride;
    if (qn < n2) {
      nX0 = ld2(xb + 2 * qn); nX1 = ld2(xb + a.hw + 2 * qn); nX2 = ld2(xb + 2 * a.hw + 2 * qn);
      nG0 = ld2(gb + 2 * qn); nG1 = ld2(gb + a.hw + 2 * qn); nG2 = ld2(gb + 2 * a.hw + 2 * qn);
    }
    float2 O0, O1, O2;
    f32_back_px(R, B, wt, l2t0, l2t1, l2t2, X0.x, X1.x, X2.x, G0.x, G1.x, G2.x, gw, O0.x, O1.x, O2.x);
    f32_back_px(R, B, wt, l2t0, l2t1, l2t2, X0.y, X1.y, X2.y, G0.y, G1.y, G2.y, gw, O0.y, O1.y, O2.y);
    st2(gxb + 2 * q, O0);
    st2(gxb + a.hw + 2 * q, O1);
    st2(gxb + 2 * a.hw + 2 * q, O2);
  }
  for (int64_t p = 2 * n2 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.hw; p += stride) {
    float o0, o1, o2;
    f32_back_px(R, B, wt, l2t0, l2t1, l2t2, xb[p], xb[a.hw + p], xb[2 * a.hw + p], gb[p],
                gb[a.hw + p], gb[2 * a.hw + p], gw, o0, o1, o2);
    gxb[p] = o0;
    gxb[a.hw + p] = o1;
    gxb[2 * a.hw + p] = o2;
  }
  // block sums of dL/dW_t in FP64, fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double x = (double)gw[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][k] = x;
  }
  __syncthreads();
  const unsigned nblocks = gridDim.x * gridDim.y;
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int w = 0; w < kF32Threads / 32; ++w) x += s_red[w][threadIdx.x];
    a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = x;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicInc(a.ticket, nblocks - 1u) == nblocks - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: every partial, thread t taking blocks t, t + 256, ...
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (unsigned i = threadIdx.x; i < nblocks; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] += __ldcg(a.partials + (size_t)i * 6 + k);
  }
  __syncthreads();   // s_red is reused
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int w = 0; w < kF32Threads / 32; ++w) x += s_red[w][threadIdx.x];
    if (!a.first) x += a.acc[threadIdx.x];
    if (a.last) a.gwt[threadIdx.x] = (float)x;
    else a.acc[threadIdx.x] = x;
  }
}

// ------------------------------------------------------------ host side
static void f32_image_consts(const spcn_stats* src, const spcn_stats* tgt, float lambda,
                             F32Img* o) {
  double g11 = 0, g22 = 0, g12 = 0;
  for (int c = 0; c < 3; ++c) {
    g11 += (double)src->W[c] * src->W[c];
    g22 += (double)src->W[3 + c] * src->W[3 + c];
    g12 += (double)src->W[c] * src->W[3 + c];
  }
  const double det = g11 * g22 - g12 * g12;
  const double ln2 = 0.69314718055994530942;
  for (int c = 0; c < 3; ++c) {
    o->wd[c] = (float)(ln2 * src->W[c] / g11);
    o->wd[3 + c] = (float)(ln2 * src->W[3 + c] / g22);
    o->ws[c] = src->W[c];
    o->ws[3 + c] = src->W[3 + c];
    o->l2i0[c] = (float)log2((double)src->i0[c]);
  }
  o->lam[0] = (float)(lambda / g11);
  o->lam[1] = (float)(lambda / g22);
  o->nrho1 = (float)(-g12 / g11);
  o->nrho2 = (float)(-g12 / g22);
  o->kappa = (float)(g11 * g22 / det);
  o->ginv[0] = (float)(g22 / det);
  o->ginv[1] = (float)(-g12 / det);
  o->ginv[2] = (float)(g11 / det);
  o->ig11 = (float)(1.0 / g11);
  o->ig22 = (float)(1.0 / g22);
  for (int j = 0; j < 2; ++j)
    o->s[j] = (float)(src->p99[j] != 0.0 ? tgt->p99[j] / src->p99[j] : 1.0);
}

// The backward's block partials live in the context's partials buffer
// (2 * 4096 * kAcc doubles): 6 per block, plus 6 for the running sum of a
// batch that takes several launches.  Each launch is reduced by its own last
// block before the next one starts, so the blocks of one launch are capped,
// not those of a batch.
constexpr size_t kF32PartialDoubles = (size_t)2 * 4096 * kAcc;
constexpr int kF32MaxBlocks = (int)((kF32PartialDoubles - 8) / 6);

int configure_grad_kernels(Context* c) {
  c->occ_f32_fwd = c->occ_f32_bwd = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_f32_fwd, k_f32_forward, kF32Threads,
                                                    0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_f32_bwd, k_f32_backward, kF32Threads,
                                                    0) != cudaSuccess)
    return SPCN_ERR_CUDA;
  return (c->occ_f32_fwd < 1 || c->occ_f32_bwd < 1) ? SPCN_ERR_CUDA : SPCN_OK;
}

int launch_f32(Context* c, bool backward, const float* x, const float* gy, int batch, int64_t hw,
               const spcn_stats* src, const spcn_stats* tgt, const float* wt, float lambda,
               float* y, float* gx, float* gwt, cudaStream_t st) {
  F32Args a;   // ~21 KB parameter block, passed by value to each launch
  // at most about 8 pixels per thread, and no more blocks than one wave holds
  int bx_work = (int)((hw + kF32Threads * 8 - 1) / (kF32Threads * 8));
  if (bx_work < 1) bx_work = 1;
  const int resident = c->num_sms * (backward ? c->occ_f32_bwd : c->occ_f32_fwd);
  const int launches = (batch + kF32MaxBatch - 1) / kF32MaxBatch;
  double* acc = c->partials + kF32PartialDoubles - 8;
  for (int l = 0; l < launches; ++l) {
    const int b0 = l * kF32MaxBatch;
    const int nb = batch - b0 < kF32MaxBatch ? batch - b0 : kF32MaxBatch;
    int bx = resident / nb;
    if (bx > bx_work) bx = bx_work;
    if (bx < 1) bx = 1;
    if (backward && bx * nb > kF32MaxBlocks) bx = kF32MaxBlocks / nb;   // nb <= 192: bx >= 85
    a.x = x + (int64_t)b0 * 3 * hw;
    a.gy = gy ? gy + (int64_t)b0 * 3 * hw : nullptr;
    a.y = y ? y + (int64_t)b0 * 3 * hw : nullptr;
    a.gx = gx ? gx + (int64_t)b0 * 3 * hw : nullptr;
    a.wt = wt;
    a.partials = c->partials;
    a.acc = acc;
    a.gwt = gwt;
    a.ticket = c->f32_ticket;
    a.err = c->err;
    a.first = l == 0;
    a.last = l == launches - 1;
    a.hw = hw;
    a.batch = nb;
    for (int k = 0; k < 3; ++k) a.l2i0t[k] = (float)log2((double)tgt->i0[k]);
    for (int i = 0; i < nb; ++i) f32_image_consts(&src[b0 + i], tgt, lambda, &a.img[i]);
    const dim3 grid(bx, nb);
    {
      TimedLaunch tl(c, backward ? SPCN_KERNEL_F32_BWD : SPCN_KERNEL_F32_FWD, st);
      if (backward) k_f32_backward<<<grid, kF32Threads, 0, st>>>(a);
      else k_f32_forward<<<grid, kF32Threads, 0, st>>>(a);
    }
    SPCN_LAUNCH_CHECK(c);
  }
  return SPCN_OK;
}

}  // namespace spcn
