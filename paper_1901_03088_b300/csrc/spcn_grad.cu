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

// Densities of one pixel from its intensities (closed form of the lasso).
__device__ __forceinline__ void f32_solve(const F32Img& I, const float (&xc)[3], float (&v)[3],
                                          float& h1, float& h2) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = I.l2i0[c] - lg2_approx(fmaxf(xc[c], 1.f));   // log2(i0/x)
  const float d1 = fmaf(I.wd[2], v[2], fmaf(I.wd[1], v[1], I.wd[0] * v[0])) - I.lam[0];
  const float d2 = fmaf(I.wd[5], v[2], fmaf(I.wd[4], v[1], I.wd[3] * v[0])) - I.lam[1];
  const float D1 = fmaxf(d1, 0.f), D2 = fmaxf(d2, 0.f);
  h1 = fminf(D1, fmaxf(0.f, I.kappa * fmaf(I.nrho1, D2, D1)));
  h2 = fminf(D2, fmaxf(0.f, I.kappa * fmaf(I.nrho2, D1, D2)));
}

__global__ void __launch_bounds__(kF32Threads) k_f32_forward(F32Args a) {
  __shared__ float s_wt[6];
  if (threadIdx.x < 6) s_wt[threadIdx.x] = a.wt[threadIdx.x];
  __syncthreads();
  // blockIdx.y selects the image, blockIdx.x strides over its pixels
  const int b = blockIdx.y;
  const F32Img& I = a.img[b];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.hw;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float* xb = a.x + (int64_t)b * 3 * a.hw + p;
    const float xc[3] = {__ldcs(xb), __ldcs(xb + a.hw), __ldcs(xb + 2 * a.hw)};
    float v[3], h1, h2;
    f32_solve(I, xc, v, h1, h2);
    const float sh1 = I.s[0] * h1, sh2 = I.s[1] * h2;
    float* yb = a.y + (int64_t)b * 3 * a.hw + p;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float vp = fmaf(s_wt[c], sh1, s_wt[3 + c] * sh2);     // Eq. 3
      __stcs(yb + c * a.hw, ex2_approx_g(fmaf(-1.4426950408889634f, vp, a.l2i0t[c])));   // Eq. 4
    }
  }
}

__global__ void __launch_bounds__(kF32Threads) k_f32_backward(F32Args a) {
  __shared__ float s_wt[6];
  __shared__ double s_red[kF32Threads / 32][6];
  if (threadIdx.x < 6) s_wt[threadIdx.x] = a.wt[threadIdx.x];
  __syncthreads();
  float gw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int b = blockIdx.y;
  const F32Img& I = a.img[b];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.hw;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = (int64_t)b * 3 * a.hw + p;
    const float xc[3] = {__ldcs(a.x + off), __ldcs(a.x + off + a.hw), __ldcs(a.x + off + 2 * a.hw)};
    const float g[3] = {__ldcs(a.gy + off), __ldcs(a.gy + off + a.hw), __ldcs(a.gy + off + 2 * a.hw)};
    float v[3], h1, h2;
    f32_solve(I, xc, v, h1, h2);
    const float sh1 = I.s[0] * h1, sh2 = I.s[1] * h2;
    float gh1 = 0.f, gh2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float vp = fmaf(s_wt[c], sh1, s_wt[3 + c] * sh2);
      const float yc = ex2_approx_g(fmaf(-1.4426950408889634f, vp, a.l2i0t[c]));
      const float gv = -g[c] * yc;                  // dL/dV'_c
      gw[c] = fmaf(gv, sh1, gw[c]);                 // dL/dW_t[c,0]
      gw[3 + c] = fmaf(gv, sh2, gw[3 + c]);         // dL/dW_t[c,1]
      gh1 = fmaf(s_wt[c], gv, gh1);
      gh2 = fmaf(s_wt[3 + c], gv, gh2);
    }
    gh1 *= I.s[0];
    gh2 *= I.s[1];
    // through the active-set solution of the lasso
    float gc1 = 0.f, gc2 = 0.f;
    if (h1 > 0.f && h2 > 0.f) {
      gc1 = fmaf(I.ginv[0], gh1, I.ginv[1] * gh2);
      gc2 = fmaf(I.ginv[1], gh1, I.ginv[2] * gh2);
    } else if (h1 > 0.f) {
      gc1 = gh1 * I.ig11;
    } else if (h2 > 0.f) {
      gc2 = gh2 * I.ig22;
    }
    float* gxb = a.gx + off;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float gvc = fmaf(I.ws[c], gc1, I.ws[3 + c] * gc2);          // dL/dv_c
      __stcs(gxb + c * a.hw, xc[c] > 1.f ? __fdividef(-gvc, xc[c]) : 0.f);   // Eq. 1
    }
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
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int w = 0; w < kF32Threads / 32; ++w) x += s_red[w][threadIdx.x];
    a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = x;
  }
}

// Sum of all block partials in a fixed order (warp k sums entry k with a
// fixed lane-strided pattern and shuffle tree); writes gwt (column-major).
__global__ void k_f32_reduce(const double* partials, int nblocks, float* gwt) {
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  if (k >= 6) return;
  double x = 0.0;
  for (int b = lane; b < nblocks; b += 32) x += partials[(size_t)b * 6 + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) gwt[k] = (float)x;
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

int launch_f32(Context* c, bool backward, const float* x, const float* gy, int batch, int64_t hw,
               const spcn_stats* src, const spcn_stats* tgt, const float* wt, float lambda,
               float* y, float* gx, float* gwt, cudaStream_t st) {
  F32Args a;   // ~17 KB parameter block, passed by value to each launch
  int bx = (int)((hw + kF32Threads * 4 - 1) / (kF32Threads * 4));   // about 4 pixels per thread
  if (bx < 1) bx = 1;
  if (bx > 1024) bx = 1024;
  const int launches = (batch + kF32MaxBatch - 1) / kF32MaxBatch;
  const size_t nblocks = (size_t)bx * batch;
  if (backward && nblocks * 6 > (size_t)2 * 4096 * kAcc) return SPCN_ERR_INVALID_ARG;
  for (int l = 0; l < launches; ++l) {
    const int b0 = l * kF32MaxBatch;
    const int nb = batch - b0 < kF32MaxBatch ? batch - b0 : kF32MaxBatch;
    a.x = x + (int64_t)b0 * 3 * hw;
    a.gy = gy ? gy + (int64_t)b0 * 3 * hw : nullptr;
    a.y = y ? y + (int64_t)b0 * 3 * hw : nullptr;
    a.gx = gx ? gx + (int64_t)b0 * 3 * hw : nullptr;
    a.wt = wt;
    a.partials = c->partials + (size_t)b0 * bx * 6;
    a.hw = hw;
    a.batch = nb;
    for (int k = 0; k < 3; ++k) a.l2i0t[k] = (float)log2((double)tgt->i0[k]);
    for (int i = 0; i < nb; ++i) f32_image_consts(&src[b0 + i], tgt, lambda, &a.img[i]);
    const dim3 grid(bx, nb);
    if (backward) k_f32_backward<<<grid, kF32Threads, 0, st>>>(a);
    else k_f32_forward<<<grid, kF32Threads, 0, st>>>(a);
    SPCN_LAUNCH_CHECK(c);
  }
  if (backward) {
    k_f32_reduce<<<1, 6 * 32, 0, st>>>(c->partials, (int)nblocks, gwt);
    SPCN_LAUNCH_CHECK(c);
  }
  return SPCN_OK;
}

}  // namespace spcn
