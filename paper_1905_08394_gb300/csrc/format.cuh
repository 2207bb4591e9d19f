// Device helpers: load / store one complex entry of the running tensor G in
// each storage format, and the power-of-two scale rule of the per-step
// renormalisation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.h"

namespace peps {

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_bf16(uint32_t w) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
  return __bfloat1622float2(h);
}
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_f16(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2 *>(&w);
  return __half22float2(h);
}

// Split v into hi + lo (both 16-bit); returns the packed words and the
// stored value hi + lo (exact in fp32).
template <bool BF>
__device__ __forceinline__ float2 split16(float2 v, uint32_t &hi, uint32_t &lo) {
  if (BF) {
    hi = pack_bf16(v.x, v.y);
    float2 h = unpack_bf16(hi);
    lo = pack_bf16(v.x - h.x, v.y - h.y);
    float2 l = unpack_bf16(lo);
    return make_float2(h.x + l.x, h.y + l.y);
  } else {
    hi = pack_f16(v.x, v.y);
    float2 h = unpack_f16(hi);
    lo = pack_f16(v.x - h.x, v.y - h.y);
    float2 l = unpack_f16(lo);
    return make_float2(h.x + l.x, h.y + l.y);
  }
}

template <int FMT>
__device__ __forceinline__ float2 load_g(const void *base, int64_t e, int64_t plane) {
  if (FMT == FMT_F32 || FMT == FMT_TF32) {
    return reinterpret_cast<const float2 *>(base)[e];
  } else if (FMT == FMT_BF16) {
    return unpack_bf16(reinterpret_cast<const uint32_t *>(base)[e]);
  } else if (FMT == FMT_FP16) {
    return unpack_f16(reinterpret_cast<const uint32_t *>(base)[e]);
  } else if (FMT == FMT_BF16X2) {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(base);
    float2 h = unpack_bf16(p[e]);
    float2 l = unpack_bf16(p[plane / 2 + e]);
    return make_float2(h.x + l.x, h.y + l.y);
  } else {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(base);
    float2 h = unpack_f16(p[e]);
    float2 l = unpack_f16(p[plane / 2 + e]);
    return make_float2(h.x + l.x, h.y + l.y);
  }
}

// Store v; returns the value actually stored (after rounding).
template <int FMT>
__device__ __forceinline__ float2 store_g(void *base, int64_t e, int64_t plane, float2 v) {
  if (FMT == FMT_F32) {
    reinterpret_cast<float2 *>(base)[e] = v;
    return v;
  } else if (FMT == FMT_TF32) {
    float2 r = make_float2(round_tf32(v.x), round_tf32(v.y));
    reinterpret_cast<float2 *>(base)[e] = r;
    return r;
  } else if (FMT == FMT_BF16) {
    uint32_t w = pack_bf16(v.x, v.y);
    reinterpret_cast<uint32_t *>(base)[e] = w;
    return unpack_bf16(w);
  } else if (FMT == FMT_FP16) {
    uint32_t w = pack_f16(v.x, v.y);
    reinterpret_cast<uint32_t *>(base)[e] = w;
    return unpack_f16(w);
  } else {
    uint32_t hi, lo;
    float2 r = split16<FMT == FMT_BF16X2>(v, hi, lo);
    uint32_t *p = reinterpret_cast<uint32_t *>(base);
    p[e] = hi;
    p[plane / 2 + e] = lo;
    return r;
  }
}

// Power-of-two scale of one absorption step.  The input's stored entries are
// bounded by mu (max of |Re|, |Im|) and the operand's column sums by beta, so
// every output entry is bounded by mu*beta; the step multiplies its output by
// 2^x with x = target - ceil(log2(mu*beta)), which keeps the stored output at
// most 2^target.  Exact (power of two), deterministic (every CTA computes the
// same x from the same inputs).
__device__ __forceinline__ int step_scale_exp(float mu, float beta, int target) {
  double p = (double)mu * (double)beta;
  if (!(p > 0.0) || !isfinite(p)) return 0;
  int e;
  double f = frexp(p, &e);  // p = f * 2^e, f in [0.5, 1)
  int ce = (f == 0.5) ? e - 1 : e;
  int x = target - ce;
  if (x > 120) x = 120;
  if (x < -120) x = -120;
  return x;
}

__device__ __forceinline__ float max_abs2(float2 v) {
  return fmaxf(fabsf(v.x), fabsf(v.y));
}

}  // namespace peps
