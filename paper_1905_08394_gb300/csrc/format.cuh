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

__device__ __forceinline__ float max_abs2(float2 v) {
  return fmaxf(fabsf(v.x), fabsf(v.y));
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

// Store 8 consecutive complex entries dest0 .. dest0+7 (dest0 % 8 == 0) from
// 16 floats (re, im interleaved) scaled by 2^x, with 16-byte vector stores.
// Returns the max |stored component|.
// 2^x as a float, x in [-126, 127] (exact).
__device__ __forceinline__ float pow2f(int x) { return __int_as_float((127 + x) << 23); }

// Store 8 consecutive complex entries dest0 .. dest0+7 (dest0 % 8 == 0) from
// 16 floats (re, im interleaved) multiplied by sc (a power of two), with
// 16-byte vector stores.  Returns the max |scaled component| before rounding
// to the storage format (step_scale_exp allows for the rounding).
template <int FMT>
__device__ __forceinline__ float store8_g(void *base, int64_t dest0, int64_t plane,
                                          const float (&v)[16], float sc) {
  float m = 0.f;
  float o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    o[i] = v[i] * sc;
    m = fmaxf(m, fabsf(o[i]));
  }
  if (FMT == FMT_F32 || FMT == FMT_TF32) {
    if (FMT == FMT_TF32) {
#pragma unroll
      for (int i = 0; i < 16; ++i) o[i] = round_tf32(o[i]);
    }
    uint4 *d = reinterpret_cast<uint4 *>(reinterpret_cast<float2 *>(base) + dest0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      d[i] = make_uint4(__float_as_uint(o[4 * i]), __float_as_uint(o[4 * i + 1]),
                        __float_as_uint(o[4 * i + 2]), __float_as_uint(o[4 * i + 3]));
  } else if (FMT == FMT_BF16 || FMT == FMT_FP16) {
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      w[j] = FMT == FMT_BF16 ? pack_bf16(o[2 * j], o[2 * j + 1]) : pack_f16(o[2 * j], o[2 * j + 1]);
    uint4 *d = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(base) + dest0);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
  } else {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (FMT == FMT_BF16X2) {
        hi[j] = pack_bf16(o[2 * j], o[2 * j + 1]);
        const float2 h = unpack_bf16(hi[j]);
        lo[j] = pack_bf16(o[2 * j] - h.x, o[2 * j + 1] - h.y);
      } else {
        hi[j] = pack_f16(o[2 * j], o[2 * j + 1]);
        const float2 h = unpack_f16(hi[j]);
        lo[j] = pack_f16(o[2 * j] - h.x, o[2 * j + 1] - h.y);
      }
    }
    uint32_t *p = reinterpret_cast<uint32_t *>(base);
    uint4 *dh = reinterpret_cast<uint4 *>(p + dest0);
    uint4 *dl = reinterpret_cast<uint4 *>(p + plane / 2 + dest0);
    dh[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    dh[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    dl[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    dl[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
  }
  return m;
}

// 8 complex entries (16 floats, re / im interleaved) in a storage format:
// F32 / TF32 two words per entry; BF16 / FP16 one word (re, im) per entry;
// the split forms one word per entry in each of the hi and lo planes.
template <int FMT>
struct Packed8 {
  uint32_t w[(FMT == FMT_F32 || FMT == FMT_TF32 || FMT == FMT_BF16X2 || FMT == FMT_FP16X2) ? 16 : 8];
};

// v * sc (sc a power of two) rounded to the storage format; returns the max
// |scaled component| before rounding (step_scale_exp allows for the rounding).
// Packed FP32 pairs (sm_100 and later): one instruction for two lanes of
// arithmetic, the same IEEE round-to-nearest results as two scalar ones.
__device__ __forceinline__ void mul2(float a0, float a1, float b0, float b1, float &r0, float &r1) {
  unsigned long long a, b, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r0), "=f"(r1) : "l"(r));
}
__device__ __forceinline__ void sub2(float a0, float a1, float b0, float b1, float &r0, float &r1) {
  unsigned long long a, b, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r0), "=f"(r1) : "l"(r));
}
// max(a, |b|, |c|)
__device__ __forceinline__ float max_abs3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(fabsf(b)), "f"(fabsf(c)));
  return r;
}

template <int FMT>
__device__ __forceinline__ float pack8(const float (&v)[16], float sc, Packed8<FMT> &p) {
  float m = 0.f;
  float o[16];
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    mul2(v[i], v[i + 1], sc, sc, o[i], o[i + 1]);
    m = max_abs3(m, o[i], o[i + 1]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (FMT == FMT_F32) {
      p.w[2 * j] = __float_as_uint(o[2 * j]);
      p.w[2 * j + 1] = __float_as_uint(o[2 * j + 1]);
    } else if (FMT == FMT_TF32) {
      p.w[2 * j] = __float_as_uint(round_tf32(o[2 * j]));
      p.w[2 * j + 1] = __float_as_uint(round_tf32(o[2 * j + 1]));
    } else if (FMT == FMT_BF16) {
      p.w[j] = pack_bf16(o[2 * j], o[2 * j + 1]);
    } else if (FMT == FMT_FP16) {
      p.w[j] = pack_f16(o[2 * j], o[2 * j + 1]);
    } else {
      // hi = the nearest 16-bit value, lo = the rounded remainder
      constexpr bool BF = FMT == FMT_BF16X2;
      p.w[j] = BF ? pack_bf16(o[2 * j], o[2 * j + 1]) : pack_f16(o[2 * j], o[2 * j + 1]);
      const float2 h = BF ? unpack_bf16(p.w[j]) : unpack_f16(p.w[j]);
      float d0, d1;
      sub2(o[2 * j], o[2 * j + 1], h.x, h.y, d0, d1);
      p.w[8 + j] = BF ? pack_bf16(d0, d1) : pack_f16(d0, d1);
    }
  }
  return m;
}

// Store entries j0 .. j0+W-1 of p at dest .. dest+W-1 (dest % W == 0), with
// vector stores of up to 16 bytes.
template <int W>
__device__ __forceinline__ void store_words(uint32_t *d, const uint32_t *w) {
  if (W == 1) {
    d[0] = w[0];
  } else if (W == 2) {
    *reinterpret_cast<uint2 *>(d) = make_uint2(w[0], w[1]);
  } else {
#pragma unroll
    for (int i = 0; i < W; i += 4)
      *reinterpret_cast<uint4 *>(d + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
  }
}
template <int FMT, int W>
__device__ __forceinline__ void store_run(void *base, int64_t dest, int64_t plane,
                                          const Packed8<FMT> &p, int j0) {
  uint32_t *b = reinterpret_cast<uint32_t *>(base);
  if (FMT == FMT_F32 || FMT == FMT_TF32) {
    store_words<2 * W>(b + 2 * dest, p.w + 2 * j0);
  } else if (FMT == FMT_BF16 || FMT == FMT_FP16) {
    store_words<W>(b + dest, p.w + j0);
  } else {
    store_words<W>(b + dest, p.w + j0);
    store_words<W>(b + plane / 2 + dest, p.w + 8 + j0);
  }
}

// 8 consecutive complex entries e0 .. e0+7 (e0 % 8 == 0) in a storage
// format, loaded with 16-byte vector loads into raw words (so that a load can
// be issued early and unpacked later), and unpacked to float2.
struct Raw8 {
  uint4 w[4];
};
template <int FMT>
__device__ __forceinline__ void load8_raw(const void *base, int64_t e0, int64_t plane, Raw8 &r) {
  if (FMT == FMT_F32 || FMT == FMT_TF32) {
    const uint4 *s = reinterpret_cast<const uint4 *>(reinterpret_cast<const float2 *>(base) + e0);
#pragma unroll
    for (int i = 0; i < 4; ++i) r.w[i] = s[i];
  } else if (FMT == FMT_BF16 || FMT == FMT_FP16) {
    const uint4 *s = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint32_t *>(base) + e0);
    r.w[0] = s[0];
    r.w[1] = s[1];
  } else {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(base);
    const uint4 *sh = reinterpret_cast<const uint4 *>(p + e0);
    const uint4 *sl = reinterpret_cast<const uint4 *>(p + plane / 2 + e0);
    r.w[0] = sh[0];
    r.w[1] = sh[1];
    r.w[2] = sl[0];
    r.w[3] = sl[1];
  }
}
template <int FMT>
__device__ __forceinline__ void unpack8(const Raw8 &r, float2 (&f)[8]) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(r.w);
  if (FMT == FMT_F32 || FMT == FMT_TF32) {
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = make_float2(__uint_as_float(w[2 * j]), __uint_as_float(w[2 * j + 1]));
  } else if (FMT == FMT_BF16) {
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = unpack_bf16(w[j]);
  } else if (FMT == FMT_FP16) {
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = unpack_f16(w[j]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 h = FMT == FMT_BF16X2 ? unpack_bf16(w[j]) : unpack_f16(w[j]);
      const float2 l = FMT == FMT_BF16X2 ? unpack_bf16(w[8 + j]) : unpack_f16(w[8 + j]);
      f[j] = make_float2(h.x + l.x, h.y + l.y);
    }
  }
}

// Power-of-two scale of one absorption step.  The input's entries are bounded
// by mu (max of |Re|, |Im| of the previous step's scaled output, taken before
// rounding to the storage format; the factor 1 + 2^-7 covers that rounding,
// at most 2^-8 relative for bf16) and the operand's column sums by beta, so
// every output entry is bounded by mu*beta; the step multiplies its output by
// 2^x with x = target - ceil(log2(mu*beta)), which keeps the stored output at
// most 2^target.  Exact (power of two), deterministic (every CTA computes the
// same x from the same inputs).
__device__ __forceinline__ int step_scale_exp(float mu, float beta, int target) {
  double p = (double)mu * (double)beta * (1.0 + 1.0 / 128.0);
  if (!(p > 0.0) || !isfinite(p)) return 0;
  int e;
  double f = frexp(p, &e);  // p = f * 2^e, f in [0.5, 1)
  int ce = (f == 0.5) ? e - 1 : e;
  int x = target - ce;
  if (x > 120) x = 120;
  if (x < -120) x = -120;
  return x;
}

}  // namespace peps
