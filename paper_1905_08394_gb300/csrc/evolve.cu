// Circuit evolution on the PEPS: initial product state, single-qubit gate
// absorption (K1), CZ absorption with bond doubling (K2) and general
// two-qubit gates by their operator-Schmidt split (bond times the rank).
//
// Site tensor layout: complex [sigma][l][r][u][d], sigma slowest, d fastest,
// held as float-float (a hi and a lo plane of float2, value = hi + lo).  The
// CZ halves only move entries and multiply them by 0 or +-1 (exact); the
// single-qubit gates use error-free products and sums (Dekker's product via
// fma, Knuth's two-sum), so the tensors reach the operand build with about
// 2^-44 relative error instead of the 2^-24 per gate of plain FP32.
#include "common.h"
#include "format.cuh"

namespace peps {

// |0> on every site: A^0 = 1, A^1 = 0 with every auxiliary leg of dim 1
// (paper, main-text PEPS equation for the product state).  Also writes the
// scalar 1 in every storage format into the status block (the running
// tensor before the first absorption).
__global__ void k_init_sites(float2 *const *bufs, const int64_t *lo_off, int n_sites,
                             DeviceStatus *st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_sites) {
    float2 *a = bufs[i];
    a[0] = make_float2(1.f, 0.f);
    a[1] = make_float2(0.f, 0.f);
    a[lo_off[i]] = make_float2(0.f, 0.f);
    a[lo_off[i] + 1] = make_float2(0.f, 0.f);
  }
  if (i == 0) {
    st->error = 0;
    st->error_info = 0;
    st->timeout = 0;
    st->unit_f32 = make_float2(1.f, 0.f);
    st->unit_h16[0] = pack_bf16(1.f, 0.f);
    st->unit_h16[1] = 0u;
    st->unit_f16[0] = pack_f16(1.f, 0.f);
    st->unit_f16[1] = 0u;
  }
}

// ---- float-float helpers (value = hi + lo, |lo| <= ulp(hi)/2) ----
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {  // Knuth: a + b = s + e exactly
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {  // Dekker product, error term by fma
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

// (re, im) of u * a, complex float-float
__device__ __forceinline__ void cmul_ff(ff ur, ff ui, ff ar, ff ai, ff &re, ff &im) {
  re = ff_add(ff_mul(ur, ar), ff_neg(ff_mul(ui, ai)));
  im = ff_add(ff_mul(ur, ai), ff_mul(ui, ar));
}

// K1: A'^tau = sum_sigma U[tau][sigma] A^sigma (paper, main-text "onebody"
// equation), in place.  The tensor is [2][half]; each thread mixes the two
// sigma slices at positions e0, e0 + de, ..., in float-float complex
// arithmetic.
__device__ __forceinline__ void gate1_mix(const ff (&ur)[4], const ff (&ui)[4], float2 h0, float2 h1,
                                          float2 l0, float2 l1, float2 &o0h, float2 &o0l,
                                          float2 &o1h, float2 &o1l) {
  const ff a0r = {h0.x, l0.x}, a0i = {h0.y, l0.y}, a1r = {h1.x, l1.x}, a1i = {h1.y, l1.y};
  ff out[2][2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    ff r0, i0, r1, i1;
    cmul_ff(ur[2 * t], ui[2 * t], a0r, a0i, r0, i0);
    cmul_ff(ur[2 * t + 1], ui[2 * t + 1], a1r, a1i, r1, i1);
    out[t][0] = ff_add(r0, r1);
    out[t][1] = ff_add(i0, i1);
  }
  o0h = make_float2(out[0][0].hi, out[0][1].hi);
  o0l = make_float2(out[0][0].lo, out[0][1].lo);
  o1h = make_float2(out[1][0].hi, out[1][1].hi);
  o1l = make_float2(out[1][0].lo, out[1][1].lo);
}

__device__ __forceinline__ void gate1_apply(const Gate1Entry &g, int64_t e0, int64_t de) {
  const int64_t half = g.half, lo = g.lo_off;
  float2 *A = g.A;
  ff ur[4], ui[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ur[i] = {g.U_hi[i].x, g.U_lo[i].x};
    ui[i] = {g.U_hi[i].y, g.U_lo[i].y};
  }
  if ((half & 1) == 0 && (lo & 1) == 0) {
    // two neighbouring positions per thread: 16-byte loads and stores
    float4 *A4 = reinterpret_cast<float4 *>(A);
    const int64_t h4 = half >> 1, l4 = lo >> 1;
    for (int64_t p = e0; p < h4; p += de) {
      const float4 h0 = A4[p], h1 = A4[h4 + p], l0 = A4[l4 + p], l1 = A4[l4 + h4 + p];
      float2 a0h, a0l, a1h, a1l, b0h, b0l, b1h, b1l;
      gate1_mix(ur, ui, make_float2(h0.x, h0.y), make_float2(h1.x, h1.y), make_float2(l0.x, l0.y),
                make_float2(l1.x, l1.y), a0h, a0l, a1h, a1l);
      gate1_mix(ur, ui, make_float2(h0.z, h0.w), make_float2(h1.z, h1.w), make_float2(l0.z, l0.w),
                make_float2(l1.z, l1.w), b0h, b0l, b1h, b1l);
      A4[p] = make_float4(a0h.x, a0h.y, b0h.x, b0h.y);
      A4[l4 + p] = make_float4(a0l.x, a0l.y, b0l.x, b0l.y);
      A4[h4 + p] = make_float4(a1h.x, a1h.y, b1h.x, b1h.y);
      A4[l4 + h4 + p] = make_float4(a1l.x, a1l.y, b1l.x, b1l.y);
    }
    return;
  }
  for (int64_t e = e0; e < half; e += de) {
    const float2 h0 = A[e], h1 = A[half + e], l0 = A[lo + e], l1 = A[lo + half + e];
    const ff a0r = {h0.x, l0.x}, a0i = {h0.y, l0.y}, a1r = {h1.x, l1.x}, a1i = {h1.y, l1.y};
    ff out[2][2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      ff r0, i0, r1, i1;
      cmul_ff(ur[2 * t], ui[2 * t], a0r, a0i, r0, i0);
      cmul_ff(ur[2 * t + 1], ui[2 * t + 1], a1r, a1i, r1, i1);
      out[t][0] = ff_add(r0, r1);
      out[t][1] = ff_add(i0, i1);
    }
    A[e] = make_float2(out[0][0].hi, out[0][1].hi);
    A[lo + e] = make_float2(out[0][0].lo, out[0][1].lo);
    A[half + e] = make_float2(out[1][0].hi, out[1][1].hi);
    A[lo + half + e] = make_float2(out[1][0].lo, out[1][1].lo);
  }
}

// A batch of single-qubit gates on distinct sites (one per blockIdx.y).
__global__ void k_gate1(const Gate1Entry *__restrict__ entries) {
  gate1_apply(entries[blockIdx.y], (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
              (int64_t)gridDim.x * blockDim.x);
}

// K2: one half of a CZ (paper, main-text "twoqubita/b" with the exact
// projector split of CZ).  The leg `axis` grows from d to 2d with the new
// Schmidt bit s as its least significant bit:
//   projector side:  A'^tau[..., 2*i + s, ...] = delta(tau, s) A^tau[..., i, ...]
//   phase side:      A'^tau[..., 2*i + s, ...] = (-1)^(s*tau) A^tau[..., i, ...]
// With fixed_s >= 0 (a sliced CZ) the leg keeps its size and only the term
// s = fixed_s is applied.  One thread per output entry (e0, e0 + de, ...).
__device__ __forceinline__ void cz_apply(const CzEntry &g, int64_t e0, int64_t de) {
  if (g.fixed_s < 0) {
    // Bundled split, by input element: [pre][D][post] -> [pre][2D][post]
    // with pre = (tau, the legs before the axis), post = the legs after it;
    // each input element gives the outputs s = 0 and s = 1, post entries
    // apart (adjacent when the axis is the fastest leg: one 16-byte store).
    int pre_inner = 1, post = 1;
    for (int a = 0; a < g.axis; ++a) pre_inner *= g.dims[a];
    for (int a = g.axis + 1; a < 4; ++a) post *= g.dims[a];
    const int D = g.dims[g.axis];
    const int64_t total = (int64_t)2 * pre_inner * D * post;
    for (int64_t u = e0; u < total; u += de) {
      const int64_t r = u / post;
      const int post_i = (int)(u - r * post);
      const int64_t pre_i = r / D;
      const int i = (int)(r - pre_i * D);
      const int tau = (int)(pre_i / pre_inner);
      const float2 v = g.in[u], vl = g.in[g.lo_off + u];
      const float f0 = g.kind == 0 ? (tau == 0 ? 1.f : 0.f) : 1.f;
      const float f1 = g.kind == 0 ? (tau == 1 ? 1.f : 0.f) : (tau ? -1.f : 1.f);
      const int64_t o0 = (pre_i * (2 * D) + 2 * i) * post + post_i;
      if (post == 1) {
        reinterpret_cast<float4 *>(g.out)[o0 >> 1] = make_float4(f0 * v.x, f0 * v.y, f1 * v.x, f1 * v.y);
        reinterpret_cast<float4 *>(g.out + g.lo_off)[o0 >> 1] =
            make_float4(f0 * vl.x, f0 * vl.y, f1 * vl.x, f1 * vl.y);
      } else {
        g.out[o0] = make_float2(f0 * v.x, f0 * v.y);
        g.out[o0 + post] = make_float2(f1 * v.x, f1 * v.y);
        g.out[g.lo_off + o0] = make_float2(f0 * vl.x, f0 * vl.y);
        g.out[g.lo_off + o0 + post] = make_float2(f1 * vl.x, f1 * vl.y);
      }
    }
    return;
  }
  int od[4] = {g.dims[0], g.dims[1], g.dims[2], g.dims[3]};
  const bool bundle = g.fixed_s < 0;
  if (bundle) od[g.axis] *= 2;
  const int64_t half_out = (int64_t)od[0] * od[1] * od[2] * od[3];
  const int64_t total = 2 * half_out;
  for (int64_t e = e0; e < total; e += de) {
    int64_t rem = e;
    int idx[4];
    idx[3] = (int)(rem % od[3]); rem /= od[3];
    idx[2] = (int)(rem % od[2]); rem /= od[2];
    idx[1] = (int)(rem % od[1]); rem /= od[1];
    idx[0] = (int)(rem % od[0]); rem /= od[0];
    const int tau = (int)rem;
    int s;
    if (bundle) {
      s = idx[g.axis] & 1;
      idx[g.axis] >>= 1;
    } else {
      s = g.fixed_s;
    }
    const int64_t in_e =
        (((((int64_t)tau * g.dims[0] + idx[0]) * g.dims[1] + idx[1]) * g.dims[2] + idx[2]) *
             g.dims[3] + idx[3]);
    const float2 v = g.in[in_e], vl = g.in[g.lo_off + in_e];
    float f;
    if (g.kind == 0) f = (tau == s) ? 1.f : 0.f;
    else f = (s & tau) ? -1.f : 1.f;
    g.out[e] = make_float2(f * v.x, f * v.y);
    g.out[g.lo_off + e] = make_float2(f * vl.x, f * vl.y);
  }
}

__global__ void k_cz(const CzEntry *__restrict__ entries) {
  cz_apply(entries[blockIdx.y], (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
           (int64_t)gridDim.x * blockDim.x);
}

// General two-qubit gate, one half (see Gate2Entry): each thread writes one
// output entry, mixing the two sigma slices of its input position with
// W_s[tau][.] in float-float complex arithmetic.
__device__ __forceinline__ void gate2_apply(const Gate2Entry &g, int64_t e0, int64_t de) {
  int od[4] = {g.dims[0], g.dims[1], g.dims[2], g.dims[3]};
  od[g.axis] *= g.chi;
  const int64_t half_in = (int64_t)g.dims[0] * g.dims[1] * g.dims[2] * g.dims[3];
  const int64_t half_out = (int64_t)od[0] * od[1] * od[2] * od[3];
  for (int64_t e = e0; e < 2 * half_out; e += de) {
    int64_t rem = e;
    int idx[4];
    idx[3] = (int)(rem % od[3]); rem /= od[3];
    idx[2] = (int)(rem % od[2]); rem /= od[2];
    idx[1] = (int)(rem % od[1]); rem /= od[1];
    idx[0] = (int)(rem % od[0]); rem /= od[0];
    const int tau = (int)rem;
    const int s = idx[g.axis] % g.chi;
    idx[g.axis] /= g.chi;
    const int64_t in_e =
        ((((int64_t)idx[0]) * g.dims[1] + idx[1]) * g.dims[2] + idx[2]) * g.dims[3] + idx[3];
    ff re = {0.f, 0.f}, im = {0.f, 0.f};
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int64_t p = (int64_t)sg * half_in + in_e;
      const float2 h = g.in[p], l = g.in[g.lo_off + p];
      const float2 wh = g.W_hi[s][2 * tau + sg], wl = g.W_lo[s][2 * tau + sg];
      ff r, i;
      cmul_ff({wh.x, wl.x}, {wh.y, wl.y}, {h.x, l.x}, {h.y, l.y}, r, i);
      re = ff_add(re, r);
      im = ff_add(im, i);
    }
    g.out[e] = make_float2(re.hi, im.hi);
    g.out[g.lo_off + e] = make_float2(re.lo, im.lo);
  }
}

__global__ void k_gate2(const Gate2Entry *__restrict__ entries) {
  gate2_apply(entries[blockIdx.y], (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
              (int64_t)gridDim.x * blockDim.x);
}

// The whole evolution in one launch, one block per site (small site tensors):
// a site's tensor evolves through its own gate halves only (a single-qubit
// gate, or one side of a CZ or general gate split), so every block applies
// its site's list in circuit order with a barrier between gates, starting
// from |0> (A^0 = 1, A^1 = 0) in its first buffer.  Block 0 also writes the
// status block's unit scalars.
__global__ void __launch_bounds__(256) k_evolve_sites(
    const Gate1Entry *__restrict__ g1, const CzEntry *__restrict__ cz,
    const Gate2Entry *__restrict__ g2, const EvoRef *__restrict__ refs,
    const int32_t *__restrict__ first, float2 *const *bufs, const int64_t *lo_off,
    DeviceStatus *st) {
  const int q = blockIdx.x;
  if (threadIdx.x == 0) {
    float2 *a = bufs[q];
    a[0] = make_float2(1.f, 0.f);
    a[1] = make_float2(0.f, 0.f);
    a[lo_off[q]] = make_float2(0.f, 0.f);
    a[lo_off[q] + 1] = make_float2(0.f, 0.f);
    if (q == 0) {
      st->error = 0;
      st->error_info = 0;
      st->timeout = 0;
      st->unit_f32 = make_float2(1.f, 0.f);
      st->unit_h16[0] = pack_bf16(1.f, 0.f);
      st->unit_h16[1] = 0u;
      st->unit_f16[0] = pack_f16(1.f, 0.f);
      st->unit_f16[1] = 0u;
    }
  }
  __syncthreads();
  for (int i = first[q]; i < first[q + 1]; ++i) {
    const EvoRef r = refs[i];
    if (r.kind == 0) gate1_apply(g1[r.idx], threadIdx.x, blockDim.x);
    else if (r.kind == 1) cz_apply(cz[r.idx], threadIdx.x, blockDim.x);
    else gate2_apply(g2[r.idx], threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

static int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_init_sites(float2 *const *bufs, const int64_t *lo_off, int n_sites,
                              DeviceStatus *st, cudaStream_t s) {
  int threads = 128;
  int blocks = (n_sites + threads - 1) / threads;
  if (blocks < 1) blocks = 1;
  k_init_sites<<<blocks, threads, 0, s>>>(bufs, lo_off, n_sites, st);
  return cudaGetLastError();
}

cudaError_t launch_evolve_sites(const Gate1Entry *g1, const CzEntry *cz, const Gate2Entry *g2,
                               const EvoRef *refs, const int32_t *first, float2 *const *bufs,
                               const int64_t *lo_off, int n_sites, DeviceStatus *st,
                               cudaStream_t s) {
  if (n_sites <= 0) return cudaSuccess;
  k_evolve_sites<<<n_sites, 256, 0, s>>>(g1, cz, g2, refs, first, bufs, lo_off, st);
  return cudaGetLastError();
}

cudaError_t launch_gate1(const Gate1Entry *d_entries, int n, int64_t max_half, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(grid_for(max_half, 256), n);
  k_gate1<<<grid, 256, 0, s>>>(d_entries);
  return cudaGetLastError();
}

cudaError_t launch_cz(const CzEntry *d_entries, int n, int64_t max_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(grid_for(max_out, 256), n);
  k_cz<<<grid, 256, 0, s>>>(d_entries);
  return cudaGetLastError();
}

cudaError_t launch_gate2(const Gate2Entry *d_entries, int n, int64_t max_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(grid_for(max_out, 256), n);
  k_gate2<<<grid, 256, 0, s>>>(d_entries);
  return cudaGetLastError();
}

}  // namespace peps
