// K6: final reduction.  After the last column the running tensor of a lane is
// a single complex number stored as m * 2^S (S = cumulative scale exponent of
// the lane's chain); the amplitude contribution is m * 2^-S in FP64, summed
// over slices in a fixed order (the "cut" technique named in the paper's
// conclusions: the amplitude is the sum of the sliced contractions).
#include "common.h"
#include "format.cuh"

namespace peps {

template <int FMT>
__global__ void k_finalize(const FinalEntry *__restrict__ entries, int n, int64_t plane,
                           const Rec *__restrict__ recs, double2 *acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const FinalEntry f = entries[i];
  const float2 m = load_g<FMT>(f.G, 0, plane);
  const int S = recs[f.rec].exp;
  double2 a = acc[f.out_index];
  a.x += ldexp((double)m.x, -S);
  a.y += ldexp((double)m.y, -S);
  acc[f.out_index] = a;
}

cudaError_t launch_finalize(const FinalEntry *d_entries, int n, int fmt, int64_t plane,
                            const Rec *d_recs, double2 *d_acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 128, blocks = (n + threads - 1) / threads;
  switch (fmt) {
    case FMT_F32: k_finalize<FMT_F32><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    case FMT_TF32: k_finalize<FMT_TF32><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    case FMT_BF16: k_finalize<FMT_BF16><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    case FMT_FP16: k_finalize<FMT_FP16><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    case FMT_BF16X2: k_finalize<FMT_BF16X2><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    case FMT_FP16X2: k_finalize<FMT_FP16X2><<<blocks, threads, 0, s>>>(d_entries, n, plane, d_recs, d_acc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Square partition, last contraction: sum_i Y[i] F[i] for each entry.  Pass
// 1: block b of entry e sums a fixed slice of the products into
// partials[e][b]; pass 2 adds the entry's nslots partials in order, applies
// 2^-(S_Y + S_F) and accumulates into the amplitude.  Where the merge that
// makes Y runs on the tensor cores, its epilogue writes the partials itself
// (Y is never stored) and only pass 2 runs.  Both passes have a fixed order, so
// repeated calls give identical results.  A thread sums its terms (n / 65536
// of them, 256 at 6x6 (1+32+1)) in FP32 on two chains; the sums across
// threads and blocks are FP64.  With terms of random phase the FP32 part
// adds about sqrt(terms per thread) 2^-24 of a partial, some 1e-6 of the
// amplitude, and keeps the kernel at the memory rate (GB300's FP64 rate is
// far below its FP32 rate).
template <int FMT>
__global__ void __launch_bounds__(256) k_dot(const DotEntry *__restrict__ entries, int64_t plane,
                                             double2 *partials) {
  const DotEntry d = entries[blockIdx.y];
  float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + stride < d.n; i += 2 * stride) {
    const float2 y0 = load_g<FMT>(d.Y, i, plane), f0 = load_g<FMT>(d.F, i, plane);
    const float2 y1 = load_g<FMT>(d.Y, i + stride, plane), f1 = load_g<FMT>(d.F, i + stride, plane);
    re0 = fmaf(y0.x, f0.x, fmaf(-y0.y, f0.y, re0));
    im0 = fmaf(y0.x, f0.y, fmaf(y0.y, f0.x, im0));
    re1 = fmaf(y1.x, f1.x, fmaf(-y1.y, f1.y, re1));
    im1 = fmaf(y1.x, f1.y, fmaf(y1.y, f1.x, im1));
  }
  if (i < d.n) {
    const float2 y0 = load_g<FMT>(d.Y, i, plane), f0 = load_g<FMT>(d.F, i, plane);
    re0 = fmaf(y0.x, f0.x, fmaf(-y0.y, f0.y, re0));
    im0 = fmaf(y0.x, f0.y, fmaf(y0.y, f0.x, im0));
  }
  __shared__ double sre[256], sim[256];
  sre[threadIdx.x] = (double)re0 + (double)re1;
  sim[threadIdx.x] = (double)im0 + (double)im1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sre[threadIdx.x] += sre[threadIdx.x + w];
      sim[threadIdx.x] += sim[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(sre[0], sim[0]);
}

// One block per entry: thread t adds slots t, t + 128, ... in order, then a
// fixed tree over the threads (the same order on every call).
__global__ void __launch_bounds__(128) k_dot_final(const DotEntry *__restrict__ entries,
                                                   const Rec *__restrict__ recs,
                                                   const double2 *__restrict__ partials,
                                                   double2 *acc) {
  const int e = blockIdx.x;
  const DotEntry d = entries[e];
  const int ns = d.nslots;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < ns; b += blockDim.x) {
    re += partials[(int64_t)e * ns + b].x;
    im += partials[(int64_t)e * ns + b].y;
  }
  __shared__ double sre[128], sim[128];
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sre[threadIdx.x] += sre[threadIdx.x + w];
      sim[threadIdx.x] += sim[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int S = recs[d.rec_y].exp + recs[d.rec_f].exp;
    double2 a = acc[d.out_index];
    a.x += ldexp(sre[0], -S);
    a.y += ldexp(sim[0], -S);
    acc[d.out_index] = a;
  }
}

cudaError_t launch_dot(const DotEntry *d_entries, int n, int fmt, int64_t plane,
                       const Rec *d_recs, double2 *d_partials, double2 *d_acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(kDotBlocks, n);
  switch (fmt) {
    case FMT_F32: k_dot<FMT_F32><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    case FMT_TF32: k_dot<FMT_TF32><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    case FMT_BF16: k_dot<FMT_BF16><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    case FMT_FP16: k_dot<FMT_FP16><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    case FMT_BF16X2: k_dot<FMT_BF16X2><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    case FMT_FP16X2: k_dot<FMT_FP16X2><<<grid, 256, 0, s>>>(d_entries, plane, d_partials); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dot_final<<<n, 128, 0, s>>>(d_entries, d_recs, d_partials, d_acc);
  return cudaGetLastError();
}

cudaError_t launch_dot_final(const DotEntry *d_entries, int n, const Rec *d_recs,
                             const double2 *d_partials, double2 *d_acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_dot_final<<<n, 128, 0, s>>>(d_entries, d_recs, d_partials, d_acc);
  return cudaGetLastError();
}

__global__ void k_store_out(const double2 *__restrict__ acc, peps_c128 *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    out[i].re = acc[i].x;
    out[i].im = acc[i].y;
  }
}

cudaError_t launch_store_out(const double2 *d_acc, peps_c128 *d_out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  k_store_out<<<(unsigned)blocks, threads, 0, s>>>(d_acc, d_out, n);
  return cudaGetLastError();
}

// Prefix reuse is only valid if every group of `group` consecutive
// bitstrings agrees on the prefix qubits (mask); a violation sets an error.
__global__ void k_check_groups(const uint64_t *__restrict__ bits, int64_t n, int group,
                               uint64_t mask, DeviceStatus *st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g0 = (i / group) * group;
  if ((bits[i] & mask) != (bits[g0] & mask)) {
    atomicExch(&st->error, 1);
    atomicExch(&st->error_info, (int)i);
  }
}

cudaError_t launch_check_groups(const uint64_t *d_bits, int64_t n, int group, uint64_t mask,
                                DeviceStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  k_check_groups<<<(unsigned)blocks, threads, 0, s>>>(d_bits, n, group, mask, st);
  return cudaGetLastError();
}

}  // namespace peps
