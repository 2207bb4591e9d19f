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
