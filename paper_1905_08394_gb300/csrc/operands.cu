// K3: projection on the output bit and operand build.
//
// For every site q and bit tau (and, when edges are sliced, every setting of
// the sliced Schmidt bits on the site's legs) this writes the projected tensor
// E = A_q^{tau} (paper, main-text "overlap" equation) as the B operand of the
// site's absorption step:
//   Ec[k][n] = E[l][r][u][d],  k = l*du + u  (contracted: h_r, v),
//                              n = r*dd + d  (new legs: h'_r, v').
// A sliced leg is restricted to the indices whose fixed bits have the slice's
// values (cutting the bond), which is the same as applying the sliced CZ as
// its single Schmidt term.  Only two operands exist per site and slice, so the
// cost does not depend on the number of bitstrings.
#include "common.h"
#include "format.cuh"

namespace peps {

__device__ __forceinline__ int deposit_bits(uint32_t v, uint32_t mask) {
  uint32_t out = 0;
  for (int b = 0; b < 32 && v; ++b) {
    if (mask & (1u << b)) {
      out |= (v & 1u) << b;
      v >>= 1;
    }
  }
  return (int)out;
}

__device__ __forceinline__ float2 fetch_E(const OpBuildEntry &g, int k, int n) {
  const int rl = g.rdims[0], rr = g.rdims[1], ru = g.rdims[2], rd = g.rdims[3];
  (void)rl; (void)rr;
  const int l_ = k / ru, u_ = k % ru;
  const int r_ = n / rd, d_ = n % rd;
  const int l = (int)g.fixed_val[0] | deposit_bits(l_, g.free_mask[0]);
  const int r = (int)g.fixed_val[1] | deposit_bits(r_, g.free_mask[1]);
  const int u = (int)g.fixed_val[2] | deposit_bits(u_, g.free_mask[2]);
  const int d = (int)g.fixed_val[3] | deposit_bits(d_, g.free_mask[3]);
  const int64_t e =
      ((((int64_t)g.tau * g.dims[0] + l) * g.dims[1] + r) * g.dims[2] + u) * g.dims[3] + d;
  const float2 h = g.A[e], lo = g.A[g.lo_off + e];
  return make_float2(h.x + lo.x, h.y + lo.y);  // float-float -> one FP32 rounding
}

// One block row per entry; threads cover Ec's K*N entries.
__global__ void k_build_ec(const OpBuildEntry *__restrict__ entries, OpDesc *ops) {
  const OpBuildEntry &g = entries[blockIdx.y];
  OpDesc &op = ops[g.op];
  const int K = g.rdims[0] * g.rdims[2];
  const int N = g.rdims[1] * g.rdims[3];
  float2 *Ec = const_cast<float2 *>(op.Ec);
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // bounds are re-accumulated by k_beta
    op.beta_c_bits = 0u;
    op.beta_t_bits = 0u;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * N; i += gridDim.x * blockDim.x) {
    const int k = i / N, n = i % N;
    Ec[i] = fetch_E(g, k, n);
  }
}

// beta = max_n sum_k (|Re E_kn| + |Im E_kn|): the factor by which one
// absorption can grow max(|Re|, |Im|) of the running tensor.
__global__ void k_beta(const OpBuildEntry *__restrict__ entries, OpDesc *ops) {
  const OpBuildEntry &g = entries[blockIdx.y];
  OpDesc &op = ops[g.op];
  const int K = g.rdims[0] * g.rdims[2];
  const int N = g.rdims[1] * g.rdims[3];
  float best = 0.f;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < K; ++k) {
      float2 v = op.Ec[(int64_t)k * N + n];
      s += fabsf(v.x) + fabsf(v.y);
    }
    best = fmaxf(best, s);
  }
  // Round the bound up slightly so that fp32 summation order cannot make it
  // smaller than the exact sum.
  best *= 1.0f + 1.0f / 256.0f;
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&op.beta_c_bits, __float_as_uint(best));
}

cudaError_t launch_build_operands(const OpBuildEntry *d_entries, int n, int max_kn,
                                  OpDesc *d_ops, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (max_kn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_build_ec<<<dim3(blocks, n), 256, 0, s>>>(d_entries, d_ops);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_beta<<<dim3(4, n), 256, 0, s>>>(d_entries, d_ops);
  return cudaGetLastError();
}

}  // namespace peps
