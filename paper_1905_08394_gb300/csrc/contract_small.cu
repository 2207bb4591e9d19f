// K4 + K5 + K6 for small lattices in one persistent launch: every column
// absorption of one bitstring's sweep (supplementary "exact computation of
// the overlap", the generic scheme transposed to columns) runs inside one
// block, with the running tensor held in shared memory from the scalar 1 to
// the final 1 x 1 tensor.  Blocks walk the bitstrings (block b takes
// b, b + gridDim.x, ...), so a call is one launch whatever the number of
// bitstrings and steps.
//
// Step s: out[M x N] = in[M x K] * Ec[K x N] in complex FP32 with the same
// permute-fused store as the step-by-step kernels (row m = m_hi (M / P) +
// m_lo, column n = h' dv' + v' goes to ((m_lo dh' + h') P + m_hi) dv' + v'),
// and the same power-of-two renormalisation: the output is multiplied by 2^x
// with x from the input's max |entry| and the operand's column bound, so that
// it stays at most 1; the exponents add up exactly and the amplitude is
// m 2^-S in FP64, added to the call's accumulator (a sum over slices when the
// call has several).
#include "common.h"
#include "format.cuh"

namespace peps {

namespace {

constexpr int SW_THREADS = 256;

__global__ void __launch_bounds__(SW_THREADS) k_sweep_small(const SmallSweep p) {
  extern __shared__ float2 sm[];
  float2 *const buf0 = sm;
  float2 *const buf1 = sm + p.cap_g;
  float2 *const E = sm + 2 * p.cap_g;
  __shared__ float red[SW_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t i = blockIdx.x; i < p.n; i += gridDim.x) {
    const uint64_t bits = p.bits[i];
    float2 *in = buf0, *out = buf1;
    if (tid == 0) in[0] = make_float2(1.f, 0.f);
    float mu = 1.f;   // max |entry| of the stored input
    int S = 0;        // stored G = true G * 2^S
    for (int s = 0; s < p.n_steps; ++s) {
      const StepShape &sh = p.steps[s];
      const OpDesc &op = p.ops[p.op_base[s] + block_variant(bits, sh)];
      const int M = (int)sh.M, K = sh.K, N = sh.N;
      const float2 *__restrict__ Ec = op.Ec;
      for (int e = tid; e < K * N; e += SW_THREADS) E[e] = Ec[e];
      const int x = step_scale_exp(mu, __uint_as_float(op.beta_c_bits), 0);
      const float sc = pow2f(x);
      __syncthreads();   // E loaded; the previous step's output complete
      const int P = (int)sh.P, Mlo = M / P, dv = sh.dv_out, dh = sh.dh_out;
      float vmax = 0.f;
      for (int e = tid; e < M * N; e += SW_THREADS) {
        const int m = e / N, n = e - m * N;
        const float2 *a = in + (int64_t)m * K;
        float re = 0.f, im = 0.f;
        for (int k = 0; k < K; ++k) {
          const float2 u = a[k], w = E[k * N + n];
          re = fmaf(u.x, w.x, re);
          re = fmaf(-u.y, w.y, re);
          im = fmaf(u.x, w.y, im);
          im = fmaf(u.y, w.x, im);
        }
        re *= sc;
        im *= sc;
        const int m_hi = m / Mlo, m_lo = m - m_hi * Mlo;
        const int hh = n / dv, vv = n - hh * dv;
        out[((m_lo * dh + hh) * P + m_hi) * dv + vv] = make_float2(re, im);
        vmax = fmaxf(vmax, fmaxf(fabsf(re), fabsf(im)));
      }
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0) red[warp] = vmax;
      __syncthreads();   // output and partial maxima complete; E free
      vmax = red[0];
#pragma unroll
      for (int w = 1; w < SW_THREADS / 32; ++w) vmax = fmaxf(vmax, red[w]);
      mu = vmax;
      S += x;
      float2 *t = in;
      in = out;
      out = t;
    }
    if (tid == 0) {
      const float2 g = in[0];
      double2 a = p.acc[i];
      a.x += ldexp((double)g.x, -S);
      a.y += ldexp((double)g.y, -S);
      p.acc[i] = a;
    }
    __syncthreads();   // red and the buffers are reused by the next bitstring
  }
}

}  // namespace

size_t small_sweep_smem(int cap_g, int cap_e) {
  return (size_t)(2 * cap_g + cap_e) * sizeof(float2);
}

cudaError_t launch_sweep_small(const SmallSweep &p, int sm_count, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  const size_t smem = small_sweep_smem(p.cap_g, p.cap_e);
  static int configured = 0;   // dynamic shared memory above 48 KiB needs the opt-in
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_small,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmallSweepMaxSmem);
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  if (smem > kSmallSweepMaxSmem) return cudaErrorInvalidValue;
  // blocks resident per SM (about 220 KiB of shared memory), at most 4
  const int per_sm = (int)((220u * 1024u) / (smem > 0 ? smem : 1));
  int64_t blocks = (int64_t)sm_count * (per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm));
  if (blocks > p.n) blocks = p.n;
  k_sweep_small<<<(unsigned)blocks, SW_THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace peps
