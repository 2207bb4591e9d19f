// K4 (CUDA-core form): one site absorption of the column sweep for a batch
// of lanes,
//   G'[rest, h'_r, v'] = sum_{h_r, v} G[rest, h_r, v] * E[h_r, v, h'_r, v']
// (supplementary "exact computation of the overlap", the absorption of one
// tensor into the running tensor, transposed to sweep columns).  As a matrix
// product: out[M x N] = G[M x K] * Ec[K x N] in complex FP32, with
//   M = product of the untouched h legs (slowest leg P first),
//   K = dim(h_r) * dim(v), N = dim(h'_r) * dim(v').
// The store is permute-fused: row m = m_hi * (M / P) + m_lo, column
// n = h' * dv' + v' goes to ((m_lo * dh' + h') * P + m_hi) * dv' + v', which
// moves the slowest untouched leg next to v' so that the next step's
// contracted legs are again the two fastest.
//
// Every output is multiplied by the step's power-of-two scale 2^x (exact), and
// the block's max |stored entry| goes to the lane's record for the next step.
#include "common.h"
#include "format.cuh"

namespace peps {

namespace {

constexpr int BM = 128;  // rows of G per block
constexpr int BN = 64;   // complex columns per block
constexpr int BK = 8;    // complex k per smem stage
constexpr int TM = 8;    // rows per thread (strided by 16)
constexpr int TN = 4;    // columns per thread (strided by 16)
constexpr int THREADS = 256;

template <int FMT>
__global__ void __launch_bounds__(THREADS, 2)
k_contract_simt(const StepShape sh, const StepItem *__restrict__ items,
                const OpDesc *__restrict__ ops, Rec *__restrict__ recs) {
  __shared__ float2 As[2][BK][BM];
  __shared__ float2 Bs[2][BK][BN];

  const StepItem it = items[blockIdx.z];
  const uint64_t bits = *it.bits;
  const OpDesc &op = ops[it.op_base + block_variant(bits, sh)];
  const float2 *__restrict__ Ec = op.Ec;
  const int64_t M = sh.M;
  const int K = sh.K, N = sh.N;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const bool unit_in = it.in_rec < 0;

  float2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);

  // A tile loader: thread -> row (tid >> 1), k chunk (tid & 1) * 4 .. +4.
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;
  // B tile loader: thread -> k (tid >> 5), n pair (tid & 31) * 2.
  const int b_k = tid >> 5, b_n = (tid & 31) * 2;

  auto load_tile = [&](int buf, int k0) {
    const int64_t m = m0 + a_row;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = k0 + a_k + c;
      float2 v = make_float2(0.f, 0.f);
      if (m < M && k < K) {
        if (unit_in) v = (m == 0 && k == 0) ? make_float2(1.f, 0.f) : v;
        else v = load_g<FMT>(it.A, m * K + k, sh.plane);
      }
      As[buf][a_k + c][a_row] = v;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int k = k0 + b_k, n = n0 + b_n + c;
      Bs[buf][b_k][b_n + c] = (k < K && n < N) ? Ec[(int64_t)k * N + n] : make_float2(0.f, 0.f);
    }
  };

  const int nk = (K + BK - 1) / BK;
  load_tile(0, 0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int cur = t & 1;
    if (t + 1 < nk) load_tile(cur ^ 1, (t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[cur][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[cur][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }

  // Epilogue: scale, permuted store, max.
  const float mu = unit_in ? 1.f : __uint_as_float(recs[it.in_rec].maxbits);
  const int s_in = unit_in ? 0 : recs[it.in_rec].exp;
  const float beta = __uint_as_float(op.beta_c_bits);
  const int x = step_scale_exp(mu, beta, sh.target);
  const float sc = pow2f(x);
  const int64_t Mr = sh.Mr > 0 ? sh.Mr : M;
  const bool batched = Mr != M;
  const int64_t Mlo = Mr / sh.P;
  const int dv = sh.dv_out, dh = sh.dh_out;
  float vmax = 0.f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t m = m0 + ty + 16 * i;
    if (m >= M) continue;
    const int64_t b = batched ? m / Mr : 0, mr = m - b * Mr;
    const int64_t m_hi = mr / Mlo, m_lo = mr - m_hi * Mlo;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      const int hh = sh.nvs ? n % dh : n / dv, vv = sh.nvs ? n / dh : n % dv;
      const int64_t rot = (m_lo * dh + hh) * sh.P + m_hi;
      const int64_t dest = sh.vb ? (b * dv + vv) * (Mr * dh) + rot
                                 : b * (Mr * N) + rot * dv + vv;
      const float2 v = make_float2(acc[i][j].x * sc, acc[i][j].y * sc);
      store_g<FMT>(it.D, dest, sh.plane, v);
      vmax = fmaxf(vmax, max_abs2(v));
    }
  }
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((tid & 31) == 0) atomicMax(&recs[it.out_rec].maxbits, __float_as_uint(vmax));
  if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) recs[it.out_rec].exp = s_in + x + op.e_c;
}

// The same step for a running tensor of at most a few rows (the first steps
// of a sweep, M = 1 .. 8): one thread per output entry, no tiling.
template <int FMT>
__global__ void __launch_bounds__(256)
k_contract_rows(const StepShape sh, const StepItem *__restrict__ items,
                const OpDesc *__restrict__ ops, Rec *__restrict__ recs) {
  const StepItem it = items[blockIdx.y];
  const uint64_t bits = *it.bits;
  const OpDesc &op = ops[it.op_base + block_variant(bits, sh)];
  const int M = (int)sh.M, K = sh.K, N = sh.N;
  const bool unit_in = it.in_rec < 0;
  const float mu = unit_in ? 1.f : __uint_as_float(recs[it.in_rec].maxbits);
  const int s_in = unit_in ? 0 : recs[it.in_rec].exp;
  const int x = step_scale_exp(mu, __uint_as_float(op.beta_c_bits), sh.target);
  const float sc = pow2f(x);
  const int64_t Mr = sh.Mr > 0 ? sh.Mr : sh.M;
  const bool batched = Mr != sh.M;
  const int64_t Mlo = Mr / sh.P;
  const int dv = sh.dv_out, dh = sh.dh_out;
  float vmax = 0.f;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < M * N) {
    const int m = e / N, n = e - m * N;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < K; ++k) {
      float2 a;
      if (unit_in) a = (m == 0 && k == 0) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
      else a = load_g<FMT>(it.A, (int64_t)m * K + k, sh.plane);
      const float2 w = op.Ec[(int64_t)k * N + n];
      re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
      im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
    }
    const int64_t b = batched ? m / Mr : 0, mr = m - b * Mr;
    const int64_t m_hi = mr / Mlo, m_lo = mr - m_hi * Mlo;
    const int hh = sh.nvs ? n % dh : n / dv, vv = sh.nvs ? n / dh : n % dv;
    const int64_t rot = (m_lo * dh + hh) * sh.P + m_hi;
    const int64_t dest = sh.vb ? (b * dv + vv) * (Mr * dh) + rot : b * (Mr * N) + rot * dv + vv;
    const float2 v = make_float2(re * sc, im * sc);
    store_g<FMT>(it.D, dest, sh.plane, v);
    vmax = max_abs2(v);
  }
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&recs[it.out_rec].maxbits, __float_as_uint(vmax));
  if (blockIdx.x == 0 && threadIdx.x == 0) recs[it.out_rec].exp = s_in + x + op.e_c;
}

}  // namespace

cudaError_t launch_contract_simt(const StepShape &sh, const StepItem *d_items, int n_items,
                                 const OpDesc *d_ops, Rec *d_recs, const DeviceStatus *st,
                                 cudaStream_t s) {
  (void)st;
  if (n_items <= 0) return cudaSuccess;
  if (sh.M <= 8 && n_items <= 65535) {
    const int64_t blocks = (sh.M * sh.N + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)blocks, n_items);
    switch (sh.fmt) {
      case FMT_F32: k_contract_rows<FMT_F32><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      case FMT_TF32: k_contract_rows<FMT_TF32><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      case FMT_BF16: k_contract_rows<FMT_BF16><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      case FMT_FP16: k_contract_rows<FMT_FP16><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      case FMT_BF16X2: k_contract_rows<FMT_BF16X2><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      case FMT_FP16X2: k_contract_rows<FMT_FP16X2><<<grid, 256, 0, s>>>(sh, d_items, d_ops, d_recs); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const int64_t mt = (sh.M + BM - 1) / BM;
  const int nt = (sh.N + BN - 1) / BN;
  if (mt > 0x7fffffffLL || nt > 65535 || n_items > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)mt, nt, n_items);
  switch (sh.fmt) {
    case FMT_F32: k_contract_simt<FMT_F32><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    case FMT_TF32: k_contract_simt<FMT_TF32><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    case FMT_BF16: k_contract_simt<FMT_BF16><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    case FMT_FP16: k_contract_simt<FMT_FP16><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    case FMT_BF16X2: k_contract_simt<FMT_BF16X2><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    case FMT_FP16X2: k_contract_simt<FMT_FP16X2><<<grid, THREADS, 0, s>>>(sh, d_items, d_ops, d_recs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace peps
