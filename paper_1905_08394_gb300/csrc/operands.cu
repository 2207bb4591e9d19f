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

// Spread the bits of v over the set bits of mask (low to high).  An all-ones
// mask means a leg with nothing fixed: the index itself (legs whose
// dimension is not a power of two, from general two-qubit gates, always
// take this path since they cannot be sliced).
__device__ __forceinline__ int deposit_bits(uint32_t v, uint32_t mask) {
  if (mask == 0xFFFFFFFFu) return (int)v;
  uint32_t out = 0;
  for (int b = 0; b < 32 && v; ++b) {
    if (mask & (1u << b)) {
      out |= (v & 1u) << b;
      v >>= 1;
    }
  }
  return (int)out;
}

// Full index of restricted value v of a role's leg: the free bits take v's
// bits, the fixed bits their values, and each linked bit the value of its
// source bit XOR the flip held in fixed_val.
__device__ __forceinline__ int expand_leg(const OpBuildEntry &g, int role, int v) {
  int full = (int)g.fixed_val[role] | deposit_bits(v, g.free_mask[role]);
  for (int i = 0; i < g.n_links[role]; ++i)
    full ^= ((full >> g.link_src[role][i]) & 1) << g.link_dst[role][i];
  return full;
}

// Element position of E[l][r][u][d] (legs by role; restricted indices mapped
// back to full ones, then through each role's physical stride).
__device__ __forceinline__ int64_t pos_E(const OpBuildEntry &g, int l_, int r_, int u_, int d_) {
  const int l = expand_leg(g, 0, l_);
  const int r = expand_leg(g, 1, r_);
  const int u = expand_leg(g, 2, u_);
  const int d = expand_leg(g, 3, d_);
  return (int64_t)g.tau * g.tau_stride + l * g.stride[0] + r * g.stride[1] + u * g.stride[2] +
         d * g.stride[3];
}

__device__ __forceinline__ float2 fetch_E(const OpBuildEntry &g, int k, int n) {
  const int ru = g.rdims[2], rr = g.rdims[1], rd = g.rdims[3];
  const int r_ = g.nvs ? n % rr : n / rd, d_ = g.nvs ? n / rr : n % rd;
  const int64_t e = pos_E(g, k / ru, r_, k % ru, d_);
  const float2 h = g.A[e], lo = g.A[g.lo_off + e];
  return make_float2(h.x + lo.x, h.y + lo.y);  // float-float -> one FP32 rounding
}

// Double-layer entry (marginals): sum over the allowed sigma of
// A^sigma[l,r,u,d] conj(A^sigma[l',r',u',d']) with every role index doubled
// as ket * dim + bra (no slicing: the full index is the role index).
__device__ __forceinline__ float2 fetch_E_dl(const OpBuildEntry &g, int k, int n) {
  const int Ru = g.rdims[2], Rr = g.rdims[1], Rd = g.rdims[3];
  const int ldl = k / Ru, udl = k % Ru;
  const int rdl = g.nvs ? n % Rr : n / Rd, ddl = g.nvs ? n / Rr : n % Rd;
  const int l0 = ldl / g.dims[0], l1 = ldl % g.dims[0];
  const int r0 = rdl / g.dims[1], r1 = rdl % g.dims[1];
  const int u0 = udl / g.dims[2], u1 = udl % g.dims[2];
  const int d0 = ddl / g.dims[3], d1 = ddl % g.dims[3];
  float re = 0.f, im = 0.f;
  for (int sg = 0; sg < 2; ++sg) {
    if (g.dl == 1 && sg != g.tau) continue;
    const int64_t base = (int64_t)sg * g.tau_stride;
    const int64_t ek = base + l0 * g.stride[0] + r0 * g.stride[1] + u0 * g.stride[2] + d0 * g.stride[3];
    const int64_t eb = base + l1 * g.stride[0] + r1 * g.stride[1] + u1 * g.stride[2] + d1 * g.stride[3];
    const float2 ah = g.A[ek], al = g.A[g.lo_off + ek], bh = g.A[eb], bl = g.A[g.lo_off + eb];
    const float ar = ah.x + al.x, ai = ah.y + al.y, br = bh.x + bl.x, bi = bh.y + bl.y;
    re += ar * br + ai * bi;      // a * conj(b)
    im += ai * br - ar * bi;
  }
  return make_float2(re, im);
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
    Ec[i] = g.dl ? fetch_E_dl(g, k, n) : fetch_E(g, k, n);
  }
}

// legs of a two-site block operand whose element offsets are tabulated in
// shared memory (longer legs compute them per entry)
constexpr int kMaxLeg2 = 256;

// Two-site block operand W (see OpBuild2Entry), summed over the internal
// vertical bond from the float-float site tensors and rounded once to FP32.
// k = (l_a * Lb + l_b) * Ua + u_a, n = (r_a * Rb + r_b) * Db + d_b.
//
// The sum is compensated: each product of the hi parts is split exactly
// into p + e (an FMA gives e), the p's are added with an error-free
// two-sum, and the errors e, the sums' rounding errors and the cross terms
// hi*lo + lo*hi (lo*lo, 2^-48 relative, is dropped as in a float-float
// product) collect in a second FP32 accumulator; W = main + correction,
// rounded once.  Its error is the final rounding plus O(2^-48) of the sum of
// |terms|, as with float-float arithmetic throughout.
__device__ __forceinline__ void acc_prod(float x, float y, float &s, float &c) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  const float t = s + p;
  const float bb = t - s;
  c += ((s - (t - bb)) + (p - bb)) + e;
  s = t;
}

// The sum is the product of two matrices, A'[(l_a, u_a, r_a), m] and
// B'[m, (l_b, r_b, d_b)], whose entries land at W[k, n] with k, n as above.
// A block takes 32 x 32 tiles of that product: the tile's rows of A' and
// columns of B' pass through shared memory 16 values of m at a time, and each
// thread accumulates four entries (one column, four rows).
constexpr int kEc2T = 32;   // tile rows and columns
constexpr int kEc2M = 16;   // m per shared-memory pass

__global__ void __launch_bounds__(256) k_build_ec2(const OpBuild2Entry *__restrict__ entries,
                                                   OpDesc *ops) {
  const OpBuild2Entry &g = entries[blockIdx.y];
  OpDesc &op = ops[g.op];
  const int La = g.a.rdims[0], Ra = g.a.rdims[1], Ua = g.a.rdims[2], Mid = g.a.rdims[3];
  const int Lb = g.b.rdims[0], Rb = g.b.rdims[1], Db = g.b.rdims[3];
  const int N = Ra * Rb * Db;
  const int Rows = La * Ua * Ra, Cols = Lb * Rb * Db;
  const int tiles_c = (Cols + kEc2T - 1) / kEc2T;
  const int n_tiles = ((Rows + kEc2T - 1) / kEc2T) * tiles_c;
  if ((int)blockIdx.x >= n_tiles) return;
  // full index of every restricted value of the shared bond, on both sites,
  // and (where the legs are short enough) element offsets of the other legs
  __shared__ int mid_a[kMaxMid], mid_b[kMaxMid];
  __shared__ int64_t off_la[kMaxLeg2], off_ra[kMaxLeg2], off_ua[kMaxLeg2];
  __shared__ int64_t off_lb[kMaxLeg2], off_rb[kMaxLeg2], off_db[kMaxLeg2];
  __shared__ float4 As[kEc2T][kEc2M + 1];   // (hi re, hi im, lo re, lo im), padded rows
  __shared__ float4 Bs[kEc2M][kEc2T];
  __shared__ int64_t row_a[kEc2T], col_b[kEc2T], row_out[kEc2T], col_out[kEc2T];
  for (int m = threadIdx.x; m < Mid; m += blockDim.x) {
    mid_a[m] = expand_leg(g.a, 3, m);
    mid_b[m] = expand_leg(g.b, 2, m);
  }
  const bool tab = La <= kMaxLeg2 && Ra <= kMaxLeg2 && Ua <= kMaxLeg2 && Lb <= kMaxLeg2 &&
                   Rb <= kMaxLeg2 && Db <= kMaxLeg2;
  if (tab) {
    auto fill = [&](int64_t *t, const OpBuildEntry &e, int role, int n) {
      for (int v = threadIdx.x; v < n; v += blockDim.x)
        t[v] = (int64_t)expand_leg(e, role, v) * e.stride[role];
    };
    fill(off_la, g.a, 0, La);
    fill(off_ra, g.a, 1, Ra);
    fill(off_ua, g.a, 2, Ua);
    fill(off_lb, g.b, 0, Lb);
    fill(off_rb, g.b, 1, Rb);
    fill(off_db, g.b, 3, Db);
  }
  __syncthreads();
  float2 *Ec = const_cast<float2 *>(op.Ec);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    op.beta_c_bits = 0u;
    op.beta_t_bits = 0u;
  }
  const float2 *__restrict__ Aa = g.a.A;
  const float2 *__restrict__ Ab = g.b.A;
  const int64_t loa = g.a.lo_off, lob = g.b.lo_off;
  const int64_t a_sd = g.a.stride[3], b_su = g.b.stride[2];  // the shared bond on each site
  const int cc = threadIdx.x & (kEc2T - 1), rq = threadIdx.x / kEc2T;  // column, row group
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int tr = t / tiles_c, tc = t - tr * tiles_c;
    // the tile's rows (a: l_a, u_a, r_a with r_a fastest) and columns
    // (b: l_b, r_b, d_b with d_b fastest): element bases at m = 0 and their
    // share of the output index k N + n
    if (threadIdx.x < kEc2T) {
      const int r = tr * kEc2T + threadIdx.x;
      int64_t base = -1, out = 0;
      if (r < Rows) {
        const int ra = r % Ra, lu = r / Ra, ua = lu % Ua, la = lu / Ua;
        base = tab ? (int64_t)g.a.tau * g.a.tau_stride + off_la[la] + off_ra[ra] + off_ua[ua]
                   : pos_E(g.a, la, ra, ua, 0) - (int64_t)mid_a[0] * a_sd;
        out = ((int64_t)la * Lb * Ua + ua) * N + (int64_t)ra * Rb * Db;
      }
      row_a[threadIdx.x] = base;
      row_out[threadIdx.x] = out;
    } else if (threadIdx.x < 2 * kEc2T) {
      const int c = tc * kEc2T + threadIdx.x - kEc2T;
      int64_t base = -1, out = 0;
      if (c < Cols) {
        const int db = c % Db, lr = c / Db, rb = lr % Rb, lb = lr / Rb;
        base = tab ? (int64_t)g.b.tau * g.b.tau_stride + off_lb[lb] + off_rb[rb] + off_db[db]
                   : pos_E(g.b, lb, rb, 0, db) - (int64_t)mid_b[0] * b_su;
        out = (int64_t)lb * Ua * N + (int64_t)rb * Db + db;
      }
      col_b[threadIdx.x - kEc2T] = base;
      col_out[threadIdx.x - kEc2T] = out;
    }
    __syncthreads();
    float sr[4] = {0.f, 0.f, 0.f, 0.f}, cr[4] = {0.f, 0.f, 0.f, 0.f};
    float si[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    for (int m0 = 0; m0 < Mid; m0 += kEc2M) {
      const int mc = Mid - m0 < kEc2M ? Mid - m0 : kEc2M;
      for (int e = threadIdx.x; e < kEc2T * kEc2M; e += blockDim.x) {
        const int r = e / kEc2M, mm = e - r * kEc2M;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mm < mc && row_a[r] >= 0) {
          const int64_t pa = row_a[r] + (int64_t)mid_a[m0 + mm] * a_sd;
          const float2 h = Aa[pa], l = Aa[loa + pa];
          v = make_float4(h.x, h.y, l.x, l.y);
        }
        As[r][mm] = v;
      }
      for (int e = threadIdx.x; e < kEc2M * kEc2T; e += blockDim.x) {
        const int mm = e / kEc2T, c = e - mm * kEc2T;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mm < mc && col_b[c] >= 0) {
          const int64_t pb = col_b[c] + (int64_t)mid_b[m0 + mm] * b_su;
          const float2 h = Ab[pb], l = Ab[lob + pb];
          v = make_float4(h.x, h.y, l.x, l.y);
        }
        Bs[mm][c] = v;
      }
      __syncthreads();
      for (int mm = 0; mm < mc; ++mm) {
        const float4 b = Bs[mm][cc];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 a = As[rq + 8 * i][mm];
          // re = ar br - ai bi, im = ar bi + ai br (hi products exact, cross terms
          // hi lo + lo hi in the correction)
          acc_prod(a.x, b.x, sr[i], cr[i]);
          acc_prod(-a.y, b.y, sr[i], cr[i]);
          acc_prod(a.x, b.y, si[i], ci[i]);
          acc_prod(a.y, b.x, si[i], ci[i]);
          cr[i] = fmaf(a.x, b.z, fmaf(a.z, b.x, cr[i]));
          cr[i] = fmaf(-a.y, b.w, fmaf(-a.w, b.y, cr[i]));
          ci[i] = fmaf(a.x, b.w, fmaf(a.z, b.y, ci[i]));
          ci[i] = fmaf(a.y, b.z, fmaf(a.w, b.x, ci[i]));
        }
      }
      __syncthreads();
    }
    if (col_b[cc] >= 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rq + 8 * i;
        if (row_a[r] >= 0) Ec[row_out[r] + col_out[cc]] = make_float2(sr[i] + cr[i], si[i] + ci[i]);
      }
    }
    __syncthreads();   // the next tile rewrites the row and column tables
  }
}

// beta = max_n sum_k (|Re E_kn| + |Im E_kn|) of every op (the factor by
// which one absorption can grow max(|Re|, |Im|) of the running tensor); one
// block row per op, after the builders.  A block takes 32 columns at a time,
// its 32 warps splitting K; the column sums meet in shared memory.
__global__ void __launch_bounds__(1024) k_beta_ops(OpDesc *ops) {
  const OpDesc &op = ops[blockIdx.y];
  if (op.Ec == nullptr) return;
  const int K = op.K, N = op.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ float part[32][33];
  float best = 0.f;
  for (int n0 = blockIdx.x * 32; n0 < N; n0 += gridDim.x * 32) {
    const int n = n0 + lane;
    float s = 0.f;
    if (n < N)
      for (int k = w; k < K; k += 32) {
        const float2 v = op.Ec[(int64_t)k * N + n];
        s += fabsf(v.x) + fabsf(v.y);
      }
    part[w][lane] = s;
    __syncthreads();
    if (w == 0) {
      float t = 0.f;
      for (int j = 0; j < 32; ++j) t += part[j][lane];
      best = fmaxf(best, t);
    }
    __syncthreads();
  }
  if (w == 0) {
    best *= 1.0f + 1.0f / 256.0f;
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) atomicMax(&ops[blockIdx.y].beta_c_bits, __float_as_uint(best));
  }
}

// Merge operand from a stored tensor: Ec[k][n] = G[k ks + n ns] 2^-target,
// e_c = exp(G) - target; the bounds are reset for k_beta_ops.
template <int FMT>
__global__ void k_tensor_op(const TensorOpEntry *__restrict__ e, int64_t plane, OpDesc *ops,
                            const Rec *recs) {
  const TensorOpEntry g = e[blockIdx.y];   // one entry per grid row
  OpDesc &op = ops[g.op];
  float2 *Ec = const_cast<float2 *>(op.Ec);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    op.beta_c_bits = 0u;
    op.beta_t_bits = 0u;
    op.e_c = recs[g.rec].exp - g.target;
  }
  const float sc = pow2f(-g.target);
  const int64_t total = (int64_t)g.K * g.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / g.N, n = i - k * g.N;
    const int64_t nh = n / g.Nlo, nl = n - nh * g.Nlo;
    const float2 v = load_g<FMT>(g.G, k * g.ks + nh * g.ns_hi + nl * g.ns, plane);
    Ec[i] = make_float2(v.x * sc, v.y * sc);
  }
}

cudaError_t launch_tensor_operand(const TensorOpEntry *d_entry, int n_entries, int64_t kn,
                                  int fmt, int64_t plane, OpDesc *d_ops, const Rec *d_recs,
                                  cudaStream_t s) {
  if (n_entries <= 0) return cudaSuccess;
  int64_t bx = (kn + 255) / 256;
  if (bx > 4096) bx = 4096;
  if (bx < 1) bx = 1;
  const dim3 blocks((unsigned)bx, (unsigned)n_entries);
  switch (fmt) {
    case FMT_F32: k_tensor_op<FMT_F32><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    case FMT_TF32: k_tensor_op<FMT_TF32><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    case FMT_BF16: k_tensor_op<FMT_BF16><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    case FMT_FP16: k_tensor_op<FMT_FP16><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    case FMT_BF16X2: k_tensor_op<FMT_BF16X2><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    case FMT_FP16X2: k_tensor_op<FMT_FP16X2><<<blocks, 256, 0, s>>>(d_entry, plane, d_ops, d_recs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_operands2(const OpBuild2Entry *d_entries, int n, int max_kn,
                                   OpDesc *d_ops, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  // 32 x 32 tiles of W; about 2048 blocks in all, each walking several tiles
  // of its entry so that its index tables (set up once per block) serve them
  int blocks = (max_kn + 1023) / 1024 + 1;
  const int share = (2048 + n - 1) / n;
  if (blocks > share) blocks = share < 8 ? 8 : share;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  k_build_ec2<<<dim3(blocks, n), 256, 0, s>>>(d_entries, d_ops);
  return cudaGetLastError();
}

cudaError_t launch_build_operands(const OpBuildEntry *d_entries, int n, int max_kn,
                                  OpDesc *d_ops, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (max_kn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_build_ec<<<dim3(blocks, n), 256, 0, s>>>(d_entries, d_ops);
  return cudaGetLastError();
}

cudaError_t launch_operand_bounds(int n_ops, OpDesc *d_ops, cudaStream_t s, int64_t n_cols) {
  if (n_ops <= 0) return cudaSuccess;
  // 32 columns per block and pass; a single op gets a block per 32 columns
  // (at least 128, at most 2048)
  int64_t g1 = (n_cols + 31) / 32;
  g1 = g1 < 128 ? 128 : (g1 > 2048 ? 2048 : g1);
  k_beta_ops<<<dim3(n_ops == 1 ? (unsigned)g1 : 8u, n_ops), 1024, 0, s>>>(d_ops);
  return cudaGetLastError();
}

}  // namespace peps
