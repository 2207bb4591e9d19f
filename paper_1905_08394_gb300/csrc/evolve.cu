// Circuit evolution on the PEPS: initial product state, single-qubit gate
// absorption (K1) and CZ absorption with bond doubling (K2).
//
// Site tensor layout: complex64 [sigma][l][r][u][d], sigma slowest, d fastest.
#include "common.h"
#include "format.cuh"

namespace peps {

// |0> on every site: A^0 = 1, A^1 = 0 with every auxiliary leg of dim 1
// (paper, main-text PEPS equation for the product state).  Also writes the
// scalar 1 in every storage format into the status block (the running
// tensor before the first absorption).
__global__ void k_init_sites(float2 *const *bufs, int n_sites, DeviceStatus *st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_sites) {
    float2 *a = bufs[i];
    a[0] = make_float2(1.f, 0.f);
    a[1] = make_float2(0.f, 0.f);
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

// K1: A'^tau = sum_sigma U[tau][sigma] A^sigma (paper, main-text "onebody"
// equation), in place, for every entry of a batch of gates on distinct sites.
// The tensor is [2][half]; each thread mixes the two sigma slices at two
// consecutive positions (16-byte accesses).
__global__ void k_gate1(const Gate1Entry *__restrict__ entries) {
  const Gate1Entry &g = entries[blockIdx.y];
  const int64_t half = g.half;
  float2 *A = g.A;
  const float2 u00 = g.U[0], u01 = g.U[1], u10 = g.U[2], u11 = g.U[3];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < half;
       e += (int64_t)gridDim.x * blockDim.x) {
    float2 a0 = A[e], a1 = A[half + e];
    float2 b0, b1;
    b0.x = u00.x * a0.x - u00.y * a0.y + u01.x * a1.x - u01.y * a1.y;
    b0.y = u00.x * a0.y + u00.y * a0.x + u01.x * a1.y + u01.y * a1.x;
    b1.x = u10.x * a0.x - u10.y * a0.y + u11.x * a1.x - u11.y * a1.y;
    b1.y = u10.x * a0.y + u10.y * a0.x + u11.x * a1.y + u11.y * a1.x;
    A[e] = b0;
    A[half + e] = b1;
  }
}

// K2: one half of a CZ (paper, main-text "twoqubita/b" with the exact
// projector split of CZ).  The leg `axis` grows from d to 2d with the new
// Schmidt bit s as its least significant bit:
//   projector side:  A'^tau[..., 2*i + s, ...] = delta(tau, s) A^tau[..., i, ...]
//   phase side:      A'^tau[..., 2*i + s, ...] = (-1)^(s*tau) A^tau[..., i, ...]
// With fixed_s >= 0 (a sliced CZ) the leg keeps its size and only the term
// s = fixed_s is applied.  One thread per output entry.
__global__ void k_cz(const CzEntry *__restrict__ entries) {
  const CzEntry &g = entries[blockIdx.y];
  int od[4] = {g.dims[0], g.dims[1], g.dims[2], g.dims[3]};
  const bool bundle = g.fixed_s < 0;
  if (bundle) od[g.axis] *= 2;
  const int64_t half_out = (int64_t)od[0] * od[1] * od[2] * od[3];
  const int64_t total = 2 * half_out;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
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
    float2 v = g.in[in_e];
    float f;
    if (g.kind == 0) f = (tau == s) ? 1.f : 0.f;
    else f = (s & tau) ? -1.f : 1.f;
    g.out[e] = make_float2(f * v.x, f * v.y);
  }
}

static int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_init_sites(float2 *const *bufs, int n_sites, DeviceStatus *st,
                              cudaStream_t s) {
  int threads = 128;
  int blocks = (n_sites + threads - 1) / threads;
  if (blocks < 1) blocks = 1;
  k_init_sites<<<blocks, threads, 0, s>>>(bufs, n_sites, st);
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

}  // namespace peps
