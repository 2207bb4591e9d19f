// Internal declarations shared by the translation units of libpeps_gb300.
// Not part of the public ABI (see include/peps_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/peps_gb300.h"

namespace peps {

// ---------------------------------------------------------------------------
// Storage formats of the running tensor G (one complex entry = re, im).
// ---------------------------------------------------------------------------
enum Format : int {
  FMT_F32 = 0,     // float2                                  (8 B / entry)
  FMT_BF16 = 1,    // bf16 re, bf16 im, interleaved            (4 B)
  FMT_FP16 = 2,    // fp16 re, fp16 im, interleaved            (4 B)
  FMT_BF16X2 = 3,  // two planes (hi, lo) of interleaved bf16  (8 B)
  FMT_FP16X2 = 4,  // two planes (hi, lo) of interleaved fp16  (8 B)
  FMT_TF32 = 5,    // float2 holding values rounded to TF32    (8 B)
};

inline int format_of(int precision) {
  switch (precision) {
    case PEPS_FP32_SIMT: return FMT_F32;
    case PEPS_TF32: return FMT_TF32;
    case PEPS_BF16: return FMT_BF16;
    case PEPS_BF16X3: return FMT_BF16X2;
    case PEPS_FP16: return FMT_FP16;
    case PEPS_FP16X3: return FMT_FP16X2;
  }
  return -1;
}

inline int format_bytes_per_entry(int fmt) {
  return (fmt == FMT_BF16 || fmt == FMT_FP16) ? 4 : 8;
}

// Largest stored magnitude the per-step scaling aims for: 2^target.  FP16
// formats keep G near the top of their range so that the lo plane of a
// hi/lo split stays normal; the other formats keep G at most 1.
inline int scale_target(int fmt) {
  return (fmt == FMT_FP16 || fmt == FMT_FP16X2) ? 14 : 0;
}

// Scale exponent of the tensor-core site operand (B) per format: the site
// tensor entries satisfy |E| <= 1, so 2^12 keeps fp16 pieces in range.
inline int operand_scale_exp(int fmt) {
  return (fmt == FMT_FP16 || fmt == FMT_FP16X2) ? 12 : 0;
}

// ---------------------------------------------------------------------------
// Device-side tables
// ---------------------------------------------------------------------------

// One site operand E = A_q^{tau} (optionally restricted to a slice), in the
// layouts the contraction kernels read.
struct OpDesc {
  const float2 *Ec;     // [K][N] complex64, k = l*du + u, n = r*dd + d
  const void *Bt[2];    // tensor-core planes [Nr_pad][Kr_pad] (hi, lo), or null
  uint32_t beta_c_bits; // max_n sum_k (|Re E_kn| + |Im E_kn|), float bits
  uint32_t beta_t_bits; // same bound for the scaled tensor-core planes
  int32_t b_t;          // scale exponent of the tensor-core planes (Bt = Ec 2^b_t)
  int32_t K, N;         // complex dims
  int32_t e_c;          // Ec = E 2^e_c (0 for site operands; a merge operand
                        // built from a stored tensor carries that tensor's scale)
};

// Per (lane, step) record: the max |stored entry| of the step's output
// (float bits, atomicMax target) and the cumulative scale exponent S:
// stored G = true G * 2^S.
struct Rec {
  uint32_t maxbits;
  int32_t exp;
};

// One work item of a contraction launch: one lane (bitstring or prefix
// chain) absorbing one site.
struct StepItem {
  const void *A;          // input G (format of the launch)
  void *D;                // output G
  const uint64_t *bits;   // the lane's bitstring (device)
  int32_t op_base;        // OpDesc index of tau = 0 (tau = 1 is op_base + 1)
  int32_t in_rec;         // Rec index of the input (-1: the unit scalar)
  int32_t out_rec;        // Rec index of the output
  int32_t a_lane;         // lane coordinate of A in the launch's tensor map
  int32_t b_slot;         // operand slot of the item past the launch's first
                          // (the tensor-core B map's variant coordinate is
                          // b_slot + the bitstring's variant; op_base already
                          // includes it): the square partition's merges of
                          // several groups, each with its own operand
  int32_t pad_;
};

// Shape shared by all items of a launch.  A step absorbs a block of nq
// vertically adjacent sites (rows r .. r+nq-1 of one column) at once.
struct StepShape {
  int64_t M;      // product of the untouched h legs
  int32_t K;      // dim(h_r) * ... * dim(h_{r+nq-1}) * dim(v)
  int32_t N;      // dim(h'_r) * ... * dim(h'_{r+nq-1}) * dim(v')
  int64_t P;      // product of the dims of the slowest M legs that the next
                  // block contracts (moved next to v' on store)
  int32_t dv_out; // dim(v')
  int32_t dh_out; // dim(h'_r) * ... * dim(h'_{r+nq-1})
  int32_t q;      // first site of the block
  int32_t fmt;    // storage format of A and D
  int64_t plane;  // element offset of the lo plane (FMT_*X2), in 16-bit units
  int32_t target; // scale target exponent
  int32_t nq;     // sites in the block (their q are q, q + qs, ...); 0 for
                  // a merge of two quarter tensors (one operand)
  int32_t qs;     // site stride (C)
  int32_t vb;     // 1: v' is an open leg; it joins the batch (below) and the
                  // stored output's v leg has dim 1
  int32_t nvs;    // N order: 0 = (h', v') with v' fastest (the operand's
                  // n = r*dd + d); 1 = (v', h') with h' fastest (n = d*dr + r),
                  // used where that makes the store contiguous (vb with P = 1)
  int32_t ksplit; // tensor cores: K segments with separate FP32 accumulators
                  // (0 or 1 = one); the tensor core's accumulation error grows
                  // with the number of MMAs summed into one accumulator
  int32_t csep;   // tensor cores, split forms: the hi*lo and lo*hi products go
                  // to an accumulator of their own (a third of the updates of
                  // the main one; their own error is 2^-11 smaller)
  int32_t nx;     // held bond bits (PEPS_FLAG_HOLD_TIES): other qubits whose
                  // output bits select the operand variant, xq[0 .. nx)
  int64_t Mr;     // M = (batch) x Mr: the slowest M legs form a batch (open
                  // legs of a quarter that are never contracted in its
                  // sweep); 0 = no batch (Mr = M).  Row m = b * Mr + m_r;
                  // the P rotation acts on m_r only, and the output is
                  //   vb = 0: b * (Mr N) + ((m_lo dh' + h') P + m_hi) dv' + v'
                  //   vb = 1: (b dv' + v') (Mr dh') + (m_lo dh' + h') P + m_hi
  int32_t xq[4];
  int32_t dot;    // tensor cores, a merge whose output is only dotted with a
                  // stored tensor (the square partition's last contraction):
                  // the item's D is that tensor, read; the epilogue writes
                  // the partial sums sum_n out[m, n] D[m N + n] (unscaled) per
                  // (tile, CTA, warp) instead of storing the output
  int32_t pad3_;
};

// Operand index of a lane for a block: bit j = output bit of the block's
// j-th site (for one site: tau), then bit nq + i = output bit of qubit xq[i]
// (the held bond bits of the block's legs that depend on a neighbour).
__host__ __device__ inline int block_variant(uint64_t bits, const StepShape &sh) {
  int v = 0;
  for (int j = 0; j < sh.nq; ++j) v |= (int)((bits >> (sh.q + j * sh.qs)) & 1ull) << j;
  for (int i = 0; i < sh.nx; ++i) v |= (int)((bits >> sh.xq[i]) & 1ull) << (sh.nq + i);
  return v;
}

// Operand variants of a step.
__host__ __device__ inline int step_variants(const StepShape &sh) { return 1 << (sh.nq + sh.nx); }

// Evolution tables.  Site tensors are kept as float-float pairs: a hi plane
// and a lo plane (value = hi + lo), the lo plane `lo_off` entries after the
// hi plane of the same buffer.
struct Gate1Entry {  // single-qubit gate on one site tensor (in place)
  float2 *A;
  int64_t half;      // elements per sigma slice
  int64_t lo_off;    // entries from the hi plane to the lo plane
  float2 U_hi[4];    // the gate as float-float: U = U_hi + U_lo
  float2 U_lo[4];
};

struct CzEntry {     // one half of a CZ on one site tensor (out of place)
  const float2 *in;
  float2 *out;
  int64_t lo_off;
  int32_t dims[4];   // input l, r, u, d
  int32_t axis;      // 0..3 = l, r, u, d
  int32_t kind;      // 0 = projector P_s, 1 = phase Z^s
  int32_t fixed_s;   // -1: bundle s into the leg; 0/1: sliced term
  int32_t pad_;
};

// One half of a general two-qubit gate split as sum_s W0_s (x) W1_s (main
// text, "factorize"; rank chi <= 4): on this site
//   A'^tau[..., i*chi + s, ...] = sum_sigma W_s[tau][sigma] A^sigma[..., i, ...]
// (the leg `axis` grows from d to d*chi, s fastest), out of place.  W as
// float-float: W = W_hi + W_lo, index [s][2*tau + sigma].
struct Gate2Entry {
  const float2 *in;
  float2 *out;
  int64_t lo_off;
  int32_t dims[4];   // input l, r, u, d
  int32_t axis;      // 0..3 = l, r, u, d
  int32_t chi;       // Schmidt rank, 1..4
  float2 W_hi[4][4];
  float2 W_lo[4][4];
};

// One gate half of a site's evolution list (the per-site evolution kernel):
// kind 0 = Gate1Entry, 1 = CzEntry, 2 = Gate2Entry; idx into that table.
struct EvoRef {
  int32_t kind;
  int32_t idx;
};

// Operand build entry (one site, one tau, one slice variant).  The four legs
// are given by their role in the sweep that absorbs the site: l and u are
// contracted (K = l u), r and d are new (N = r d).  For the column sweep the
// roles are the physical legs; a quarter swept from another corner or
// transposed maps them to other physical legs through `stride`.
// most linked bits on one leg (bond bits tied to another bit of the same bond)
constexpr int kMaxLinks = 6;

struct OpBuildEntry {
  const float2 *A;      // site tensor [2][l][r][u][d] (full dims), hi plane
  int64_t lo_off;       // entries from the hi plane to the lo plane
  int32_t dims[4];      // full dims by role l, r, u, d
  int32_t rdims[4];     // restricted dims by role
  uint32_t free_mask[4];// bits of the full index that vary (by role); all ones
                        // = nothing fixed (the index is the full index)
  uint32_t fixed_val[4];// value of the fixed bits (by role)
  uint8_t n_links[4];   // linked bits by role: bit link_dst = bit link_src XOR
  uint8_t link_src[4][kMaxLinks];  // (the dst bit's value in fixed_val)
  uint8_t link_dst[4][kMaxLinks];
  int64_t stride[4];    // element stride of each role's physical leg
  int64_t tau_stride;   // elements per sigma slice
  int32_t tau;
  int32_t op;           // OpDesc index to fill
  int32_t nvs;          // N order of the operand (StepShape::nvs)
  int32_t dl;           // 0: E = A^tau; double layer (marginals): 1 = sum over
                        // sigma = tau, 2 = over sigma in {0, 1} of A^sigma (x)
                        // conj(A^sigma).  Then `dims` are the single-layer
                        // dims and `rdims` their squares; a doubled index is
                        // ket * dim + bra.
};

// largest internal vertical bond of a two-site block operand
constexpr int kMaxMid = 1024;

// Operand build of a two-site block (rows r, r+1 of a column):
//   W[(l_a, l_b, u_a), (r_a, r_b, d_b)] = sum_m E_a[l_a, r_a, u_a, m] E_b[l_b, r_b, m, d_b]
// with E_a = A_a^{tau_a}, E_b = A_b^{tau_b} (restricted legs as for one site).
struct OpBuild2Entry {
  OpBuildEntry a, b;
  int32_t op;
  int32_t pad_;
};

// Operand of a merge built from a finished quarter (or half) tensor G held in
// the running-tensor format:  Ec[k][n] = G[k ks + n_hi ns_hi + n_lo ns] 2^-target
// with n = n_hi * Nlo + n_lo (so that |Ec| <= 1), and e_c of the op =
// exp(G's record) - target, which carries G's scale into the merge's output
// exponent.  The two-level N index reorders the operand's columns (a leg
// moved to the front); Nlo = N gives the plain strided gather.
struct TensorOpEntry {
  const void *G;
  int64_t ks, ns;       // element strides of the operand's K and (low) N indices
  int64_t ns_hi;        // element stride of the high N index
  int64_t Nlo;          // size of the low N index
  int32_t K, N;
  int32_t rec;          // G's record
  int32_t op;           // OpDesc to fill
  int32_t target;       // scale target of G's storage
  int32_t pad_;
};

// amplitude += sum_i Y[i] F[i] 2^-(S_Y + S_F): the final contraction of the
// square partition (Y and F in the running-tensor format, same layout).
// nslots: partial sums of the entry to add (kDotBlocks for the separate dot
// kernel; the fused merge's slot count otherwise).
struct DotEntry {
  const void *Y, *F;
  int64_t n;
  int32_t rec_y, rec_f;
  int32_t out_index;
  int32_t nslots;
};

struct FinalEntry {     // one output amplitude contribution
  const void *G;        // final 1x1 G of a lane
  int32_t rec;          // its Rec
  int32_t out_index;    // bitstring index
};

// Status words at the head of the workspace.
struct DeviceStatus {
  int32_t error;        // nonzero: a device check failed
  int32_t error_info;
  int32_t timeout;      // nonzero: a bounded wait expired
  int32_t pad_;
  float2 unit_f32;      // the scalar 1 in each format
  uint32_t unit_h16[2]; // bf16 (re=1, im=0) hi plane / lo plane
  uint32_t unit_f16[2]; // fp16 (re=1, im=0) hi plane / lo plane
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
cudaError_t launch_init_sites(float2 *const *bufs, const int64_t *lo_off, int n_sites,
                              DeviceStatus *st, cudaStream_t s);
cudaError_t launch_gate1(const Gate1Entry *d_entries, int n, int64_t max_half,
                         cudaStream_t s);
// The whole evolution in one launch: block q applies site q's gate halves
// refs[first[q] .. first[q+1]) in order, from |0> in bufs[q].
cudaError_t launch_evolve_sites(const Gate1Entry *g1, const CzEntry *cz, const Gate2Entry *g2,
                               const EvoRef *refs, const int32_t *first, float2 *const *bufs,
                               const int64_t *lo_off, int n_sites, DeviceStatus *st,
                               cudaStream_t s);
cudaError_t launch_cz(const CzEntry *d_entries, int n, int64_t max_out, cudaStream_t s);
cudaError_t launch_gate2(const Gate2Entry *d_entries, int n, int64_t max_out, cudaStream_t s);
cudaError_t launch_build_operands(const OpBuildEntry *d_entries, int n, int max_kn,
                                  OpDesc *d_ops, cudaStream_t s);
// `n_cols`: the widest operand's N (sizes the grid of a single op)
cudaError_t launch_operand_bounds(int n_ops, OpDesc *d_ops, cudaStream_t s,
                                  int64_t n_cols = 4096);
cudaError_t launch_tensor_operand(const TensorOpEntry *d_entries, int n_entries, int64_t kn,
                                  int fmt, int64_t plane, OpDesc *d_ops, const Rec *d_recs,
                                  cudaStream_t s);
// Blocks per DotEntry; `d_partials` holds kDotBlocks double2 per entry.
constexpr int kDotBlocks = 256;
cudaError_t launch_dot(const DotEntry *d_entries, int n, int fmt, int64_t plane,
                       const Rec *d_recs, double2 *d_partials, double2 *d_acc, cudaStream_t s);
// Only the final pass (the partial sums were written by a fused merge).
cudaError_t launch_dot_final(const DotEntry *d_entries, int n, const Rec *d_recs,
                             const double2 *d_partials, double2 *d_acc, cudaStream_t s);
cudaError_t launch_build_operands2(const OpBuild2Entry *d_entries, int n, int max_kn,
                                   OpDesc *d_ops, cudaStream_t s);
// A merge operand's tensor-core planes and bound straight from the stored
// tensor (no Ec); K, N are the operand's sizes.
cudaError_t launch_tensor_operand_tc(const TensorOpEntry *d_entries, int n_entries, int K, int N,
                                     int fmt, int64_t plane, OpDesc *d_ops, const Rec *d_recs,
                                     cudaStream_t s);
// Tensor-core planes (and their bound) of ops [0, n_ops) from their Ec.
cudaError_t launch_build_tc_operands(int n_ops, int64_t max_kn, OpDesc *d_ops, int fmt,
                                     cudaStream_t s);
cudaError_t launch_contract_simt(const StepShape &sh, const StepItem *d_items, int n_items,
                                 const OpDesc *d_ops, Rec *d_recs, const DeviceStatus *st,
                                 cudaStream_t s);
// Whole sweeps of small lattices in one persistent launch (contract_small.cu):
// the plan's steps and their first operand index, the bitstrings and the
// FP64 amplitude accumulators; cap_g / cap_e = entries of the largest running
// tensor / operand (shared memory: two running tensors and one operand).
struct SmallSweep {
  const StepShape *steps;
  const int32_t *op_base;
  const OpDesc *ops;
  const uint64_t *bits;
  double2 *acc;
  int64_t n;
  int32_t n_steps;
  int32_t cap_g;
  int32_t cap_e;
  int32_t pad_;
};
constexpr size_t kSmallSweepMaxSmem = 96 * 1024;
size_t small_sweep_smem(int cap_g, int cap_e);
cudaError_t launch_sweep_small(const SmallSweep &p, int sm_count, cudaStream_t s);

cudaError_t launch_finalize(const FinalEntry *d_entries, int n, int fmt, int64_t plane,
                            const Rec *d_recs, double2 *d_acc, cudaStream_t s);
cudaError_t launch_store_out(const double2 *d_acc, peps_c128 *d_out, int64_t n,
                             cudaStream_t s);
cudaError_t launch_check_groups(const uint64_t *d_bits, int64_t n, int group,
                                uint64_t mask, DeviceStatus *st, cudaStream_t s);

// tcgen05 contraction (contract_tc.cu).
bool tc_supports(const StepShape &sh, int fmt);
bool tc_tuning_valid(int kchunk, int cluster, int epi);
// Encode the launch's tensor maps (A over the lanes' input buffers, Bt for
// tau = 0/1 and each plane); returns 0 and an opaque handle, or < 0.
// The B operands: plane pl of variant t at b_base[pl] + t * b_var_stride
// bytes (n_var variants, equally spaced).
int tc_prepare(const StepShape &sh, int fmt, const void *a_base, int a_lanes,
               int64_t a_lane_stride, int64_t plane_stride_bytes, const void *const b_base[2],
               int n_var, int64_t b_var_stride, int kchunk, int cluster, int epi,
               void **out_handle);
void tc_release(void *handle);
// One-time set-up of the kernel a handle launches (attributes, occupancy);
// done before a stream capture so that no such call happens inside it.
cudaError_t tc_warm(void *handle);
cudaError_t launch_contract_tc(void *handle, const StepItem *d_items, int n_items,
                               const OpDesc *d_ops, Rec *d_recs, DeviceStatus *st,
                               int64_t watchdog_ns, int sm_count, cudaStream_t s,
                               double2 *dot_partials = nullptr);
// Partial-sum slots per item of a fused-dot launch (sh.dot).
int tc_dot_slots(const void *handle);
int tc_Kr_pad(int K);   // real K of a tensor-core operand
int tc_Nr_pad(int N);   // real N

// For the allocation-free entry point (noalloc.cu): set the thread's error
// text and return `code`; drop a context's cached plan and built site tensors.
int internal_fail(int code, const char *fmt, ...);
void internal_forget_workspace(peps_ctx *ctx);

}  // namespace peps
