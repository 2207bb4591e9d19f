// K4 (tensor-core forms): one site absorption of the column sweep as a
// complex-as-real GEMM on the 5th-generation tensor cores (tcgen05), for a
// batch of lanes,
//   D[M x Nr] = A[M x Kr] * Bt[Nr x Kr]^T,   Kr = 2K, Nr = 2N,
// A = the running tensor G (interleaved re/im, the contracted legs (h_r, v)
// fastest), Bt = the real embedding of the site operand E:
//   Bt[2n  ][2k] =  Re E_kn   Bt[2n  ][2k+1] = -Im E_kn
//   Bt[2n+1][2k] =  Im E_kn   Bt[2n+1][2k+1] =  Re E_kn
// so that D's row is the interleaved complex output row (supplementary
// exact-overlap absorption step, transposed to columns).
//
// Forms: BF16 / FP16 (kind::f16, one MMA per k-step), BF16X2 / FP16X2 (hi/lo
// planes of A and Bt, three MMAs hi*hi + hi*lo + lo*hi accumulated in FP32),
// TF32 (kind::tf32, one MMA).
//
// Structure: persistent CTAs (one per SM) walk tiles (lane, M block, N block
// of up to 256 real columns).  Warp 0 issues TMA loads of A and Bt tiles
// (128-byte or 64-byte swizzle) into a ring of shared-memory stages, warp 1
// issues tcgen05.mma into one of two TMEM accumulators, warps 2..5 drain the
// other accumulator with tcgen05.ld, apply the step's power-of-two scale,
// split into the storage format and store permuted (the slowest untouched leg
// moves next to v'), and record the max |entry|.
//
// CG = 2 (the default where the row tiles pair up): a cluster of two CTAs on
// neighbouring SMs computes a 256-row tile with the 2-SM UMMA
// (tcgen05.mma.cta_group::2, M = 256).  Each CTA loads its own 128 rows of A
// and only half of the Bt tile; the even CTA issues the MMAs for both, and
// the TMA completions of both CTAs arrive on its barriers.  Per SM this
// halves the Bt bytes ingested per multiply-add, which is what bounds the
// single-CTA form (the MMA warp waits on operand arrival, not on the
// epilogue).  Every wait is bounded by a %globaltimer budget; on expiry the
// CTA raises the abort flag in both CTAs, sets the device timeout word,
// drains and releases TMEM before returning.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.h"
#include "format.cuh"

namespace peps {

namespace {

constexpr int BM = 128;
// Warps: a TMA producer, an MMA issuer and EPI epilogue warps; EPI = 4 (one per
// TMEM lane quadrant) or 8 (two per quadrant, each draining half of the
// tile's columns, for steps whose epilogue outlasts their MMAs).
constexpr int threads_of(int epi) { return 64 + 32 * epi; }

template <int FMT> struct FormTraits;
template <> struct FormTraits<FMT_BF16>   { static constexpr int NP = 1, ESZ = 2, KIND = 0, AB = 1; };
template <> struct FormTraits<FMT_FP16>   { static constexpr int NP = 1, ESZ = 2, KIND = 0, AB = 0; };
template <> struct FormTraits<FMT_BF16X2> { static constexpr int NP = 2, ESZ = 2, KIND = 0, AB = 1; };
template <> struct FormTraits<FMT_FP16X2> { static constexpr int NP = 2, ESZ = 2, KIND = 0, AB = 0; };
template <> struct FormTraits<FMT_TF32>   { static constexpr int NP = 1, ESZ = 4, KIND = 1, AB = 2; };

// x / d and x % d for a divisor fixed per launch (d > 0, x >= 0): a shift and
// a mask when d is a power of two (every dimension made of CZ bonds), a
// division otherwise (bonds of general two-qubit gates of Schmidt rank 3).
struct Div {
  int64_t d;
  int32_t s;   // log2(d), or -1
  int32_t pad_;
  __device__ __forceinline__ int64_t q(int64_t x) const { return s >= 0 ? (x >> s) : x / d; }
  __device__ __forceinline__ int64_t r(int64_t x) const {
    return s >= 0 ? (x & (d - 1)) : x % d;
  }
};
inline Div make_div(int64_t d) {
  Div v{d > 0 ? d : 1, -1, 0};
  if ((v.d & (v.d - 1)) == 0) {
    int k = 0;
    while (((int64_t)1 << k) < v.d) ++k;
    v.s = k;
  }
  return v;
}

struct __align__(128) TcParams {   // the tensor maps need 128-byte alignment
  CUtensorMap mapA;        // {k, m, plane, lane}; m_hi-major steps: {k, m_hi, m_lo, b, plane/lane}
  CUtensorMap mapB[2];     // [plane] {k, n, operand variant}
  StepShape sh;
  const StepItem *items;
  const OpDesc *ops;
  Rec *recs;
  DeviceStatus *st;
  int n_items;
  int tiles_m, tiles_n;
  int BN;
  int stages;
  int tmem_cols;
  int ksplit;   // K segments accumulated in separate TMEM columns, summed in the
                // epilogue with round-to-nearest FP32 adds (long-K steps)
  int csep;     // 1: the split form's correction products (hi*lo, lo*hi) have
                // their own accumulator after the K segments
  int nacc;     // accumulators per buffer: ksplit + csep
  int nbuf;     // accumulator buffers (2: the epilogue of a tile overlaps the
                // next tile's MMAs)
  int mhi;      // 1: a tile's rows are ph consecutive m_hi x lh consecutive m_lo
                // (ph lh = BM) at one b, so that the open-leg store (contiguous
                // in m_hi only) coalesces
  int lp_mul;   // m_hi-major: the A map's last coordinate is lane * lp_mul + plane
  int ph, lh;   // m_hi-major: tile extent in m_hi (min(P, BM)) and in m_lo
  int gm;       // tile order: gm row groups at a time, n fastest within them
                // (1: n fastest over a whole row group)
  int64_t mlo;  // m_hi-major: Mr / P
  int64_t watchdog_ns;
  double2 *dot_partials;   // sh.dot: [item][tiles_per_item * CG * EPI]
  int blocked;  // 1: CTA pair c takes the consecutive tiles [c per, (c + 1) per)
                // (an item's tiles in a row, so its variant, scale and
                // addresses are set up once); 0: tiles c, c + pairs, ...
  // divisors of the tile and store index arithmetic
  Div d_tpi, d_tn;             // tiles per item, column tiles
  Div d_hper, d_lper, d_ph;    // m_hi-major tiles: P / ph, (Mr / P) / lh, ph
  Div d_Mr, d_Mlo, d_dv, d_dh; // output rows per batch slice, Mr / P, dim(v'), dim(h')
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Set the int at the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ void st_cluster_flag(volatile int *local, uint32_t rank, int v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote)
               : "r"(smem_u32((const void *)local)), "r"(rank));
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
}

struct Watch {
  volatile int *abort;
  DeviceStatus *st;
  uint64_t deadline;
  int where;
  int cs;  // cluster size: an expired wait raises the abort flag in every CTA
};

// Bounded wait on an mbarrier phase.  Returns false on abort or timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, Watch &w) {
  uint32_t spins = 0;
  while (!mbar_test(bar, parity)) {
    if ((++spins & 63) == 0) {
      if (*w.abort) return false;
      if (globaltimer() > w.deadline) {
        *w.abort = 1;
        if (w.cs > 1)
          for (int r = 0; r < w.cs; ++r) st_cluster_flag(w.abort, (uint32_t)r, 1);
        atomicExch(&w.st->timeout, 1);
        atomicExch(&w.st->error_info, w.where);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
// Shared::cluster address of the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
  return r;
}
// Arrive on an mbarrier given by its shared::cluster address (any CTA).
// Relaxed: the epilogue's arrival only has to follow its own completed TMEM
// reads (tcgen05.wait::ld, in program order); its global stores are for the
// next launch, so a release (which waits for them) would stall the epilogue.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   bar_cluster_addr)
               : "memory");
}
// Arrive with release semantics on an mbarrier given by its shared::cluster
// address: the stores to the cluster's shared memory before it are visible to
// a thread that sees the phase complete.
__device__ __forceinline__ void mbar_arrive_cluster_release(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   bar_cluster_addr)
               : "memory");
}
// Count `bytes` of transactions as complete on a local mbarrier (bytes that
// will never arrive: the pair's other CTA issued no load for that stage).
__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// TMA loads of a CTA pair: the data lands in this CTA's shared memory and the
// completion is counted on the mbarrier at `bar_cluster_addr` (the even CTA's).
__device__ __forceinline__ void tma_load_4d_cg2(void *dst, const CUtensorMap *map,
                                                uint32_t bar_cluster_addr, int c0, int c1, int c2,
                                                int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar_cluster_addr)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d_cg2(void *dst, const CUtensorMap *map,
                                                uint32_t bar_cluster_addr, int c0, int c1, int c2,
                                                int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar_cluster_addr)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d_cg2(void *dst, const CUtensorMap *map,
                                                uint32_t bar_cluster_addr, int c0, int c1,
                                                int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar_cluster_addr)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Tile `rem` of an item -> (row group mg, column tile nt).  Blocks of gm row
// groups are walked column by column, so that the tiles in flight at once
// (one per CTA pair) share the k-slabs of gm A row panels and of a few B
// column panels in L2; gm = 1 is the plain n-fastest order.
__device__ __forceinline__ void tile_of(int rem, int mgroups, int tiles_n, int gm, int &mg,
                                        int &nt) {
  if (gm <= 1) {
    mg = rem / tiles_n;
    nt = rem - mg * tiles_n;
    return;
  }
  const int blk = rem / (gm * tiles_n), within = rem - blk * gm * tiles_n;
  const int g0 = blk * gm, gsz = mgroups - g0 < gm ? mgroups - g0 : gm;
  nt = within / gsz;
  mg = g0 + (within - nt * gsz);
}

// Shared-memory matrix descriptor of a K-major swizzled tile (rows of
// `rowb` bytes, 8-row core groups `8 * rowb` bytes apart).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t rowb) {
  const uint64_t layout = rowb == 128 ? 2ull : 4ull;  // SWIZZLE_128B : SWIZZLE_64B
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                               // leading offset (unused, K-major swizzled)
  d |= (uint64_t)(((8u * rowb) >> 4) & 0x3FFFu) << 32;  // stride offset between 8-row groups
  d |= (uint64_t)1 << 46;                               // descriptor version
  d |= layout << 61;
  return d;
}

template <int KIND, int CG>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if (CG == 2) {
    if (KIND == 0)
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
          "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
          "l"(a), "l"(b), "r"(idesc), "r"(acc));
    return;
  }
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// Commit of the pair's MMAs: arrives on the mbarrier at this offset in both CTAs.
__device__ __forceinline__ void mma_commit_cg2(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Issue a 32-lane x 16-column TMEM load (asynchronous: the registers are
// valid after tmem_wait()).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Wait for the outstanding TMEM loads; the registers of the last load are
// in/out operands so that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// ---------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------
// CG: CTAs per MMA.  CG = 1: one CTA per 128-row tile.  CG = 2: a cluster of
// two CTAs per 256-row tile (2-SM UMMA), see the file comment.
template <int FMT, int ROWB, int CG, int EPI>
__global__ void __launch_bounds__(threads_of(EPI), 1)
    k_contract_tc(const __grid_constant__ TcParams p) {
  using T = FormTraits<FMT>;
  constexpr int NP = T::NP;
  constexpr int KSTEPS = ROWB / 32;  // 32-byte MMA k-steps per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem =
      (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const int BN = p.BN;              // real output columns per tile (MMA N)
  const int BNL = BN / CG;          // Bt rows held by this CTA
  const int S = p.stages;
  const uint32_t a_bytes = BM * ROWB;
  const uint32_t b_bytes = (uint32_t)BNL * ROWB;
  const uint32_t stage_bytes = NP * (a_bytes + b_bytes);  // this CTA's share
  uint64_t *bars = (uint64_t *)(smem + (size_t)S * stage_bytes);
  uint64_t *full = bars;
  uint64_t *empty = bars + S;
  uint64_t *tfull = bars + 2 * S;
  uint64_t *tempty = bars + 2 * S + 2;
  uint64_t *done = bars + 2 * S + 4;
  uint64_t *pdone = bars + 2 * S + 5;  // CG = 2: the odd producer has finished issuing
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * S + 6);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  volatile uint32_t *odd_issued = tmem_slot + 2;  // CG = 2: stages the odd CTA issued

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = CG > 1 ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      // the pair's epilogue warps (one elected lane each) release an accumulator
      mbar_init(&tempty[a], CG == 2 ? 2 * EPI : 32 * EPI);
    }
    mbar_init(done, 1);
    mbar_init(pdone, 1);
    *abort_flag = 0;
    *odd_issued = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(p.tmem_cols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(p.tmem_cols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (CG > 1) cluster_sync();  // both CTAs' barriers exist before any remote signal
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int cid = blockIdx.x / CG, ncl = gridDim.x / CG;
  const int mgroups = p.tiles_m / CG;               // CG == 2 only when tiles_m is even
  const int tiles_per_item = mgroups * p.tiles_n;  // tiles of the pair
  const int total = p.n_items * tiles_per_item;
  // this pair's tiles: a consecutive range (blocked) or every ncl-th
  const int per = p.blocked ? (total + ncl - 1) / ncl : 1;
  const int t_first = p.blocked ? cid * per : cid;
  const int t_end = p.blocked ? (t_first + per < total ? t_first + per : total) : total;
  const int t_step = p.blocked ? 1 : ncl;
  // a row of A holds 2K real entries of ESZ bytes; one stage covers ROWB bytes
  const int kb_count = (2 * p.sh.K * T::ESZ) / ROWB;
  Watch w{abort_flag, p.st, globaltimer() + (uint64_t)p.watchdog_ns, p.sh.q, CG};
  // the even CTA's barriers, as cluster addresses
  const uint32_t full0 = CG == 2 ? cluster_addr(full, 0) : 0u;
  const uint32_t tempty0 = CG == 2 ? cluster_addr(tempty, 0) : 0u;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      uint32_t it = 0;
      int cached_item = -1, tau = 0, a_lane = 0;
      for (int t = t_first; t < t_end; t += t_step) {
        const int item = (int)p.d_tpi.q(t);
        const int rem = t - item * tiles_per_item;
        int mg, nt;
        if (p.gm <= 1) {
          mg = (int)p.d_tn.q(rem);
          nt = rem - mg * p.tiles_n;
        } else {
          tile_of(rem, mgroups, p.tiles_n, p.gm, mg, nt);
        }
        const int mt = mg * CG + (int)rank;
        if (item != cached_item) {
          cached_item = item;
          const StepItem &si = p.items[item];
          tau = block_variant(*si.bits, p.sh) + si.b_slot;
          a_lane = si.a_lane;
        }
        // m_hi-major: tile mt is rows m_hi = hb0 .. hb0+ph-1, m_lo = mlo_t ..
        // mlo_t+lh-1 at b_t
        int64_t b_t = 0, mlo_t = 0;
        int hb0 = 0;
        if (p.mhi) {
          const int64_t rest = p.d_hper.q(mt);
          hb0 = (int)p.d_hper.r(mt) * p.ph;
          b_t = p.d_lper.q(rest);
          mlo_t = p.d_lper.r(rest) * p.lh;
        }
        bool ok = true;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, w)) { ok = false; break; }
          unsigned char *st = smem + (size_t)s * stage_bytes;
          const int k0 = kb * (ROWB / T::ESZ);
          if (CG == 1) {
            mbar_expect_tx(&full[s], stage_bytes);
            for (int pl = 0; pl < NP; ++pl) {
              if (p.mhi)
                tma_load_5d(st + pl * a_bytes, &p.mapA, &full[s], k0, hb0, (int)mlo_t, (int)b_t,
                            a_lane * p.lp_mul + pl);
              else
                tma_load_4d(st + pl * a_bytes, &p.mapA, &full[s], k0, mt * BM, pl, a_lane);
              tma_load_3d(st + NP * a_bytes + pl * b_bytes, &p.mapB[pl], &full[s], k0,
                          nt * BN, tau);
            }
          } else {
            // the even CTA's full barrier counts both CTAs' bytes
            if (leader) mbar_expect_tx(&full[s], 2 * stage_bytes);
            for (int pl = 0; pl < NP; ++pl) {
              if (p.mhi)
                tma_load_5d_cg2(st + pl * a_bytes, &p.mapA, full0 + (uint32_t)s * 8u, k0, hb0,
                                (int)mlo_t, (int)b_t, a_lane * p.lp_mul + pl);
              else
                tma_load_4d_cg2(st + pl * a_bytes, &p.mapA, full0 + (uint32_t)s * 8u, k0,
                                mt * BM, pl, a_lane);
              tma_load_3d_cg2(st + NP * a_bytes + pl * b_bytes, &p.mapB[pl],
                              full0 + (uint32_t)s * 8u, k0, nt * BN + (int)rank * BNL, tau);
            }
          }
        }
        if (!ok) break;
      }
      // Every issued stage must have landed before the pair may exit.  The
      // full barriers live in the even CTA and count the loads of both CTAs;
      // after an abort the two producers may have stopped at different
      // stages (at most S apart: a stage is issued only after the MMAs of
      // the stage S before it, which needed both CTAs' loads).  So the odd
      // producer reports how many stages it issued, and the even one settles
      // the difference: for a stage only the odd CTA issued it arrives with
      // the odd share's bytes, for a stage only it issued it counts the
      // missing odd share as complete; then it waits (bounded) on the full
      // barriers of the last S stages.  The odd CTA leaves only after the
      // teardown's cluster barrier, which the even CTA reaches after this.
      if (CG == 2 && !leader) {
        uint32_t slot;
        asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(slot)
                     : "r"(smem_u32((const void *)odd_issued)));
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(slot), "r"(it) : "memory");
        mbar_arrive_cluster_release(cluster_addr(pdone, 0));
      }
      if (leader) {
        Watch w2{abort_flag, p.st, globaltimer() + 100000000ull, p.sh.q, 1};
        volatile int zero = 0;
        w2.abort = &zero;
        uint32_t end = it;
        if (CG == 2 && mbar_wait(pdone, 0u, w2)) {
          asm volatile("fence.acq_rel.cluster;" ::: "memory");
          const uint32_t io = *odd_issued;
          const uint32_t half = stage_bytes;   // one CTA's share of a stage
          for (uint32_t j = it; j < io; ++j) mbar_expect_tx(&full[j % S], half);
          for (uint32_t j = io; j < it; ++j) mbar_complete_tx(&full[j % S], half);
          if (io > end) end = io;
        }
        for (uint32_t j = end > (uint32_t)S ? end - S : 0u; j < end; ++j)
          if (!mbar_wait(&full[j % S], (j / S) & 1u, w2)) break;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (the even CTA) ----------------
    if (lane == 0 && leader) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)T::AB << 7) | ((uint32_t)T::AB << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((BM * CG) >> 4) << 24);
      uint32_t it = 0, local = 0;
      const int KSP = p.ksplit, NB = p.nbuf;
      for (int t = t_first; t < t_end; t += t_step, ++local) {
        const int acc = NB == 2 ? (int)(local & 1) : 0;
        const uint32_t aph = NB == 2 ? (local >> 1) & 1u : local & 1u;
        if (!mbar_wait(&tempty[acc], aph ^ 1u, w)) break;
        tc_fence_after();
        const uint32_t dbuf = tmem_base + (uint32_t)(acc * BN * p.nacc);
        const uint32_t dcorr = dbuf + (uint32_t)(KSP * BN);   // used when csep
        bool ok = true;
        int seg_prev = -1;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1u;
          if (!mbar_wait(&full[s], ph, w)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t sb = sa + NP * a_bytes;
          // K segment of this stage (each segment has its own accumulator)
          const int seg = (kb * KSP) / kb_count;
          const bool seg_start = seg != seg_prev;
          seg_prev = seg;
          const uint32_t dt = dbuf + (uint32_t)(seg * BN);
          const bool cs = NP == 2 && p.csep != 0;
          const uint32_t dc = cs ? dcorr : dt;
#pragma unroll
          for (int j = 0; j < KSTEPS; ++j) {
            const uint32_t first = (seg_start && j == 0) ? 0u : 1u;
            const uint64_t a0 = sdesc(sa + 32 * j, ROWB);
            const uint64_t b0 = sdesc(sb + 32 * j, ROWB);
            mma<T::KIND, CG>(dt, a0, b0, idesc, first);
            if (NP == 2) {
              const uint64_t a1 = sdesc(sa + a_bytes + 32 * j, ROWB);
              const uint64_t b1 = sdesc(sb + b_bytes + 32 * j, ROWB);
              const uint32_t cfirst = cs ? ((kb == 0 && j == 0) ? 0u : 1u) : 1u;
              mma<T::KIND, CG>(dc, a0, b1, idesc, cfirst);
              mma<T::KIND, CG>(dc, a1, b0, idesc, 1u);
            }
          }
          if (CG == 1) mma_commit(&empty[s]);
          else mma_commit_cg2(&empty[s]);  // frees the stage in both CTAs
        }
        if (!ok) break;
        if (CG == 1) mma_commit(&tfull[acc]);
        else mma_commit_cg2(&tfull[acc]);   // both CTAs' epilogues may drain
      }
      // all issued MMAs retire before TMEM is released
      if (CG == 1) mma_commit(done);
      else mma_commit_cg2(done);
      Watch w2{abort_flag, p.st, globaltimer() + 100000000ull, p.sh.q, 1};
      volatile int zero = 0;
      w2.abort = &zero;
      mbar_wait(done, 0u, w2);
    }
  } else {
    // ---------------- epilogue (both CTAs) ----------------
    // Warp w drains TMEM lanes 32*(w%4) .. +31 (the rows it may access), all
    // columns of the tile, 16 at a time; the load of chunk c+1 is in flight
    // while chunk c is scaled, split and stored.
    const int quad = warp & 3;
    const int row = 32 * quad + lane;
    // EPI = 8: warps ew and ew + 4 share a quadrant and split its columns
    // (a 16-column tile stays with the first)
    const int ew = warp - 2;
    const bool split_cols = EPI == 8 && p.BN >= 32;
    const int c_begin = split_cols ? (ew >> 2) * (p.BN / 2) : 0;
    const bool idle = EPI == 8 && !split_cols && ew >= 4;
    const int c_end = idle ? 0 : (split_cols ? c_begin + p.BN / 2 : p.BN);
    const int dv = p.sh.dv_out, dh = p.sh.dh_out;
    const int64_t M = p.sh.M, P = p.sh.P;
    const int64_t Mr = p.sh.Mr > 0 ? p.sh.Mr : M;
    const int64_t MrN = Mr * (int64_t)p.sh.N, Mrdh = Mr * (int64_t)dh;
    const bool vbm = p.sh.vb != 0;
    uint32_t local = 0;
    int cached_item = -1;
    const OpDesc *op = nullptr;
    const StepItem *si = nullptr;
    float sc = 1.f;
    int x = 0, s_in = 0;
    for (int t = t_first; t < t_end; t += t_step, ++local) {
      const int item = (int)p.d_tpi.q(t);
      const int rem = t - item * tiles_per_item;
      int mg, nt;
      if (p.gm <= 1) {
        mg = (int)p.d_tn.q(rem);
        nt = rem - mg * p.tiles_n;
      } else {
        tile_of(rem, mgroups, p.tiles_n, p.gm, mg, nt);
      }
      const int mt = mg * CG + (int)rank;
      if (item != cached_item) {
        cached_item = item;
        si = &p.items[item];
        op = &p.ops[si->op_base + block_variant(*si->bits, p.sh)];
        const bool unit_in = si->in_rec < 0;
        const float mu = unit_in ? 1.f : __uint_as_float(p.recs[si->in_rec].maxbits);
        s_in = unit_in ? 0 : p.recs[si->in_rec].exp;
        // a fused dot keeps the accumulator unscaled (nothing is stored)
        x = p.sh.dot ? 0 : step_scale_exp(mu, __uint_as_float(op->beta_t_bits), p.sh.target);
        sc = pow2f(x);
      }
      const int acc = p.nbuf == 2 ? (int)(local & 1) : 0;
      const uint32_t aph = p.nbuf == 2 ? (local >> 1) & 1u : local & 1u;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&tfull[acc], aph, w) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      int64_t b, m_hi, m_lo;
      bool live;
      if (p.mhi) {
        // row = l ph + h: m_hi = hb0 + h, m_lo = mlo_t + l (the tile of the producer)
        const int64_t rest = p.d_hper.q(mt);
        m_hi = p.d_hper.r(mt) * p.ph + p.d_ph.r(row);
        b = p.d_lper.q(rest);
        m_lo = p.d_lper.r(rest) * p.lh + p.d_ph.q(row);
        live = true;
      } else {
        const int64_t m = (int64_t)mt * BM + row;
        live = m < M;
        // row m = b * Mr + m_r (b: the batch of open legs, when there is one)
        b = live ? p.d_Mr.q(m) : 0;
        const int64_t mr = live ? m - b * Mr : 0;
        m_hi = p.d_Mlo.q(mr);
        m_lo = p.d_Mlo.r(mr);
      }
      float vmax = 0.f;
      const int KSP = p.nacc;   // K segments, then the correction accumulator
      const uint32_t tbase =
          tmem_base + ((uint32_t)(32 * quad) << 16) + (uint32_t)(acc * BN * KSP);
      void *D = si->D;
      const bool dotm = p.sh.dot != 0;
      float dre = 0.f, dim = 0.f;   // fused dot: this row's partial sum
      // The columns in chunks of 16 (8 complex entries), the next chunk (or
      // pair) loaded from TMEM while the current one is used.
      uint32_t ra[16], rb[16];
      if (!idle) tmem_ld16_issue(tbase + (uint32_t)c_begin, ra);
      if (dotm) {
        // fused dot: the partner entries of row m (P = 1, row-major m N + n),
        // loaded one chunk ahead of their use
        const int64_t dot_e = m_lo * (int64_t)p.sh.N + ((nt * BN + c_begin) >> 1);
        Raw8 fcur, fnext;
        if (live && !idle) load8_raw<FMT>(D, dot_e, p.sh.plane, fcur);
        tmem_wait(ra);
        for (int c = c_begin; c < c_end; c += 16) {
          const bool more = c + 16 < c_end;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(ra[i]);
          if (more) tmem_ld16_issue(tbase + (uint32_t)(c + 16), ra);
          if (live && more) load8_raw<FMT>(D, dot_e + ((c + 16 - c_begin) >> 1), p.sh.plane, fnext);
          for (int sg = 1; sg < KSP; ++sg) {
            uint32_t rc[16];
            tmem_ld16_issue(tbase + (uint32_t)(sg * BN + c), rc);
            tmem_wait(rc);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += __uint_as_float(rc[i]);
          }
          if (live) {
            float2 f[8];
            unpack8<FMT>(fcur, f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              dre = fmaf(v[2 * j], f[j].x, fmaf(-v[2 * j + 1], f[j].y, dre));
              dim = fmaf(v[2 * j], f[j].y, fmaf(v[2 * j + 1], f[j].x, dim));
            }
            fcur = fnext;
          }
          if (more) tmem_wait(ra);
        }
      } else {
        // Destination of complex column nc of this row:
        //   base + q(nc) * stride_q + r(nc) * stride_r  (q, r: nc / R, nc % R)
        //   vb = 0:          n = h' dv' + v', entry b Mr N + ((m_lo dh' + h') P + m_hi) dv' + v'
        //   vb = 1, nvs = 0: n = h' dv' + v', entry (b dv' + v') Mr dh' + (m_lo dh' + h') P + m_hi
        //   vb = 1, nvs = 1: n = v' dh' + h', the same entry
        // Runs of consecutive nc with stride_r = 1 are contiguous: they are
        // stored W entries at a time (W = 8, 4, 2 dividing R), else one by one.
        const bool nvs = p.sh.nvs != 0;
        const Div &dR = vbm && nvs ? p.d_dh : p.d_dv;
        const int64_t base = !vbm ? b * MrN + (m_lo * dh * P + m_hi) * dv
                                  : b * dv * Mrdh + m_lo * dh * P + m_hi;
        const int64_t stride_q = !vbm ? P * dv : (nvs ? Mrdh : P);
        const int64_t stride_r = !vbm ? 1 : (nvs ? P : Mrdh);
        const int64_t R = dR.d;
        const int W = stride_r != 1 ? 1 : (R % 8 == 0 ? 8 : (R % 4 == 0 ? 4 : (R % 2 == 0 ? 2 : 1)));
        // chunk c (16 columns, 8 complex entries): scaled, rounded to the
        // storage format and stored in runs of W
        auto emit = [&](int c, const float (&o)[16]) {
          Packed8<FMT> w;
          vmax = fmaxf(vmax, pack8<FMT>(o, sc, w));
          const int nc0 = (nt * BN + c) >> 1;
          switch (W) {
            case 8:
              store_run<FMT, 8>(D, base + dR.q(nc0) * stride_q + dR.r(nc0), p.sh.plane, w, 0);
              break;
            case 4:
#pragma unroll
              for (int j = 0; j < 8; j += 4)
                store_run<FMT, 4>(D, base + dR.q(nc0 + j) * stride_q + dR.r(nc0 + j), p.sh.plane,
                                  w, j);
              break;
            case 2:
#pragma unroll
              for (int j = 0; j < 8; j += 2)
                store_run<FMT, 2>(D, base + dR.q(nc0 + j) * stride_q + dR.r(nc0 + j), p.sh.plane,
                                  w, j);
              break;
            default:
#pragma unroll
              for (int j = 0; j < 8; ++j)
                store_run<FMT, 1>(D, base + dR.q(nc0 + j) * stride_q + dR.r(nc0 + j) * stride_r,
                                  p.sh.plane, w, j);
          }
        };
        // the other K segments of chunk c, added with FP32 round-to-nearest
        auto add_segments = [&](int c, float (&o)[16]) {
          for (int sg = 1; sg < KSP; ++sg) {
            uint32_t rc[16];
            tmem_ld16_issue(tbase + (uint32_t)(sg * BN + c), rc);
            tmem_wait(rc);
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] += __uint_as_float(rc[i]);
          }
        };
        if (EPI == 4) {
          // two chunks per iteration (twice the independent work in flight);
          // the next pair's TMEM loads overlap this pair's arithmetic
          if (c_begin + 16 < c_end) tmem_ld16_issue(tbase + (uint32_t)(c_begin + 16), rb);
          tmem_wait(ra);
          for (int c = c_begin; c < c_end; c += 32) {
            const bool two = c + 16 < c_end;
            float o0[16], o1[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              o0[i] = __uint_as_float(ra[i]);
              o1[i] = __uint_as_float(rb[i]);
            }
            const bool more = c + 32 < c_end;
            if (more) {
              tmem_ld16_issue(tbase + (uint32_t)(c + 32), ra);
              if (c + 48 < c_end) tmem_ld16_issue(tbase + (uint32_t)(c + 48), rb);
            }
            add_segments(c, o0);
            if (two) add_segments(c + 16, o1);
            if (live) {
              emit(c, o0);
              if (two) emit(c + 16, o1);
            }
            if (more) tmem_wait(ra);
          }
        } else {
          // one chunk at a time (the register budget of eight epilogue warps),
          // one copy of the code in the loop (the instruction cache holds the
          // three roles' loops at once): chunk c is copied out of the load
          // registers, chunk c + 16 loads into them while c is used
          tmem_wait(ra);
          for (int c = c_begin; c < c_end; c += 16) {
            const bool more = c + 16 < c_end;
            float o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = __uint_as_float(ra[i]);
            if (more) tmem_ld16_issue(tbase + (uint32_t)(c + 16), ra);
            add_segments(c, o);
            if (live) emit(c, o);
            if (more) tmem_wait(ra);
          }
        }
      }
      tc_fence_before();
      if (CG == 1) {
        mbar_arrive(&tempty[acc]);
      } else {
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(tempty0 + (uint32_t)acc * 8u);
      }
      if (dotm) {
        // the warp's 32 rows summed in FP64, one slot per (tile, CTA, warp)
        double r = (double)dre, i = (double)dim;
        for (int o = 16; o > 0; o >>= 1) {
          r += __shfl_xor_sync(0xffffffffu, r, o);
          i += __shfl_xor_sync(0xffffffffu, i, o);
        }
        if (lane == 0)
          p.dot_partials[((int64_t)item * tiles_per_item + rem) * (CG * EPI) + (int)rank * EPI +
                         ew] = make_double2(r, i);
      } else {
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0) atomicMax(&p.recs[si->out_rec].maxbits, __float_as_uint(vmax));
      }
      if (mt == 0 && nt == 0 && warp == 2 && lane == 0) p.recs[si->out_rec].exp = s_in + op->b_t + x + op->e_c;
    }
  }

  // teardown: everyone done issuing; the last MMAs have retired (done
  // barrier) and the last loads have landed (full barriers) before the pair
  // releases TMEM and leaves.
  tc_fence_before();
  __syncthreads();
  if (CG > 1) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(p.tmem_cols));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(p.tmem_cols));
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &f, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  });
  return fn;
}

int esz_of(int fmt) { return fmt == FMT_TF32 ? 4 : 2; }
int np_of(int fmt) { return (fmt == FMT_BF16X2 || fmt == FMT_FP16X2) ? 2 : 1; }

// Bytes of K per pipeline stage (the swizzle width): 128 where the row
// length allows and nothing else is asked, else 64.
int rowb_for(int Kr, int esz, int want = 0) {
  const int bytes = Kr * esz;
  if (want != 64 && bytes % 128 == 0) return 128;
  if (bytes % 64 == 0) return 64;
  return 0;
}

}  // namespace

int tc_Kr_pad(int K) { return 2 * K; }

bool tc_tuning_valid(int kchunk, int cluster, int epi) {
  return (kchunk == 0 || kchunk == 64 || kchunk == 128) && (cluster >= 0 && cluster <= 2) &&
         (epi == 0 || epi == 4 || epi == 8);
}
int tc_Nr_pad(int N) { return 2 * N; }

bool tc_supports(const StepShape &sh, int fmt) {
  if (!(fmt == FMT_BF16 || fmt == FMT_FP16 || fmt == FMT_BF16X2 || fmt == FMT_FP16X2 ||
        fmt == FMT_TF32))
    return false;
  const int Kr = 2 * sh.K, Nr = 2 * sh.N;
  if (rowb_for(Kr, esz_of(fmt)) == 0) return false;
  // fewer rows than a tile: the A box reaches past the tensor's M extent,
  // where TMA fills zeros, and the epilogue stores live rows only
  if (sh.M < 32) return false;
  if (!(Nr % 256 == 0 || (Nr % 16 == 0 && Nr <= 256))) return false;
  if (sh.M > 0x7fffffffLL) return false;
  return true;
}

struct TcLaunchData {
  TcParams prm;
  int rowb;
  int cg;   // CTAs per MMA: 1, or 2 for the 2-SM UMMA
  int epi;  // epilogue warps: 4, or 8 where the epilogue bounds the step
};

int tc_prepare(const StepShape &sh, int fmt, const void *a_base, int a_lanes,
               int64_t a_lane_stride, int64_t plane_stride_bytes, const void *const b_base[2],
               int n_var, int64_t b_var_stride, int kchunk, int cluster, int epi,
               void **out_handle) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return -1;
  const int esz = esz_of(fmt), np = np_of(fmt);
  const int Kr = 2 * sh.K, Nr = 2 * sh.N;
  const int rowb = rowb_for(Kr, esz, kchunk);
  if (!rowb) return -2;
  auto *d = new TcLaunchData();
  std::memset(&d->prm, 0, sizeof(TcParams));
  d->rowb = rowb;
  const CUtensorMapDataType dt =
      esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  const CUtensorMapSwizzle sw =
      rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  // unused dimensions (one plane, one lane) get the packed stride
  const int64_t packed = (int64_t)Kr * esz * sh.M;
  // A step that stores its open bottom leg into the batch (vb) writes
  // (b dv' + v') Mr dh' + ((m_lo dh' + h') P + m_hi): contiguous in m_hi
  // only.  Its tiles then take ph = min(P, BM) consecutive m_hi by lh = BM / ph
  // consecutive m_lo at one b, through a 5-d map {k, m_hi, m_lo, b,
  // plane/lane} (the plane and the lane share a coordinate: lane * lp_mul +
  // plane), so that a warp's stores cover 32 consecutive entries.  The box
  // lands in shared memory as the usual 128 rows (row = l ph + h).
  bool mhi = false;
  int64_t lp_mul = 1, lp_stride = 0, lp_ext = 1;
  const int64_t ph = sh.P < BM ? sh.P : BM, lh = BM / (ph > 0 ? ph : 1);
  if (sh.vb && sh.nvs == 0 && sh.P >= 32 && (sh.P % BM == 0 || BM % sh.P == 0) && sh.Mr > 0 &&
      sh.Mr % sh.P == 0 && sh.M % sh.Mr == 0 && (sh.Mr / sh.P) % lh == 0) {
    if (np > 1) {
      if (a_lanes == 1) {
        mhi = true;
        lp_stride = plane_stride_bytes;
        lp_ext = np;
      } else if (plane_stride_bytes > 0 && a_lane_stride % plane_stride_bytes == 0) {
        mhi = true;
        lp_mul = a_lane_stride / plane_stride_bytes;
        lp_stride = plane_stride_bytes;
        lp_ext = (int64_t)(a_lanes - 1) * lp_mul + np;
      }
    } else {
      mhi = true;
      lp_stride = a_lanes > 1 ? a_lane_stride : packed;
      lp_ext = a_lanes;
    }
    if (lp_stride % 16 != 0) mhi = false;
  }
  if (mhi) {
    const int64_t Mlo = sh.Mr / sh.P, B = sh.M / sh.Mr;
    cuuint64_t dims[5] = {(cuuint64_t)Kr, (cuuint64_t)sh.P, (cuuint64_t)Mlo, (cuuint64_t)B,
                          (cuuint64_t)lp_ext};
    cuuint64_t strides[4] = {(cuuint64_t)(Mlo * Kr * esz), (cuuint64_t)Kr * esz,
                             (cuuint64_t)(sh.Mr * Kr * esz), (cuuint64_t)lp_stride};
    cuuint32_t box[5] = {(cuuint32_t)(rowb / esz), (cuuint32_t)ph, (cuuint32_t)lh, 1, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(&d->prm.mapA, dt, 5, const_cast<void *>(a_base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      delete d;
      return -3;
    }
    d->prm.mhi = 1;
    d->prm.lp_mul = (int)lp_mul;
    d->prm.ph = (int)ph;
    d->prm.lh = (int)lh;
    d->prm.mlo = Mlo;
  } else {
    cuuint64_t dims[4] = {(cuuint64_t)Kr, (cuuint64_t)sh.M, (cuuint64_t)np,
                          (cuuint64_t)a_lanes};
    const int64_t plane_st = np > 1 ? plane_stride_bytes : packed;
    const int64_t lane_st = a_lanes > 1 ? a_lane_stride : plane_st * np;
    cuuint64_t strides[3] = {(cuuint64_t)Kr * esz, (cuuint64_t)((plane_st + 15) / 16 * 16),
                             (cuuint64_t)((lane_st + 15) / 16 * 16)};
    cuuint32_t box[4] = {(cuuint32_t)(rowb / esz), (cuuint32_t)BM, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(&d->prm.mapA, dt, 4, const_cast<void *>(a_base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      delete d;
      return -3;
    }
  }
  // K segments (long-K steps): at most one per k-chunk, and BN small enough
  // that KS accumulators are double-buffered within TMEM's 512 columns
  const int kb_count = (Kr * esz) / rowb;
  int KS = sh.ksplit > 1 ? sh.ksplit : 1;
  if (KS > kb_count) KS = kb_count;
  const int CS = (sh.csep && np == 2) ? 1 : 0;
  const int NA = KS + CS;
  // BN: the widest tile whose NA accumulators fit TMEM (double-buffered when
  // they fit twice)
  int BN = Nr >= 256 ? 256 : Nr;
  while (BN > 16 && NA * BN > 512) BN /= 2;
  // a short K (at most 16 k-chunks) needs the epilogue overlap of two buffers
  if (kb_count <= 16)
    while (BN > 16 && 2 * NA * BN > 512) BN /= 2;
  const int tiles_m = (int)((sh.M + BM - 1) / BM);
  // The 2-SM UMMA when the 128-row tiles pair up and each CTA's half of the
  // Bt tile is a whole number of 8-row swizzle groups.
  d->cg = ((BN / 2) % 8 == 0 && tiles_m % 2 == 0 && cluster != 1) ? 2 : 1;
  // B: one map per plane over every operand variant {k, n, variant}; the
  // variants are equally spaced (a single variant gets the packed stride)
  const int64_t bpacked = (int64_t)Kr * esz * Nr;
  const int64_t vstride = n_var > 1 ? b_var_stride : bpacked;
  if (n_var < 1 || n_var > 64 || vstride < bpacked || vstride % 16 != 0) {
    delete d;
    return -6;
  }
  for (int pl = 0; pl < np; ++pl) {
    cuuint64_t dims[3] = {(cuuint64_t)Kr, (cuuint64_t)Nr, (cuuint64_t)n_var};
    cuuint64_t strides[2] = {(cuuint64_t)Kr * esz, (cuuint64_t)vstride};
    cuuint32_t box[3] = {(cuuint32_t)(rowb / esz), (cuuint32_t)(BN / d->cg), 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&d->prm.mapB[pl], dt, 3, const_cast<void *>(b_base[pl]), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      delete d;
      return -4;
    }
  }
  d->prm.sh = sh;
  d->prm.BN = BN;
  d->prm.tiles_m = (int)((sh.M + BM - 1) / BM);
  d->prm.tiles_n = Nr / BN;
  // wide launches (the merges): 8 row groups at a time, so that concurrent
  // tiles reuse both operands' k-slabs from L2 instead of streaming one B
  // column panel per tile
  {
    const int mgroups = d->prm.tiles_m / d->cg;
    d->prm.gm = (d->prm.tiles_n >= 32 && mgroups >= 16) ? 8 : 1;
    // outside the grouped order a pair walks consecutive tiles
    d->prm.blocked = d->prm.gm == 1 ? 1 : 0;
    d->prm.d_tpi = make_div((int64_t)mgroups * d->prm.tiles_n);
    d->prm.d_tn = make_div(d->prm.tiles_n);
  }
  {
    const int64_t Mr = sh.Mr > 0 ? sh.Mr : sh.M, P = sh.P > 0 ? sh.P : 1;
    d->prm.d_Mr = make_div(Mr);
    d->prm.d_Mlo = make_div(Mr / P);
    d->prm.d_dv = make_div(sh.dv_out);
    d->prm.d_dh = make_div(sh.dh_out);
    const int ph = d->prm.mhi ? d->prm.ph : 1, lh = d->prm.mhi ? d->prm.lh : 1;
    d->prm.d_ph = make_div(ph);
    d->prm.d_hper = make_div(d->prm.mhi ? P / ph : 1);
    d->prm.d_lper = make_div(d->prm.mhi ? d->prm.mlo / lh : 1);
  }
  d->prm.ksplit = KS;
  d->prm.csep = CS;
  d->prm.nacc = NA;
  d->prm.nbuf = 2 * BN * NA <= 512 ? 2 : 1;
  int cols = 32;
  while (cols < d->prm.nbuf * BN * NA) cols *= 2;
  d->prm.tmem_cols = cols;
  const int stage_bytes = np * (BM + BN / d->cg) * rowb;  // this CTA's share
  // 227 KiB per CTA, less the 1 KiB alignment pad and the barriers
  const int budget = 227 * 1024 - 1024 - 256;
  int stages = budget / stage_bytes;
  if (stages > 8) stages = 8;
  d->prm.stages = stages;
  // Epilogue warps (measured on the square partition's steps): four where
  // wide tiles store runs of 8 entries (each warp keeps two chunks in
  // flight), eight where the stores go out 1 to 4 entries at a time, where
  // nothing is stored (the fused dot) and on narrower tiles
  const bool runs8 = !sh.dot && ((!sh.vb && sh.dv_out % 8 == 0) ||
                                 (sh.vb && sh.nvs && sh.P == 1 && sh.dh_out % 8 == 0));
  d->epi = epi == 4 || epi == 8 ? epi : ((runs8 && BN >= 256) ? 4 : 8);
  *out_handle = d;
  return stages >= 2 ? 0 : -5;
}

void tc_release(void *h) { delete (TcLaunchData *)h; }

template <int FMT, int ROWB, int CG, int EPI>
static int &max_clusters_of() {
  static int v = -1;  // co-resident clusters at the largest smem size (-1: not set up)
  return v;
}

template <int FMT, int ROWB, int CG, int EPI>
static cudaError_t init_kernel() {
  auto kern = k_contract_tc<FMT, ROWB, CG, EPI>;
  int &max_clusters = max_clusters_of<FMT, ROWB, CG, EPI>();
  if (max_clusters < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t q = {};
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = CG;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.gridDim = dim3(CG * 64);
    q.blockDim = dim3(threads_of(EPI));
    q.dynamicSmemBytes = 227 * 1024;
    q.attrs = qa;
    q.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, (void *)kern, &q);
    if (e != cudaSuccess || n <= 0) {
      (void)cudaGetLastError();
      n = 0;
    }
    max_clusters = n;
  }
  return cudaSuccess;
}

template <int FMT, int ROWB, int CG, int EPI>
static cudaError_t launch_one(const TcParams &prm, int units, size_t smem, cudaStream_t s) {
  auto kern = k_contract_tc<FMT, ROWB, CG, EPI>;
  cudaError_t e0 = init_kernel<FMT, ROWB, CG, EPI>();
  if (e0 != cudaSuccess) return e0;
  const int max_clusters = max_clusters_of<FMT, ROWB, CG, EPI>();
  // units = SMs to use; one CTA per SM, clusters of CG
  int clusters = units / CG;
  if (max_clusters > 0 && clusters > max_clusters) clusters = max_clusters;
  if (clusters < 1) clusters = 1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CG;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(clusters * CG);
  cfg.blockDim = dim3(threads_of(EPI));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, prm);
}

template <int FMT, int EPI>
static cudaError_t warm_epi(int rowb, int cg) {
  if (rowb == 128)
    return cg == 2 ? init_kernel<FMT, 128, 2, EPI>() : init_kernel<FMT, 128, 1, EPI>();
  return cg == 2 ? init_kernel<FMT, 64, 2, EPI>() : init_kernel<FMT, 64, 1, EPI>();
}
template <int FMT>
static cudaError_t warm_fmt(int rowb, int cg, int epi) {
  return epi == 8 ? warm_epi<FMT, 8>(rowb, cg) : warm_epi<FMT, 4>(rowb, cg);
}

cudaError_t tc_warm(void *handle) {
  TcLaunchData *d = (TcLaunchData *)handle;
  switch (d->prm.sh.fmt) {
    case FMT_BF16: return warm_fmt<FMT_BF16>(d->rowb, d->cg, d->epi);
    case FMT_FP16: return warm_fmt<FMT_FP16>(d->rowb, d->cg, d->epi);
    case FMT_BF16X2: return warm_fmt<FMT_BF16X2>(d->rowb, d->cg, d->epi);
    case FMT_FP16X2: return warm_fmt<FMT_FP16X2>(d->rowb, d->cg, d->epi);
    case FMT_TF32: return warm_fmt<FMT_TF32>(d->rowb, d->cg, d->epi);
  }
  return cudaErrorInvalidValue;
}

template <int FMT, int EPI>
static cudaError_t launch_epi(const TcParams &prm, int rowb, int cg, int units, size_t smem,
                              cudaStream_t s) {
  if (rowb == 128)
    return cg == 2 ? launch_one<FMT, 128, 2, EPI>(prm, units, smem, s)
                   : launch_one<FMT, 128, 1, EPI>(prm, units, smem, s);
  return cg == 2 ? launch_one<FMT, 64, 2, EPI>(prm, units, smem, s)
                 : launch_one<FMT, 64, 1, EPI>(prm, units, smem, s);
}
template <int FMT>
static cudaError_t launch_fmt(const TcParams &prm, int rowb, int cg, int epi, int units,
                              size_t smem, cudaStream_t s) {
  return epi == 8 ? launch_epi<FMT, 8>(prm, rowb, cg, units, smem, s)
                  : launch_epi<FMT, 4>(prm, rowb, cg, units, smem, s);
}

int tc_dot_slots(const void *handle) {
  const TcLaunchData *d = (const TcLaunchData *)handle;
  return d->prm.tiles_m * d->prm.tiles_n * d->epi;
}

cudaError_t launch_contract_tc(void *handle, const StepItem *d_items, int n_items,
                               const OpDesc *d_ops, Rec *d_recs, DeviceStatus *st,
                               int64_t watchdog_ns, int sm_count, cudaStream_t s,
                               double2 *dot_partials) {
  TcLaunchData *d = (TcLaunchData *)handle;
  TcParams prm = d->prm;
  prm.dot_partials = dot_partials;
  if (prm.sh.dot && !dot_partials) return cudaErrorInvalidValue;
  prm.items = d_items;
  prm.n_items = n_items;
  prm.ops = d_ops;
  prm.recs = d_recs;
  prm.st = st;
  prm.watchdog_ns = watchdog_ns;
  const int cg = d->cg;
  const int pair_tiles = n_items * (prm.tiles_m / cg) * prm.tiles_n;
  if (pair_tiles < 1) return cudaSuccess;
  const int units = pair_tiles * cg < sm_count ? pair_tiles * cg : sm_count;
  const int np = np_of(prm.sh.fmt);
  const size_t smem = (size_t)prm.stages * np * (BM + prm.BN / cg) * d->rowb + 1024 +
                      (2 * prm.stages + 6) * 8 + 16;
  switch (prm.sh.fmt) {
    case FMT_BF16: return launch_fmt<FMT_BF16>(prm, d->rowb, cg, d->epi, units, smem, s);
    case FMT_FP16: return launch_fmt<FMT_FP16>(prm, d->rowb, cg, d->epi, units, smem, s);
    case FMT_BF16X2: return launch_fmt<FMT_BF16X2>(prm, d->rowb, cg, d->epi, units, smem, s);
    case FMT_FP16X2: return launch_fmt<FMT_FP16X2>(prm, d->rowb, cg, d->epi, units, smem, s);
    case FMT_TF32: return launch_fmt<FMT_TF32>(prm, d->rowb, cg, d->epi, units, smem, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Tensor-core operand build: the real embedding of E (scaled by 2^b_t), split
// into the form's planes, K-major [Nr][Kr].  Also the bound beta_t.
// ---------------------------------------------------------------------------
template <int FMT>
__global__ void __launch_bounds__(256) k_build_bt(OpDesc *ops) {
  OpDesc &op = ops[blockIdx.y];
  if (op.Bt[0] == nullptr) return;
  const int K = op.K, N = op.N;
  const float sc = ldexpf(1.f, op.b_t);
  // 32 x 32 complex tiles of Ec through shared memory: read along n, written
  // along k, two real columns (a = 0, 1 of one k) per store
  __shared__ float2 tile[32][33];
  const int tn = (N + 31) / 32, n_tiles = ((K + 31) / 32) * tn;
  const int64_t Kr = 2 * (int64_t)K;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int k0 = (t / tn) * 32, n0 = (t % tn) * 32;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int kk = e >> 5, nn = e & 31;
      tile[kk][nn] = (k0 + kk < K && n0 + nn < N) ? op.Ec[(int64_t)(k0 + kk) * N + n0 + nn]
                                                    : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int kk = threadIdx.x & 31, k = k0 + kk;
    for (int r = threadIdx.x >> 5; r < 64; r += blockDim.x >> 5) {
      const int nn = r >> 1, b = r & 1, n = n0 + nn;
      if (k >= K || n >= N) continue;
      // row 2n holds (re, -im) at columns 2k, 2k+1; row 2n+1 holds (im, re)
      const float2 e = tile[kk][nn];
      const float v0 = (b == 0 ? e.x : e.y) * sc, v1 = (b == 0 ? -e.y : e.x) * sc;
      const int64_t w = ((int64_t)(2 * n + b) * Kr + 2 * (int64_t)k) >> 1;   // in column pairs
      if (FMT == FMT_TF32) {
        ((float2 *)op.Bt[0])[w] = make_float2(round_tf32(v0), round_tf32(v1));
      } else if (FMT == FMT_BF16) {
        ((uint32_t *)op.Bt[0])[w] = pack_bf16(v0, v1);
      } else if (FMT == FMT_FP16) {
        ((uint32_t *)op.Bt[0])[w] = pack_f16(v0, v1);
      } else {
        constexpr bool BF = FMT == FMT_BF16X2;
        uint32_t h, l;
        split16<BF>(make_float2(v0, v1), h, l);
        ((uint32_t *)op.Bt[0])[w] = h;
        ((uint32_t *)op.Bt[1])[w] = l;
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // beta_t = beta_c * 2^b_t (beta_c already carries a rounding margin; the
    // rounded planes differ from the scaled values by at most 2^-8 relative)
    const float bc = __uint_as_float(op.beta_c_bits);
    op.beta_t_bits = __float_as_uint(bc * sc * (1.0f + 1.0f / 128.0f));
  }
}

// A merge operand straight from a stored tensor G whose k index is contiguous:
// Ec[k][n] = G[k + nh ns_hi + nl ns] 2^-target (n = nh Nlo + nl) is never
// written out.  k_tensor_bound takes the column bound beta_c = max_n
// sum_k |Ec[k][n]|_1 (one block per column, the threads along k), k_tensor_bt
// the complex-as-real planes Bt[(n, b)][(k, a)] (reads and writes both run
// along k).  Same values as Ec -> k_beta_ops -> k_build_bt.
__global__ void k_tensor_init(const TensorOpEntry *__restrict__ e, int n, OpDesc *ops,
                              const Rec *recs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const TensorOpEntry g = e[i];
  OpDesc &op = ops[g.op];
  op.beta_c_bits = 0u;
  op.beta_t_bits = 0u;
  op.e_c = recs[g.rec].exp - g.target;
}

template <int FMT>
__global__ void __launch_bounds__(256) k_tensor_bound(const TensorOpEntry *__restrict__ e,
                                                      int64_t plane, OpDesc *ops) {
  const TensorOpEntry g = e[blockIdx.y];   // one entry per grid row
  const float sc = pow2f(-g.target);
  __shared__ float red[8];
  float best = 0.f;
  for (int64_t n = blockIdx.x; n < g.N; n += gridDim.x) {
    const int64_t nh = n / g.Nlo, nl = n - nh * g.Nlo;
    const int64_t base = nh * g.ns_hi + nl * g.ns;
    float s = 0.f;
    for (int64_t k = threadIdx.x; k < g.K; k += blockDim.x) {
      const float2 v = load_g<FMT>(g.G, base + k * g.ks, plane);
      s += fabsf(v.x * sc) + fabsf(v.y * sc);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < 8; ++w) t += red[w];
      best = fmaxf(best, t);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    atomicMax(&ops[g.op].beta_c_bits, __float_as_uint(best * (1.0f + 1.0f / 256.0f)));
}

template <int FMT>
__global__ void k_tensor_bt(const TensorOpEntry *__restrict__ e, int64_t plane, OpDesc *ops) {
  const TensorOpEntry g = e[blockIdx.y];   // one entry per grid row
  OpDesc &op = ops[g.op];
  const int64_t K = g.K, N = g.N;
  const float sc = pow2f(-g.target), sb = ldexpf(1.f, op.b_t);
  const bool narrow = K * N < ((int64_t)1 << 31) && g.Nlo < ((int64_t)1 << 31);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t n, k, nh, nl;
    if (narrow) {   // 32-bit index arithmetic
      const uint32_t i32 = (uint32_t)i, n32 = i32 / (uint32_t)K, lo = (uint32_t)g.Nlo;
      n = n32;
      k = i32 - n32 * (uint32_t)K;
      nh = n32 / lo;
      nl = n32 - (uint32_t)nh * lo;
    } else {
      n = i / K;
      k = i - n * K;
      nh = n / g.Nlo;
      nl = n - nh * g.Nlo;
    }
    const float2 v = load_g<FMT>(g.G, k * g.ks + nh * g.ns_hi + nl * g.ns, plane);
    const float re = (v.x * sc) * sb, im = (v.y * sc) * sb;
    // row 2n holds (re, -im) at columns 2k, 2k+1; row 2n+1 holds (im, re)
    const float2 r0 = make_float2(re, -im), r1 = make_float2(im, re);
    const int64_t w0 = 2 * n * K + k, w1 = (2 * n + 1) * K + k;   // in column pairs
    if (FMT == FMT_TF32) {
      ((float2 *)op.Bt[0])[w0] = make_float2(round_tf32(r0.x), round_tf32(r0.y));
      ((float2 *)op.Bt[0])[w1] = make_float2(round_tf32(r1.x), round_tf32(r1.y));
    } else if (FMT == FMT_BF16) {
      ((uint32_t *)op.Bt[0])[w0] = pack_bf16(r0.x, r0.y);
      ((uint32_t *)op.Bt[0])[w1] = pack_bf16(r1.x, r1.y);
    } else if (FMT == FMT_FP16) {
      ((uint32_t *)op.Bt[0])[w0] = pack_f16(r0.x, r0.y);
      ((uint32_t *)op.Bt[0])[w1] = pack_f16(r1.x, r1.y);
    } else {
      constexpr bool BF = FMT == FMT_BF16X2;
      uint32_t h0, l0, h1, l1;
      split16<BF>(r0, h0, l0);
      split16<BF>(r1, h1, l1);
      ((uint32_t *)op.Bt[0])[w0] = h0;
      ((uint32_t *)op.Bt[0])[w1] = h1;
      ((uint32_t *)op.Bt[1])[w0] = l0;
      ((uint32_t *)op.Bt[1])[w1] = l1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const float bc = __uint_as_float(op.beta_c_bits);
    op.beta_t_bits = __float_as_uint(bc * sb * (1.0f + 1.0f / 128.0f));
  }
}

cudaError_t launch_tensor_operand_tc(const TensorOpEntry *d_entry, int n_entries, int K, int N,
                                     int fmt, int64_t plane, OpDesc *d_ops, const Rec *d_recs,
                                     cudaStream_t s) {
  if (n_entries <= 0) return cudaSuccess;
  const int64_t kn = (int64_t)K * N;
  int64_t gb = N < 16384 ? N : 16384;
  if (gb < 1) gb = 1;
  int64_t gt = (kn + 255) / 256;
  if (gt > 16384) gt = 16384;
  if (gt < 1) gt = 1;
  k_tensor_init<<<(n_entries + 127) / 128, 128, 0, s>>>(d_entry, n_entries, d_ops, d_recs);
  const dim3 grid_b((unsigned)gb, (unsigned)n_entries), grid_t((unsigned)gt, (unsigned)n_entries);
  switch (fmt) {
#define PEPS_TOP_CASE(F)                                                              \
  case F:                                                                            \
    k_tensor_bound<F><<<grid_b, 256, 0, s>>>(d_entry, plane, d_ops);                 \
    k_tensor_bt<F><<<grid_t, 256, 0, s>>>(d_entry, plane, d_ops);                    \
    break;
    PEPS_TOP_CASE(FMT_TF32)
    PEPS_TOP_CASE(FMT_BF16)
    PEPS_TOP_CASE(FMT_FP16)
    PEPS_TOP_CASE(FMT_BF16X2)
    PEPS_TOP_CASE(FMT_FP16X2)
#undef PEPS_TOP_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_tc_operands(int n, int64_t max_kn, OpDesc *d_ops, int fmt,
                                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  // 32 x 32 tiles of the largest operand (ops with fewer tiles leave early)
  int64_t blocks = (max_kn + 1023) / 1024 + 2;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  dim3 grid(blocks, n);
  switch (fmt) {
    case FMT_TF32: k_build_bt<FMT_TF32><<<grid, 256, 0, s>>>(d_ops); break;
    case FMT_BF16: k_build_bt<FMT_BF16><<<grid, 256, 0, s>>>(d_ops); break;
    case FMT_FP16: k_build_bt<FMT_FP16><<<grid, 256, 0, s>>>(d_ops); break;
    case FMT_BF16X2: k_build_bt<FMT_BF16X2><<<grid, 256, 0, s>>>(d_ops); break;
    case FMT_FP16X2: k_build_bt<FMT_FP16X2><<<grid, 256, 0, s>>>(d_ops); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace peps
