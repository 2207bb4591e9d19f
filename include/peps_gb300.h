/*
 * peps_gb300.h -- C ABI of the GB300 (sm_103a) PEPS amplitude engine.
 *
 * Computes exact output amplitudes <x| C |0...0> of circuits on an R x C
 * qubit lattice whose gates are single-qubit gates and nearest-neighbour CZ
 * gates.  The state is held as an untruncated PEPS (paper, main text: the PEPS
 * equation, single-qubit absorption "onebody", two-qubit split "factorize" and
 * bundling "twoqubita/b"); each amplitude is obtained by projecting every site
 * on its output bit (main text, "overlap") and contracting the network
 * exactly, column by column (supplementary "exact computation of the
 * overlap", generic scheme, transposed to sweep columns left to right).
 *
 * Conventions shared by every call:
 *  - qubit index q = r*C + c, 0 <= r < R, 0 <= c < C, R*C <= 64;
 *  - bit q of a uint64 bitstring is the output bit of qubit q;
 *  - a 2x2 gate matrix U is row-major, U[tau*2 + sigma] = <tau|U|sigma>;
 *  - CZ on an edge is split exactly as P_0 (x) I + P_1 (x) Z; the projector
 *    factor goes on the site with the lower q; the new Schmidt bit s is the
 *    least significant bit of the grown bond index (new = old*2 + s) on both
 *    sites, so the k-th CZ applied to an edge owns bit (n_cz - 1 - k).
 *
 * Memory: the library never allocates device memory.  Every call that touches
 * the GPU takes a caller-owned device workspace (size from
 * peps_workspace_bytes) and a cudaStream_t passed as void*.  Host pointers
 * stay owned by the caller and are not retained after a call returns.
 *
 * Errors: every function returns a peps_status.  On failure the outputs are
 * left untouched and peps_last_error() returns a text for the calling thread.
 * A device-side watchdog expiry returns PEPS_ETIMEOUT and marks the context
 * PEPS_ESTATE until it is destroyed.
 *
 * Thread safety: a context may be used by one thread at a time.
 */
#ifndef PEPS_GB300_H
#define PEPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PEPS_API __attribute__((visibility("default")))
#else
#define PEPS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct peps_ctx peps_ctx;

typedef struct {
    double re, im;
} peps_c128;

typedef enum {
    PEPS_OK = 0,
    PEPS_EINVAL = -1,       /* bad argument (range, null, size)              */
    PEPS_ENOTADJ = -2,      /* CZ on qubits that are not lattice neighbours  */
    PEPS_ENOMEM = -3,       /* workspace smaller than peps_workspace_bytes   */
    PEPS_ECUDA = -4,        /* a CUDA runtime/driver call failed             */
    PEPS_ETIMEOUT = -5,     /* a device wait exceeded the watchdog budget    */
    PEPS_ESTATE = -6,       /* context unusable after an earlier failure     */
    PEPS_EUNSUPPORTED = -7  /* valid request this library cannot run         */
} peps_status;

/* Arithmetic of the column-absorption contraction (the other kernels are
 * FP32 complex; the final reduction is FP64).  Storage of the running tensor
 * G between absorptions follows the form:
 *   FP32_SIMT  fp32 complex, CUDA-core FMA                     (8 B / entry)
 *   TF32       tcgen05 kind::tf32, G stored fp32 rounded to TF32 (8 B)
 *   BF16       tcgen05 kind::f16 (bf16 inputs), G stored bf16   (4 B)
 *   BF16X3     bf16 hi/lo split of G and of the site operand, three
 *              products hi*hi + hi*lo + lo*hi                    (8 B)
 *   FP16       tcgen05 kind::f16 (fp16 inputs), G stored fp16   (4 B)
 *   FP16X3     fp16 hi/lo split, three products, G held in range by the
 *              per-step power-of-two scaling                    (8 B)
 * All tensor-core forms accumulate in FP32. */
typedef enum {
    PEPS_FP32_SIMT = 0,
    PEPS_TF32 = 1,
    PEPS_BF16 = 2,
    PEPS_BF16X3 = 3,
    PEPS_FP16 = 4,
    PEPS_FP16X3 = 5,
    PEPS_N_PRECISIONS = 6
} peps_precision;

enum {
    PEPS_FLAG_REBUILD = 1,  /* re-run the circuit evolution even if unchanged */
    PEPS_FLAG_TIMING = 2,   /* time every contraction launch with CUDA events */
    PEPS_FLAG_NO_TC = 4,    /* run every absorption on the CUDA-core kernel   */
    PEPS_FLAG_GRAPH = 8,    /* capture the call's launch sequence (evolution
                               included) into a CUDA graph on the first call
                               and replay it on later calls with the same
                               plan; with PEPS_FLAG_TIMING a second graph
                               that also records the events around its
                               contraction launches (captured on its first
                               use) is replayed, and reports their times */
    PEPS_FLAG_MARGINALS = 16, /* return marginal probabilities P(x_S) =
                               <psi| Pi_S |psi> instead of amplitudes: S = the
                               set bits of opts.measured_mask, their values
                               from each bitstring; the other qubits are summed
                               over.  Computed as the double-layer network
                               (every site sum_sigma A^sigma (x) conj(A^sigma),
                               every bond squared); out[i].re = P, .im ~ 0.
                               Not with slicing or held CZ bits.          */
    PEPS_FLAG_ESTIMATE = 32,/* planning only: peps_plan_info_get and
                               peps_workspace_bytes report the figures of a
                               plan whose running tensor exceeds the 2^36
                               entries an amplitude call accepts (a slice-set
                               search starts there); an amplitude call with
                               this flag returns PEPS_EINVAL.              */
    PEPS_FLAG_STEPWISE = 128,/* one launch per absorption step and per gate
                               batch even where a small lattice's whole
                               column sweep fits one block's shared memory
                               (where it does, and the form is FP32 or a
                               split form, the sweeps of all bitstrings run
                               as one persistent launch in FP32, and the
                               evolution of small site tensors as one launch
                               with a block per site)                       */
    PEPS_FLAG_HOLD_TIES = 64 /* hold every CZ Schmidt bit that the output
                               bitstring (or the initial state) fixes, and
                               tie every linked bit to its source bit, as
                               peps_output_ties lists them: the bond index
                               takes only the values these ties allow in each
                               bitstring's contraction, which halves the bond
                               per tied bit for the whole sweep.  Exact: every
                               dropped term of the bond sum is zero.  Each site operand
                               then has a variant per value of the output bits
                               it depends on (its own and those of the
                               neighbours whose projector bits touch its
                               legs).  Not with slicing, held CZ bits
                               (n_fixed) or marginals (PEPS_EINVAL).        */
};

/* Options of an amplitude call.  All-zero means: FP32_SIMT, no prefix reuse,
 * lanes chosen from the workspace, no slicing, default watchdog. */
typedef struct {
    int32_t precision;        /* peps_precision                               */
    int32_t flags;            /* PEPS_FLAG_*                                  */
    int32_t prefix_cols;      /* >0: bitstrings are in groups of prefix_group
                                 consecutive entries that share the bits of
                                 every qubit in columns < prefix_cols; the
                                 running tensor after those columns is
                                 computed once per group (checked on device;
                                 a violating group gives PEPS_EINVAL)          */
    int32_t prefix_group;     /* group size for prefix_cols (>= 1)            */
    int32_t max_lanes;        /* bitstrings contracted concurrently; 0 = as
                                 many as the workspace holds (<= 64)          */
    int32_t n_sliced;         /* number of sliced CZ gates                    */
    const uint32_t *sliced_cz;/* ordinals (0 = first CZ applied) of the CZ
                                 gates whose Schmidt bit is fixed per slice   */
    const uint64_t *slice_ids;/* slices to sum: bit j = fixed s of
                                 sliced_cz[j]; NULL = all 2^n_sliced          */
    int64_t n_slice_ids;
    int64_t watchdog_ns;      /* device wait budget; 0 = 2 s                  */
    int32_t n_fixed;          /* CZ gates whose Schmidt bit is held at one
                                 value in every slice of the call (evaluates a
                                 sub-slice: a slice with more bits fixed)     */
    int32_t tc_ksplit;        /* tensor cores: accumulate K in this many
                                 segments (separate FP32 accumulators summed
                                 with round-to-nearest).  0 = automatic: the
                                 split forms give their hi*lo and lo*hi products
                                 an accumulator of their own on steps with K >=
                                 2048 real, and on every step of a chain longer
                                 than 32 steps; 1 = one accumulator; 2-4 = that
                                 many K segments; -1 = separate corrections on
                                 every step (the last three for measurement) */
    const uint32_t *fixed_cz; /* their ordinals (disjoint from sliced_cz)     */
    const uint8_t *fixed_s;   /* their values, 0 or 1                         */
    int32_t tc_kchunk;        /* tensor-core tuning: bytes of K per pipeline
                                 stage, 64 or 128 (0 = 128 where the row
                                 length allows); smaller means more stages  */
    int32_t tc_cluster;       /* tensor-core tuning: 2 = CTA pairs compute
                                 256-row tiles with the 2-SM MMA, 1 = one CTA
                                 per 128-row tile (0 = pairs where the row
                                 tiles pair up)                              */
    int32_t fuse_rows;        /* contraction order: 0 = absorb the two top and
                                 the two bottom rows of a column in one step
                                 each where that costs no more multiply-adds
                                 (the running tensor between them is never
                                 stored); 1 = one site per step              */
    int32_t scheme;           /* PEPS_SCHEME_*: the contraction scheme        */
    uint64_t measured_mask;   /* with PEPS_FLAG_MARGINALS: bit q set = qubit q
                                 is measured                                 */
    int32_t tc_epi;           /* tensor-core tuning: epilogue warps per CTA, 4
                                 (one per accumulator lane quadrant) or 8 (two,
                                 each draining half of a tile's columns); 0 =
                                 8 on steps of at most 16 K stages per tile,
                                 where the epilogue outlasts the MMAs, else 4 */
    int32_t pad_;
} peps_opts;

/* Contraction schemes (supplementary, "exact contraction"):
 *   COLUMNS   the generic scheme of Fig. S2(a), transposed: one running
 *             tensor absorbs the lattice column by column (any R x C);
 *   QUADRANTS the square partition of Fig. S2(b) (even R and C): each
 *             quarter is contracted from its lattice corner into one tensor
 *             holding the legs it shares with the other quarters; then the
 *             left half F_l = F_ul F_bl (once per prefix group when
 *             prefix_cols = C/2), Y = F_br F_l^T per bitstring, and the
 *             amplitude = sum Y * F_ur.  prefix_cols must be 0 or C/2. */
enum {
    PEPS_SCHEME_COLUMNS = 0,
    PEPS_SCHEME_QUADRANTS = 1
};

/* Counters of the last amplitude call (kernel launches are the library's own
 * kernels; times are CUDA-event times on the call's stream). */
typedef struct {
    int64_t launches_total;
    int64_t launches_evolve;     /* K1/K2: gate absorption                   */
    int64_t launches_operand;    /* K3: projection + operand build           */
    int64_t launches_contract;   /* K4: column absorption (all forms)        */
    int64_t launches_contract_tc;/* of which tcgen05 kernels                 */
    int64_t launches_finalize;   /* K6 (+checks)                             */
    double contract_flops;       /* algorithmic real flops of K4 (8/cMAC)    */
    double contract_bytes;       /* algorithmic bytes of K4 (read G + write G') */
    double contract_ms;          /* summed event time of K4 launches (TIMING) */
    double contract_tc_ms;       /* of which tcgen05 launches                */
    double contract_tc_flops;
    double contract_tc_bytes;
    int64_t n_steps;             /* site absorptions per lane chain           */
    int64_t n_lanes;             /* lanes used                                */
} peps_stats;

/* Create an empty circuit on an R x C lattice: the state |0...0> as a PEPS of
 * rank-5 site tensors A_q^sigma[l, r, u, d] with every auxiliary leg of
 * dimension 1, A^0 = 1 and A^1 = 0 (paper, main text: the PEPS equation for
 * the state as a product of site tensors summed over shared legs).  Host-only:
 * no GPU work, no device memory; the workspace and the stream are arguments
 * of the calls that run on the GPU.  R, C >= 1, R*C <= 64; *out receives the
 * context (owned by the caller until peps_destroy).  PEPS_EINVAL on a bad
 * size or a NULL out. */
PEPS_API int peps_create(int R, int C, peps_ctx **out);

/* Destroy a context.  Does not touch caller memory. */
PEPS_API int peps_destroy(peps_ctx *ctx);

/* Queue a single-qubit gate on qubit (r, c): A'^tau = sum_sigma U[tau][sigma]
 * A^sigma (paper, main-text "onebody" equation).  U: 4 complex, row-major. */
PEPS_API int peps_apply_1q(peps_ctx *ctx, int r, int c, const peps_c128 U[4]);

/* Queue a CZ on nearest neighbours (r0,c0), (r1,c1) (|dr| + |dc| == 1;
 * otherwise PEPS_ENOTADJ).  The bond on that edge doubles (paper, main-text
 * "factorize" and "twoqubita/b" equations with chi_o = 2). */
PEPS_API int peps_apply_cz(peps_ctx *ctx, int r0, int c0, int r1, int c1);

/* Absorb a general two-qubit gate on the nearest neighbours (r0,c0), (r1,c1),
 * in call order with the other gates.  G is 4x4, row-major, in the basis
 * |t0 t1> with qubit (r0,c0) first: G[(2*t0 + t1)*4 + (2*s0 + s1)].  The
 * gate is split by its operator-Schmidt decomposition (main text,
 * "factorize": SVD, singular values absorbed into the factor on the
 * lower-indexed site; FP64 on the host), and the shared bond grows by the
 * rank (1..4; CNOT 2, iSWAP and SWAP 4).  Any matrix is accepted (unitarity
 * is not needed).  Errors: PEPS_ENOTADJ, PEPS_EINVAL (non-finite entries, a
 * zero matrix), PEPS_EUNSUPPORTED (a bond above 2^20).  CZ gates on an edge
 * that carries a general gate cannot be sliced or held. */
PEPS_API int peps_apply_2q(peps_ctx *ctx, int r0, int c0, int r1, int c1, const peps_c128 G[16]);

/* Bond dimension of the edge between neighbours (r0,c0), (r1,c1):
 * 2^(number of CZ gates applied to it) (paper, "chi" bound equation) times
 * the ranks of the general two-qubit gates applied to it. */
PEPS_API int peps_bond_dim(const peps_ctx *ctx, int r0, int c0, int r1, int c1, int64_t *dim);

/* Static description of the contraction an amplitude call would run. */
typedef struct {
    int64_t n_steps;          /* contraction steps per chain                  */
    int64_t max_entries;      /* largest running tensor, complex entries     */
    double flops_per_chain;   /* algorithmic real flops of one full sweep:
                                 8 * sum over steps of M*K*N                 */
    double bytes_per_chain;   /* algorithmic bytes of one full sweep: the
                                 storage size of G read + G' written         */
    double flops_call;        /* the same summed over every chain of the call
                                 (prefix chains once per group, slices each) */
    double bytes_call;
    int64_t n_launches;       /* contraction launches of the call            */
    int64_t n_tc_launches;    /* of which tcgen05                            */
    int64_t n_slices;         /* slices summed                               */
    int64_t lanes;            /* bitstrings contracted concurrently          */
    double flops_lower;       /* odd-side square partition, one bitstring:
                                 the part of flops_per_chain in the lower half
                                 (bl, br -> F_b), which a slice skips when its
                                 lower bits equal the previous slice's; the
                                 call's slices run with equal lower bits
                                 adjacent (flops_call counts the skips)      */
    int64_t n_lower_bits;     /* sliced bits the lower half depends on (all
                                 of them where nothing is skipped)           */
} peps_plan_info;

/* Plan of an amplitude call on n_bitstrings with opts (host only). */
PEPS_API int peps_plan_info_get(const peps_ctx *ctx, int64_t n_bitstrings, const peps_opts *opts,
                                peps_plan_info *info);

/* One contraction step of a plan: the complex GEMM out[M x N] = G[M x K] E[K x N]
 * that absorbs a block of `sites` sites (0: a merge of two stored tensors),
 * with `variants` operands selected per bitstring, and where it runs. */
typedef struct {
    int64_t M;
    int32_t K, N;
    int32_t sites;            /* 1, 2, or 0 for a merge                      */
    int32_t variants;         /* operands of the step (per output bits)      */
    int32_t tensor_cores;     /* 1: tcgen05 kernel, 0: CUDA-core kernel      */
    int32_t part;             /* column sweep: -1; square partition: the
                                 quarter 0..3 (ul, bl, ur, br) or 4 = merge  */
    int64_t launches;         /* launches of the step in the call            */
    double flops;             /* algorithmic real flops of the step over the
                                 call (8 per complex multiply-add)           */
    /* layout of the stored output (row m = b Mr + m_hi (Mr / P) + m_lo,
     * column n = h' dv + v'): entry ((m_lo dh + h') P + m_hi) dv + v' of
     * batch slice b, or with open_leg = 1 entry (b dv + v') (Mr dh) +
     * (m_lo dh + h') P + m_hi (v' joins the batch)                         */
    int64_t P;                /* rotated row legs (moved next to v')         */
    int64_t Mr;               /* rows per batch slice (M when no batch)      */
    int32_t dv, dh;           /* dims of v' and of the h' legs               */
    int32_t open_leg;         /* 1: v' is an open leg stored into the batch  */
    int32_t fused_dot;        /* 1: the output is only dotted with a stored
                                 tensor in the epilogue (never written)      */
} peps_step_info;

/* The steps of the plan of an amplitude call, in sweep order: writes at most
 * `cap` entries (steps may be NULL when cap = 0) and the number of steps to
 * *n_out.  Host only. */
PEPS_API int peps_plan_steps(const peps_ctx *ctx, int64_t n_bitstrings, const peps_opts *opts,
                             peps_step_info *steps, int64_t cap, int64_t *n_out);

/* Device workspace needed for an amplitude call on n_bitstrings with opts. */
PEPS_API int peps_workspace_bytes(const peps_ctx *ctx, int64_t n_bitstrings, const peps_opts *opts,
                         size_t *bytes);

/* Amplitudes <x_i| C |0...0> for host bitstrings[0..n) into host out[0..n):
 * each is the network of the evolved PEPS with every site projected on its
 * output bit, E_q = A_q^{x_q}, contracted exactly (paper, main text: the
 * "overlap" equation; supplementary: the exact contraction of the overlap,
 * by the column sweep or the square partition as opts.scheme says).
 * Copies the bitstrings to the device on `stream`, runs the device path,
 * copies the results back and synchronises the stream before returning.
 * d_workspace: caller-owned device memory of ws_bytes >= peps_workspace_bytes
 * (PEPS_ENOMEM otherwise); it must stay allocated until the call returns and
 * no other call may use it concurrently.  `stream` is a cudaStream_t.
 * With slicing, out[i] is the FP64 sum over the selected slices.  On any
 * error `out` is untouched. */
PEPS_API int peps_amplitudes(peps_ctx *ctx, const uint64_t *bitstrings, int64_t n, peps_c128 *out,
                    const peps_opts *opts, void *d_workspace, size_t ws_bytes, void *stream);

/* Same with device-resident bitstrings (d_bitstrings) and results (d_out,
 * n peps_c128).  Enqueued on `stream`; returns after the host-side launch
 * sequence, without synchronising unless PEPS_FLAG_TIMING is set or a check
 * needs the device (prefix-group validation reads one int back). */
PEPS_API int peps_amplitudes_device(peps_ctx *ctx, const uint64_t *d_bitstrings, int64_t n,
                           peps_c128 *d_out, const peps_opts *opts, void *d_workspace,
                           size_t ws_bytes, void *stream);

/* Allocation-free variant of peps_amplitudes_device, for callers that cannot
 * call cudaMalloc (code running inside another framework's memory pool, a
 * plug-in whose host owns every device allocation, a tool that must not grow
 * device memory after start-up).  The paper has no counterpart; this is a
 * deployment convenience.
 *
 * The workspace is a static device array of 64 MiB inside this library: every
 * GPU that loads the library holds it until the process exits.  The caller
 * still passes the device bitstrings (n uint64) and the device output (n
 * peps_c128), and the stream.  Calls whose workspace (peps_workspace_bytes)
 * exceeds 64 MiB return PEPS_ENOMEM with a message; PEPS_FLAG_TIMING (which
 * creates CUDA events) and PEPS_FLAG_GRAPH (which creates a capture stream and
 * instantiates a graph) are rejected with PEPS_EINVAL.  The function calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call, from any context, shares the one array, which keeps the
 * previous call's contents: each call clears what must start at zero and
 * rebuilds the site tensors and tables it needs (the tables are copied in on
 * `stream`, after the work already enqueued there), so results never depend
 * on an earlier call.  Calls on one stream are therefore safe back to back;
 * calls that overlap on the GPU (other streams, other threads) race on the
 * array and must be serialised by the caller. */
PEPS_API int peps_amplitudes_noalloc(peps_ctx *ctx, const uint64_t *d_bitstrings, int64_t n,
                                     peps_c128 *d_out, const peps_opts *opts, void *stream);

/* CZ Schmidt bits fixed by the circuit's output or tied to one another (an
 * extension of the paper's exact contraction: zero terms of a bond sum are
 * skipped).  The CZ split P_0 (x) I + P_1 (x) Z puts the projector P_s on the
 * lower-index qubit q.  Between two events on q every CZ factor acting on q
 * is diagonal; where the single-qubit gates between them multiply to a
 * monomial matrix (diagonal or anti-diagonal), a basis state of q stays a
 * basis state, so consecutive projector bits on q are tied, the first to the
 * initial |0> and the last to the measured output bit x_q.  Lists every tied
 * CZ: its ordinal cz[i] (0 = the first CZ applied) and kind[i]:
 *   1: s = flip[i] (tied to the initial state);
 *   2: s = x_q XOR flip[i] for every output bitstring x (q = that CZ's
 *      lower-index qubit);
 *   3: s = (the bit of CZ src[i]) XOR flip[i], where src[i] is an earlier
 *      CZ on the same edge whose bit is free: a run of tied projectors that
 *      reaches neither end, with two of its bits in one bond index, so that
 *      index only takes half its values.
 * src[i] = 0xFFFFFFFF for kinds 1 and 2.  Writes at most `cap` entries (the
 * arrays may be NULL when cap = 0) and the total count to *n_out.  Host
 * only. */
PEPS_API int peps_output_ties(const peps_ctx *ctx, uint32_t *cz, uint8_t *kind, uint8_t *flip,
                              uint32_t *src, int64_t cap, int64_t *n_out);

/* One contraction launch of a timed call: its algorithmic work (real flops,
 * 8 per complex multiply-add; bytes of the running tensor read and written in
 * its storage format), its CUDA-event time, the kernel and the plan step. */
typedef struct {
    double flops;
    double bytes;
    float ms;
    int32_t tensor_cores;     /* 1: tcgen05 kernel, 0: CUDA-core kernels      */
    int32_t step;             /* peps_plan_steps index (-1: a whole-sweep
                                 launch of a small lattice)                   */
    int32_t pad_;
} peps_launch_info;

/* The contraction launches of the last amplitude call made with
 * PEPS_FLAG_TIMING (eager or as a CUDA graph), in launch order: writes at
 * most `cap` entries (out may be NULL when cap = 0) and the count to *n_out.
 * Host only; the call has synchronised its stream. */
PEPS_API int peps_launch_log(const peps_ctx *ctx, peps_launch_info *out, int64_t cap,
                             int64_t *n_out);

/* Counters of the last amplitude call on this context. */
PEPS_API int peps_get_stats(const peps_ctx *ctx, peps_stats *out);

/* Number of CZ gates queued so far (their ordinals are 0..n-1). */
PEPS_API int peps_cz_count(const peps_ctx *ctx, int64_t *n);

/* Text of the last error on the calling thread ("" if none). */
PEPS_API const char *peps_last_error(void);

/* Library version string. */
PEPS_API const char *peps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PEPS_GB300_H */
