// C ABI of the PEPS amplitude engine: circuit bookkeeping, the host planner
// (evolution schedule, step list of the column sweep, lanes, prefix reuse,
// slices, workspace layout) and the launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <complex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.h"

using namespace peps;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(PEPS_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                 \
  } while (0)

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
namespace {

struct GateRec {
  int kind;        // 0 = 1q, 1 = cz, 2 = general two-qubit gate
  int q0, q1;      // q0 < q1 for cz and general gates
  int horiz;       // two-qubit gate on a horizontal edge (same row)
  double U[8];     // re, im of U00, U01, U10, U11
  int chi = 0;     // general gate: Schmidt rank
  std::complex<double> W0[4][4], W1[4][4];  // [s][2*tau + sigma] on q0 / q1
};

struct Launch {
  int kind;        // 0 = contraction step, 1 = finalize, 2 = merge operand from a
                   // stored tensor, 3 = final dot product (square partition)
  StepShape shape;
  bool tc;
  void *tc_handle = nullptr;  // tensor maps of a tcgen05 launch
  int op_base = 0;            // first OpDesc of the step
  size_t a_base_rel = 0;      // input buffer of item lane 0 (relative to the buffer area)
  int a_lanes = 1;            // lanes addressed through the A tensor map
  int64_t items_off;  // index into the item array
  int n_items;
  int64_t fin_off;
  int n_fin;
  int64_t aux_off = 0;  // kind 2: TensorOpEntry index; kind 3: first DotEntry
  int n_aux = 0;
  int op = -1;          // kind 2: the OpDesc built
  int64_t kn = 0;       // kind 2: K * N of that operand
  double flops, bytes;
  bool lower = false;   // odd side: a launch of the lower half (bl, br -> F_b)
  bool small = false;   // kind 0: every step of every bitstring in one launch
  int step = -1;        // kind 0: the plan step it runs (-1: the whole sweep); kind 2:
                        // the merge step whose operands it builds
  int fused_merge = -1; // kind 3: index of the merge launch whose epilogue wrote
                        // the dot's partial sums (-1: the separate dot kernel)
};

struct Plan {
  // key
  uint64_t generation = 0;
  int64_t n = 0;
  peps_opts opts{};
  std::vector<uint32_t> sliced;
  std::vector<uint64_t> slice_ids;
  std::vector<uint32_t> fixed;
  std::vector<uint8_t> fixed_s;
  const void *ws = nullptr;
  size_t ws_bytes = 0;
  const uint64_t *bits = nullptr;
  bool host_bits = false;

  // layout
  size_t need = 0;
  int fmt = FMT_F32;
  int64_t cap = 0;          // entries per G buffer
  int64_t plane = 0;        // lo-plane offset in 16-bit units
  int n_steps = 0;
  int lanes = 0;
  int n_groups = 0;
  int glanes = 1;           // square partition: groups whose left quarters share a launch
  size_t off_status = 0, off_site_ptrs = 0, off_site_lo = 0, off_g1 = 0, off_cz = 0, off_g2 = 0, off_opdesc = 0,
         off_opbuild = 0, off_recs = 0, off_items = 0, off_fin = 0, off_acc = 0,
         off_bits = 0, off_out = 0, off_tables_end = 0;
  std::vector<size_t> site_buf_off[2];
  std::vector<int64_t> site_elems;
  std::vector<size_t> ec_off, bt_off[2];
  size_t lane_off = 0, prefix_off = 0;
  size_t gbuf_bytes = 0;
  size_t odd_bytes = 0;         // odd side: bytes of all sweep buffers

  // evolution batches
  struct EvoBatch {
    int kind;             // 0 = gate1, 1 = cz, 2 = general two-qubit gate
    int64_t off;          // first entry
    int n;
    int64_t max_work;
  };
  std::vector<EvoBatch> evo;
  std::vector<int> final_buf;  // which ping-pong buffer holds the final site tensor

  // step shapes
  std::vector<StepShape> steps;
  std::vector<std::array<int, 4>> step_roles;  // physical leg of the roles l, r, u, d
  int scheme = PEPS_SCHEME_COLUMNS;
  struct Quarter {
    int first = 0, count = 0;  // its sweep's steps
    int64_t batch = 1, rest = 1;  // stored as [batch][rest]
    int64_t rest_last = 1;     // dim of the fastest rest leg
    int64_t batch_last = 1;    // dim of the fastest batch leg
    int64_t span = 1;          // largest running tensor of its sweep (entries)
  } quarter[4];                 // ul, bl, ur, br
  bool odd = false;             // odd-side partition (Fig. S2(c))
  size_t obuf_off[8] = {};      // odd side: buffer offsets (hi planes), ul ur bl br pairs
  size_t obuf_fb = 0;           // odd side: F_b's own buffer
  // odd side, one bitstring: the slice-id bits the lower half depends on (its
  // sites' sliced CZs); a slice whose lower bits equal the previous slice's
  // keeps F_b and skips the lower half
  uint64_t lower_mask = 0;
  bool lower_skip = false;
  double flops_lower = 0;       // per slice
  int s_m1 = -1, s_m2 = -1;     // merge steps F_l = F_ul F_bl, Y = F_br F_l^T
  int op_m1 = -1, op_m2 = -1;
  int merge_slots = 1;          // operands per merge step: even square partition,
                                // one per group of a chunk (glanes), so that the
                                // chunk's merges share one launch
  int n_site_ops = 0;           // ops rebuilt from the site tensors per slice
  int64_t max_kn_merge = 0;
  size_t off_tops = 0, off_dots = 0, off_partials = 0;
  int bufs_per_lane = 2;
  std::vector<int> step_site;
  std::vector<int> step_opbase;  // first OpDesc of each step (2^nq variants)
  int n_ops = 0;
  int64_t n_obe2_per_slice = 0;
  int max_kn2 = 0;
  size_t off_opbuild2 = 0;

  // launches (per slice iteration)
  std::vector<Launch> launches;
  int n_recs = 0;
  int64_t n_opbuild_per_slice = 0;
  // per slice: first entry and count of the operand builds it launches (the
  // first slice builds every operand, a later one only those whose
  // restriction differs from the slice before it)
  std::vector<int64_t> obe_first, obe_count, obe2_first, obe2_count;
  int max_kn = 0;
  std::vector<int64_t> slice_list;
  double flops_per_slice = 0, bytes_per_slice = 0;

  // small lattices: the whole sweep of every bitstring in one launch
  // (running tensors in shared memory), the evolution in one launch with a
  // block per site
  bool small = false;
  int small_cap_g = 0, small_cap_e = 0;
  size_t off_small_steps = 0, off_small_opbase = 0;
  const uint64_t *small_bits = nullptr;
  bool evo_sites = false;       // the whole evolution in one launch
  int evo_prefix = 0;           // leading gate batches done by that launch (a block
                                // per site) while every site tensor is small; the
                                // rest one launch per batch
  size_t off_evo_refs = 0, off_evo_first = 0;

  // host copy of the tables (uploaded once): [off_site_ptrs, off_ops_begin)
  // then [off_opdesc, off_tables_end); the operand storage between them is
  // written on the device only
  std::vector<unsigned char> blob;
  size_t off_ops_begin = 0;

  // CUDA graphs of the whole launch sequence (PEPS_FLAG_GRAPH): [0] plain,
  // [1] with timing events around its contraction launches; each captured
  // on its first use
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  size_t graph_n_timed = 0;
  std::vector<int> graph_timed_idx;   // launch index of each timed launch

  ~Plan() {
    for (auto g : graph_exec)
      if (g) cudaGraphExecDestroy(g);
    for (auto &l : launches)
      if (l.tc_handle) tc_release(l.tc_handle);
  }
};

}  // namespace

struct peps_ctx {
  int R = 0, C = 0, n = 0;
  std::vector<GateRec> gates;
  std::vector<int> ncz_h, ncz_v;  // CZ count per horizontal / vertical edge
  std::vector<int64_t> gmul_h, gmul_v;  // product of the general gates' ranks
  std::vector<int> ngen_h, ngen_v;      // general gates per edge
  uint64_t generation = 1;
  uint64_t built_generation = 0;
  const void *built_ws = nullptr;
  std::unique_ptr<Plan> plan;
  peps_stats stats{};
  bool broken = false;
  std::vector<cudaEvent_t> ev;
  int sm_count = 0;
  std::vector<peps_launch_info> launch_log;  // contraction launches of the last timed call
  cudaStream_t cap_stream = nullptr;  // records CUDA graphs (the caller's stream
                                      // may be the legacy default stream)
};

static int edge_h(const peps_ctx *c, int r, int col) { return r * (c->C - 1) + col; }
static int edge_v(const peps_ctx *c, int r, int col) { return r * c->C + col; }

// ---------------------------------------------------------------------------
// Circuit bookkeeping
// ---------------------------------------------------------------------------
extern "C" int peps_create(int R, int C, peps_ctx **out) {
  if (!out) return fail(PEPS_EINVAL, "peps_create: out is NULL");
  if (R < 1 || C < 1 || (int64_t)R * C > 64)
    return fail(PEPS_EINVAL, "peps_create: need R, C >= 1 and R*C <= 64 (got %d x %d)", R, C);
  peps_ctx *c = new peps_ctx();
  c->R = R;
  c->C = C;
  c->n = R * C;
  c->ncz_h.assign(R * std::max(C - 1, 0), 0);
  c->ncz_v.assign(std::max(R - 1, 0) * C, 0);
  c->gmul_h.assign(c->ncz_h.size(), 1);
  c->gmul_v.assign(c->ncz_v.size(), 1);
  c->ngen_h.assign(c->ncz_h.size(), 0);
  c->ngen_v.assign(c->ncz_v.size(), 0);
  *out = c;
  return PEPS_OK;
}

extern "C" int peps_destroy(peps_ctx *c) {
  if (!c) return fail(PEPS_EINVAL, "peps_destroy: NULL context");
  for (auto e : c->ev) cudaEventDestroy(e);
  c->plan.reset();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return PEPS_OK;
}

extern "C" int peps_apply_1q(peps_ctx *c, int r, int col, const peps_c128 U[4]) {
  if (!c || !U) return fail(PEPS_EINVAL, "peps_apply_1q: NULL argument");
  if (c->broken) return fail(PEPS_ESTATE, "context unusable after an earlier device failure");
  if (r < 0 || r >= c->R || col < 0 || col >= c->C)
    return fail(PEPS_EINVAL, "peps_apply_1q: qubit (%d,%d) outside %dx%d", r, col, c->R, c->C);
  GateRec g{};
  g.kind = 0;
  g.q0 = g.q1 = r * c->C + col;
  for (int i = 0; i < 4; ++i) {
    if (!std::isfinite(U[i].re) || !std::isfinite(U[i].im))
      return fail(PEPS_EINVAL, "peps_apply_1q: non-finite matrix entry");
    g.U[2 * i] = U[i].re;
    g.U[2 * i + 1] = U[i].im;
  }
  c->gates.push_back(g);
  c->generation++;
  return PEPS_OK;
}

extern "C" int peps_apply_cz(peps_ctx *c, int r0, int c0, int r1, int c1) {
  if (!c) return fail(PEPS_EINVAL, "peps_apply_cz: NULL context");
  if (c->broken) return fail(PEPS_ESTATE, "context unusable after an earlier device failure");
  if (r0 < 0 || r0 >= c->R || c0 < 0 || c0 >= c->C || r1 < 0 || r1 >= c->R || c1 < 0 ||
      c1 >= c->C)
    return fail(PEPS_EINVAL, "peps_apply_cz: qubit outside the %dx%d lattice", c->R, c->C);
  if (std::abs(r0 - r1) + std::abs(c0 - c1) != 1)
    return fail(PEPS_ENOTADJ, "peps_apply_cz: (%d,%d) and (%d,%d) are not nearest neighbours",
                r0, c0, r1, c1);
  int qa = r0 * c->C + c0, qb = r1 * c->C + c1;
  if (qa > qb) std::swap(qa, qb);
  const int ra = qa / c->C, ca = qa % c->C;
  const bool horiz = r0 == r1;  // by coordinates: on a one-column lattice qb == qa + 1 is vertical
  const int e = horiz ? edge_h(c, ra, ca) : edge_v(c, ra, ca);
  int &cnt = horiz ? c->ncz_h[e] : c->ncz_v[e];
  const int64_t gm = horiz ? c->gmul_h[e] : c->gmul_v[e];
  if (((int64_t)1 << (cnt + 1)) * gm > ((int64_t)1 << 20))
    return fail(PEPS_EUNSUPPORTED, "peps_apply_cz: bond dimension above 2^20 on one edge");
  cnt++;
  GateRec g{};
  g.kind = 1;
  g.q0 = qa;
  g.q1 = qb;
  g.horiz = horiz ? 1 : 0;
  c->gates.push_back(g);
  c->generation++;
  return PEPS_OK;
}

// Operator-Schmidt split of a two-qubit gate (main text, "factorize"):
// M[(t0 s0), (t1 s1)] = G[(t0 t1), (s0 s1)] = sum_k W0_k[t0 s0] W1_k[t1 s1]
// with W0_k = M v_k and W1_k = conj(v_k), v_k the eigenvectors of M^H M with
// nonzero eigenvalue (the right singular vectors; the singular values end up
// in W0, as the paper absorbs them into U).  Cyclic complex Jacobi on the
// 4x4 Hermitian matrix.  Returns the rank (0 for a zero matrix).
static int split_2q(const std::complex<double> G[4][4], std::complex<double> W0[4][4],
                    std::complex<double> W1[4][4]) {
  typedef std::complex<double> cd;
  cd M[4][4], H[4][4], V[4][4];
  for (int t0 = 0; t0 < 2; ++t0)
    for (int t1 = 0; t1 < 2; ++t1)
      for (int s0 = 0; s0 < 2; ++s0)
        for (int s1 = 0; s1 < 2; ++s1) M[2 * t0 + s0][2 * t1 + s1] = G[2 * t0 + t1][2 * s0 + s1];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd acc = 0;
      for (int k = 0; k < 4; ++k) acc += std::conj(M[k][i]) * M[k][j];
      H[i][j] = acc;
      V[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        tot += std::norm(H[i][j]);
        if (i != j) off += std::norm(H[i][j]);
      }
    if (off <= 1e-32 * tot || tot == 0) break;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 4; ++q) {
        const double a = std::abs(H[p][q]);
        if (a == 0) continue;
        // rotate in the (p, q) plane: H' = J^H H J zeroes H[p][q]
        const cd ph = H[p][q] / a;
        const double theta = 0.5 * std::atan2(2 * a, (H[q][q] - H[p][p]).real());
        const double cs = std::cos(theta), sn = std::sin(theta);
        // J = [[c, s ph], [-s conj(ph), c]] on columns p, q
        for (int k = 0; k < 4; ++k) {
          const cd hkp = H[k][p], hkq = H[k][q];
          H[k][p] = cs * hkp - sn * std::conj(ph) * hkq;
          H[k][q] = sn * ph * hkp + cs * hkq;
        }
        for (int k = 0; k < 4; ++k) {
          const cd hpk = H[p][k], hqk = H[q][k];
          H[p][k] = cs * hpk - sn * ph * hqk;
          H[q][k] = sn * std::conj(ph) * hpk + cs * hqk;
        }
        for (int k = 0; k < 4; ++k) {
          const cd vkp = V[k][p], vkq = V[k][q];
          V[k][p] = cs * vkp - sn * std::conj(ph) * vkq;
          V[k][q] = sn * ph * vkp + cs * vkq;
        }
      }
  }
  int order[4] = {0, 1, 2, 3};
  std::sort(order, order + 4, [&](int x, int y) { return H[x][x].real() > H[y][y].real(); });
  const double lmax = H[order[0]][order[0]].real();
  int chi = 0;
  for (int r = 0; r < 4; ++r) {
    const int k = order[r];
    if (!(lmax > 0) || H[k][k].real() <= 1e-24 * lmax) break;
    for (int i = 0; i < 4; ++i) {
      cd acc = 0;
      for (int j = 0; j < 4; ++j) acc += M[i][j] * V[j][k];
      W0[chi][i] = acc;
      W1[chi][i] = std::conj(V[i][k]);
    }
    ++chi;
  }
  return chi;
}

extern "C" int peps_apply_2q(peps_ctx *c, int r0, int c0, int r1, int c1, const peps_c128 G[16]) {
  if (!c || !G) return fail(PEPS_EINVAL, "peps_apply_2q: NULL argument");
  if (c->broken) return fail(PEPS_ESTATE, "context unusable after an earlier device failure");
  if (r0 < 0 || r0 >= c->R || c0 < 0 || c0 >= c->C || r1 < 0 || r1 >= c->R || c1 < 0 ||
      c1 >= c->C)
    return fail(PEPS_EINVAL, "peps_apply_2q: qubit outside the %dx%d lattice", c->R, c->C);
  if (std::abs(r0 - r1) + std::abs(c0 - c1) != 1)
    return fail(PEPS_ENOTADJ, "peps_apply_2q: (%d,%d) and (%d,%d) are not nearest neighbours",
                r0, c0, r1, c1);
  std::complex<double> g[4][4];
  for (int i = 0; i < 16; ++i) {
    if (!std::isfinite(G[i].re) || !std::isfinite(G[i].im))
      return fail(PEPS_EINVAL, "peps_apply_2q: non-finite matrix entry");
    g[i / 4][i % 4] = std::complex<double>(G[i].re, G[i].im);
  }
  int qa = r0 * c->C + c0, qb = r1 * c->C + c1;
  if (qa > qb) {  // the lower site first: G'[(t1 t0), (s1 s0)] = G[(t0 t1), (s0 s1)]
    std::swap(qa, qb);
    std::complex<double> t[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t[((i & 1) << 1) | (i >> 1)][((j & 1) << 1) | (j >> 1)] = g[i][j];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) g[i][j] = t[i][j];
  }
  GateRec rec{};
  rec.kind = 2;
  rec.q0 = qa;
  rec.q1 = qb;
  const int ra = qa / c->C, ca = qa % c->C;
  rec.horiz = (r0 == r1) ? 1 : 0;
  rec.chi = split_2q(g, rec.W0, rec.W1);
  if (rec.chi == 0) return fail(PEPS_EINVAL, "peps_apply_2q: zero matrix");
  const int e = rec.horiz ? edge_h(c, ra, ca) : edge_v(c, ra, ca);
  int64_t &gm = rec.horiz ? c->gmul_h[e] : c->gmul_v[e];
  const int ncz = rec.horiz ? c->ncz_h[e] : c->ncz_v[e];
  if (((int64_t)1 << ncz) * gm * rec.chi > ((int64_t)1 << 20))
    return fail(PEPS_EUNSUPPORTED, "peps_apply_2q: bond dimension above 2^20 on one edge");
  gm *= rec.chi;
  (rec.horiz ? c->ngen_h[e] : c->ngen_v[e])++;
  c->gates.push_back(rec);
  c->generation++;
  return PEPS_OK;
}

extern "C" int peps_bond_dim(const peps_ctx *c, int r0, int c0, int r1, int c1, int64_t *dim) {
  if (!c || !dim) return fail(PEPS_EINVAL, "peps_bond_dim: NULL argument");
  if (r0 < 0 || r0 >= c->R || c0 < 0 || c0 >= c->C || r1 < 0 || r1 >= c->R || c1 < 0 ||
      c1 >= c->C)
    return fail(PEPS_EINVAL, "peps_bond_dim: qubit outside the lattice");
  if (std::abs(r0 - r1) + std::abs(c0 - c1) != 1)
    return fail(PEPS_ENOTADJ, "peps_bond_dim: not nearest neighbours");
  int qa = r0 * c->C + c0, qb = r1 * c->C + c1;
  if (qa > qb) std::swap(qa, qb);
  const int ra = qa / c->C, ca = qa % c->C;
  const bool h = r0 == r1;
  const int e = h ? edge_h(c, ra, ca) : edge_v(c, ra, ca);
  const int cnt = h ? c->ncz_h[e] : c->ncz_v[e];
  *dim = ((int64_t)1 << cnt) * (h ? c->gmul_h[e] : c->gmul_v[e]);
  return PEPS_OK;
}

extern "C" int peps_cz_count(const peps_ctx *c, int64_t *n) {
  if (!c || !n) return fail(PEPS_EINVAL, "peps_cz_count: NULL argument");
  int64_t k = 0;
  for (auto &g : c->gates) k += g.kind == 1;
  *n = k;
  return PEPS_OK;
}

extern "C" const char *peps_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *peps_version(void) { return "peps_gb300 0.1 (sm_103a)"; }

extern "C" int peps_launch_log(const peps_ctx *c, peps_launch_info *out, int64_t cap,
                               int64_t *n_out) {
  if (!c || !n_out) return fail(PEPS_EINVAL, "peps_launch_log: NULL argument");
  if (cap < 0 || (cap > 0 && !out)) return fail(PEPS_EINVAL, "peps_launch_log: bad output array");
  const int64_t n = (int64_t)c->launch_log.size();
  for (int64_t i = 0; i < std::min(cap, n); ++i) out[i] = c->launch_log[i];
  *n_out = n;
  return PEPS_OK;
}

extern "C" int peps_get_stats(const peps_ctx *c, peps_stats *out) {
  if (!c || !out) return fail(PEPS_EINVAL, "peps_get_stats: NULL argument");
  *out = c->stats;
  return PEPS_OK;
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

struct LegInfo {
  // per edge: full dim, sliced-bit mask (bits of the bond index that are fixed)
  std::vector<int> dim_h, dim_v;
  std::vector<uint32_t> fix_h, fix_v;
};

int popcount32(uint32_t x) { return __builtin_popcount(x); }
int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// Which edge and bond bit a CZ ordinal owns.
struct CzPos {
  bool horiz;
  int edge;
  int bit;
};

int locate_cz(const peps_ctx *c, std::vector<CzPos> &pos) {
  std::vector<int> seen_h(c->ncz_h.size(), 0), seen_v(c->ncz_v.size(), 0);
  for (auto &g : c->gates) {
    if (g.kind != 1) continue;
    const int ra = g.q0 / c->C, ca = g.q0 % c->C;
    CzPos p{};
    if (g.horiz) {
      p.horiz = true;
      p.edge = edge_h(c, ra, ca);
      p.bit = c->ncz_h[p.edge] - 1 - seen_h[p.edge]++;
    } else {
      p.horiz = false;
      p.edge = edge_v(c, ra, ca);
      p.bit = c->ncz_v[p.edge] - 1 - seen_v[p.edge]++;
    }
    pos.push_back(p);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Schmidt bits that the output bitstring fixes.  A CZ split as
// P_0 (x) I + P_1 (x) Z puts the projector P_s on its lower-index qubit q and
// Z^s on the other.  Between two events on q (CZ factors of either kind, or
// the measurement) every CZ factor acting on q is diagonal in its basis; if
// each run of single-qubit gates in between is a monomial matrix (diagonal or
// anti-diagonal), a basis state of q is carried to a basis state.  So the
// bits of consecutive projectors on q are tied (equal or flipped), the first
// one to the initial |0> and the last one to the measured bit x_q, wherever
// the runs between them are monomial.  Every term of the bond sum that breaks
// such a tie is exactly zero: the bit can be held at its tied value.  A run
// of tied projectors that reaches neither end is free as a whole, but where
// two of its bits belong to one bond (the same edge), that bond index only
// takes the values in which the later bit equals the earlier one (or its
// flip): the bond keeps half its values per such linked bit.
// ---------------------------------------------------------------------------
struct CzTie {
  int kind;   // 0 = free, 1 = constant (bit = flip), 2 = output (bit = x_q ^ flip),
              // 3 = linked (bit = bit of CZ `src` ^ flip, src on the same edge)
  int q;      // the projector's qubit (the CZ's lower-index qubit)
  int flip;
  int src = -1;
};

// 0 = diagonal, 1 = anti-diagonal, -1 = neither (relative tolerance 1e-12)
int monomial_kind(const std::complex<double> M[4]) {
  double s = 0;
  for (int i = 0; i < 4; ++i) s = std::max(s, std::abs(M[i]));
  const double tol = 1e-12 * s;
  if (std::abs(M[1]) <= tol && std::abs(M[2]) <= tol) return 0;
  if (std::abs(M[0]) <= tol && std::abs(M[3]) <= tol) return 1;
  return -1;
}

void output_ties(const peps_ctx *c, std::vector<CzTie> &ties) {
  typedef std::complex<double> cd;
  const int n = c->n;
  std::vector<std::vector<int>> runs(n);   // per qubit: monomial kind of each closed run
  std::vector<std::array<cd, 4>> cur(n, std::array<cd, 4>{cd(1), cd(0), cd(0), cd(1)});
  struct Ev { int k, ev; };
  std::vector<std::vector<Ev>> proj(n);    // per qubit: its projector events in order
  auto close = [&](int q, bool bad) {
    runs[q].push_back(bad ? -1 : monomial_kind(cur[q].data()));
    cur[q] = {cd(1), cd(0), cd(0), cd(1)};
  };
  int k = 0;
  std::vector<int> cz_edge;   // per CZ ordinal: its edge (h edges, then v edges)
  for (auto &g : c->gates) {
    if (g.kind == 1) {
      const int ra = g.q0 / c->C, ca = g.q0 % c->C;
      cz_edge.push_back(g.horiz ? edge_h(c, ra, ca) : (int)c->ncz_h.size() + edge_v(c, ra, ca));
    }
    if (g.kind == 0) {
      const int q = g.q0;
      cd U[4], M[4];
      for (int i = 0; i < 4; ++i) U[i] = cd(g.U[2 * i], g.U[2 * i + 1]);
      for (int r = 0; r < 2; ++r)
        for (int col = 0; col < 2; ++col)
          M[2 * r + col] = U[2 * r] * cur[q][col] + U[2 * r + 1] * cur[q][2 + col];
      for (int i = 0; i < 4; ++i) cur[q][i] = M[i];
    } else if (g.kind == 1) {
      proj[g.q0].push_back({k++, (int)runs[g.q0].size()});
      close(g.q0, false);
      close(g.q1, false);
    } else {
      close(g.q0, true);
      close(g.q1, true);
    }
  }
  for (int q = 0; q < n; ++q) close(q, false);   // the last run ends at the measurement
  ties.assign(k, CzTie{0, -1, 0});
  for (int q = 0; q < n; ++q) {
    const auto &R = runs[q];
    // parity of runs lo .. hi-1, or -1 if one of them is not monomial
    auto span = [&](int lo, int hi) {
      int par = 0;
      for (int i = lo; i < hi; ++i) {
        if (R[i] < 0) return -1;
        par ^= R[i];
      }
      return par;
    };
    const auto &E = proj[q];
    const int m = (int)E.size();
    if (!m) continue;
    // forward from the initial |0>
    int val = 0, prev = -1;
    for (int i = 0; i < m; ++i) {
      const int f = span(prev + 1, E[i].ev + 1);
      if (f < 0) break;
      val ^= f;
      ties[E[i].k] = CzTie{1, q, val};
      prev = E[i].ev;
    }
    // backward from the measured bit x_q
    int flip = span(E[m - 1].ev + 1, (int)R.size());
    for (int i = m - 1; i >= 0 && flip >= 0; --i) {
      if (ties[E[i].k].kind == 0) ties[E[i].k] = CzTie{2, q, flip};
      if (i > 0) {
        const int f = span(E[i - 1].ev + 1, E[i].ev + 1);
        flip = f < 0 ? -1 : flip ^ f;
      }
    }
    // free runs: link later bits of one edge to the run's first bit on it
    int a = 0;
    while (a < m) {
      int b = a + 1;
      std::vector<int> par(1, 0);
      while (b < m) {
        const int f = span(E[b - 1].ev + 1, E[b].ev + 1);
        if (f < 0) break;
        par.push_back(par.back() ^ f);
        ++b;
      }
      if (ties[E[a].k].kind == 0) {
        for (int i = a; i < b; ++i)
          for (int j = a; j < i; ++j)
            if (cz_edge[E[j].k] == cz_edge[E[i].k] && ties[E[j].k].kind == 0) {
              CzTie t{3, q, par[i - a] ^ par[j - a]};
              t.src = E[j].k;
              ties[E[i].k] = t;
              break;
            }
      }
      a = b;
    }
  }
}

}  // namespace

extern "C" int peps_output_ties(const peps_ctx *c, uint32_t *cz, uint8_t *kind, uint8_t *flip,
                                uint32_t *src, int64_t cap, int64_t *n_out) {
  if (!c || !n_out) return fail(PEPS_EINVAL, "peps_output_ties: NULL argument");
  if (cap < 0) return fail(PEPS_EINVAL, "peps_output_ties: negative capacity");
  std::vector<CzTie> ties;
  output_ties(c, ties);
  int64_t k = 0;
  for (size_t j = 0; j < ties.size(); ++j) {
    if (ties[j].kind == 0) continue;
    if (k < cap) {
      if (!cz || !kind || !flip || !src)
        return fail(PEPS_EINVAL, "peps_output_ties: NULL output array");
      cz[k] = (uint32_t)j;
      kind[k] = (uint8_t)ties[j].kind;
      flip[k] = (uint8_t)ties[j].flip;
      src[k] = ties[j].src < 0 ? 0xFFFFFFFFu : (uint32_t)ties[j].src;
    }
    ++k;
  }
  *n_out = k;
  return PEPS_OK;
}

static bool opts_equal(const peps_opts &a, const peps_opts &b) {
  return a.precision == b.precision && (a.flags & ~PEPS_FLAG_TIMING) == (b.flags & ~PEPS_FLAG_TIMING) &&
         a.prefix_cols == b.prefix_cols && a.prefix_group == b.prefix_group &&
         a.max_lanes == b.max_lanes && a.n_sliced == b.n_sliced &&
         a.n_slice_ids == b.n_slice_ids && a.n_fixed == b.n_fixed &&
         a.tc_kchunk == b.tc_kchunk && a.tc_cluster == b.tc_cluster &&
         a.fuse_rows == b.fuse_rows && a.scheme == b.scheme && a.tc_ksplit == b.tc_ksplit &&
         a.measured_mask == b.measured_mask;
}

// Build (or size) the plan.  With ws == nullptr only sizes are computed.
// Operand slots of step s: the bitstring variants of a site step, or the
// per-group slots of a square-partition merge.
static int op_slots(const Plan &P, int s) {
  if (P.scheme == PEPS_SCHEME_QUADRANTS && (s == P.s_m1 || s == P.s_m2)) return P.merge_slots;
  return step_variants(P.steps[s]);
}

static int build_plan(peps_ctx *c, int64_t n, const peps_opts &o, const void *ws,
                      size_t ws_bytes, const uint64_t *bits_dev, bool host_bits, Plan &P) {
  const int R = c->R, C = c->C, NQ = c->n;
  if (n < 0) return fail(PEPS_EINVAL, "negative bitstring count");
  if (o.precision < 0 || o.precision >= PEPS_N_PRECISIONS)
    return fail(PEPS_EINVAL, "unknown precision %d", o.precision);
  if (o.prefix_cols < 0 || o.prefix_cols >= C)
    return fail(PEPS_EINVAL, "prefix_cols must be in [0, C) (got %d)", o.prefix_cols);
  if (o.prefix_cols > 0 && o.prefix_group < 1)
    return fail(PEPS_EINVAL, "prefix_group must be >= 1 with prefix_cols > 0");
  if (o.prefix_cols > 0 && n % o.prefix_group != 0)
    return fail(PEPS_EINVAL, "n (%lld) must be a multiple of prefix_group (%d)", (long long)n,
                o.prefix_group);
  if (o.max_lanes < 0 || o.max_lanes > 4096) return fail(PEPS_EINVAL, "max_lanes out of range");
  if (o.n_sliced < 0 || o.n_sliced > 62) return fail(PEPS_EINVAL, "n_sliced out of range");
  if (o.n_sliced > 0 && !o.sliced_cz) return fail(PEPS_EINVAL, "sliced_cz is NULL");
  if (o.n_slice_ids < 0) return fail(PEPS_EINVAL, "n_slice_ids < 0");
  if (o.n_fixed < 0) return fail(PEPS_EINVAL, "n_fixed < 0");
  if (o.fuse_rows < 0 || o.fuse_rows > 1) return fail(PEPS_EINVAL, "fuse_rows must be 0 or 1");
  if (o.tc_ksplit < -1 || o.tc_ksplit > 4) return fail(PEPS_EINVAL, "tc_ksplit must be in [-1, 4]");
  if (o.scheme != PEPS_SCHEME_COLUMNS && o.scheme != PEPS_SCHEME_QUADRANTS)
    return fail(PEPS_EINVAL, "unknown contraction scheme %d", o.scheme);
  const bool quad = o.scheme == PEPS_SCHEME_QUADRANTS;
  // marginals: the double-layer network, every bond squared (no slicing)
  const bool dl = (o.flags & PEPS_FLAG_MARGINALS) != 0;
  if (dl && (o.n_sliced > 0 || o.n_fixed > 0))
    return fail(PEPS_EINVAL, "marginals do not combine with slicing or held CZ bits");
  // even R and C: Fig. S2(b); an odd square side 2m+1: Fig. S2(c)
  const bool odd = quad && (R % 2 || C % 2);
  if (odd && (R != C || R < 3))
    return fail(PEPS_EINVAL, "the square partition needs even R and C, or R = C odd (got %d x %d)",
                R, C);
  if (quad && !odd && o.prefix_cols != 0 && o.prefix_cols != C / 2)
    return fail(PEPS_EINVAL, "with the square partition prefix_cols must be 0 or C/2");
  if (odd && o.prefix_cols != 0)
    return fail(PEPS_EINVAL, "the odd-side partition takes no prefix groups");
  if (!tc_tuning_valid(o.tc_kchunk, o.tc_cluster, o.tc_epi))
    return fail(PEPS_EINVAL, "tc_kchunk must be 0, 64 or 128, tc_cluster 0, 1 or 2, tc_epi 0, 4 or 8");
  if (o.n_fixed > 0 && (!o.fixed_cz || !o.fixed_s)) return fail(PEPS_EINVAL, "fixed_cz / fixed_s is NULL");

  P.generation = c->generation;
  P.n = n;
  P.opts = o;
  P.ws = ws;
  P.ws_bytes = ws_bytes;
  P.bits = bits_dev;
  P.host_bits = host_bits;
  P.fmt = format_of(o.precision);
  const int fmt = P.fmt;
  const int bpe = format_bytes_per_entry(fmt);

  // ---- slicing: which bond bits are fixed ----
  std::vector<CzPos> czpos;
  locate_cz(c, czpos);
  LegInfo L;
  L.dim_h.resize(c->ncz_h.size());
  L.dim_v.resize(c->ncz_v.size());
  for (size_t e = 0; e < c->ncz_h.size(); ++e) L.dim_h[e] = (int)((1LL << c->ncz_h[e]) * c->gmul_h[e]);
  for (size_t e = 0; e < c->ncz_v.size(); ++e) L.dim_v[e] = (int)((1LL << c->ncz_v[e]) * c->gmul_v[e]);
  L.fix_h.assign(c->ncz_h.size(), 0u);
  L.fix_v.assign(c->ncz_v.size(), 0u);
  P.sliced.assign(o.sliced_cz ? o.sliced_cz : nullptr, o.sliced_cz ? o.sliced_cz + o.n_sliced : nullptr);
  for (int j = 0; j < o.n_sliced; ++j) {
    const uint32_t k = o.sliced_cz[j];
    if (k >= czpos.size()) return fail(PEPS_EINVAL, "sliced CZ ordinal %u out of range", k);
    const CzPos &p = czpos[k];
    if (p.horiz ? c->ngen_h[p.edge] : c->ngen_v[p.edge])
      return fail(PEPS_EINVAL, "CZ ordinal %u shares its edge with a general two-qubit gate "
                  "(its bond bit is not addressable); it cannot be sliced", k);
    uint32_t &m = p.horiz ? L.fix_h[p.edge] : L.fix_v[p.edge];
    if (m & (1u << p.bit)) return fail(PEPS_EINVAL, "CZ ordinal %u sliced twice", k);
    m |= 1u << p.bit;
  }
  // CZ bits held at one value in every slice (sub-slices)
  std::vector<uint32_t> fixval_h(c->ncz_h.size(), 0u), fixval_v(c->ncz_v.size(), 0u);
  P.fixed.assign(o.fixed_cz ? o.fixed_cz : nullptr, o.fixed_cz ? o.fixed_cz + o.n_fixed : nullptr);
  P.fixed_s.assign(o.fixed_s ? o.fixed_s : nullptr, o.fixed_s ? o.fixed_s + o.n_fixed : nullptr);
  for (int j = 0; j < o.n_fixed; ++j) {
    const uint32_t k = o.fixed_cz[j];
    if (k >= czpos.size()) return fail(PEPS_EINVAL, "fixed CZ ordinal %u out of range", k);
    if (o.fixed_s[j] > 1) return fail(PEPS_EINVAL, "fixed_s[%d] must be 0 or 1", j);
    const CzPos &p = czpos[k];
    if (p.horiz ? c->ngen_h[p.edge] : c->ngen_v[p.edge])
      return fail(PEPS_EINVAL, "CZ ordinal %u shares its edge with a general two-qubit gate; "
                  "it cannot be held", k);
    uint32_t &m = p.horiz ? L.fix_h[p.edge] : L.fix_v[p.edge];
    if (m & (1u << p.bit)) return fail(PEPS_EINVAL, "CZ ordinal %u fixed or sliced twice", k);
    m |= 1u << p.bit;
    if (o.fixed_s[j]) (p.horiz ? fixval_h[p.edge] : fixval_v[p.edge]) |= 1u << p.bit;
  }
  // held bits (PEPS_FLAG_HOLD_TIES): per edge the held mask joins the fixed
  // mask (the bond shrinks), and the held values are hv0 / hv1 for the
  // output bit 0 / 1 of the edge's projector qubit hq (-1: no held bit on
  // the edge depends on the output; then hv0 == hv1)
  const bool hold = (o.flags & PEPS_FLAG_HOLD_TIES) != 0;
  if (hold && (o.n_sliced > 0 || o.n_fixed > 0 || dl))
    return fail(PEPS_EINVAL, "PEPS_FLAG_HOLD_TIES does not combine with slicing, held CZ bits "
                "or marginals");
  std::vector<uint32_t> hv0_h(c->ncz_h.size(), 0u), hv1_h(c->ncz_h.size(), 0u);
  std::vector<uint32_t> hv0_v(c->ncz_v.size(), 0u), hv1_v(c->ncz_v.size(), 0u);
  std::vector<int> hq_h(c->ncz_h.size(), -1), hq_v(c->ncz_v.size(), -1);
  // linked bits: per edge, (source bit, linked bit) pairs; the linked bit's
  // value is the source bit's XOR its flip (the flip sits in hv0/hv1)
  typedef std::vector<std::pair<int, int>> Links;
  std::vector<Links> lk_h(c->ncz_h.size()), lk_v(c->ncz_v.size());
  if (hold) {
    std::vector<CzTie> ties;
    output_ties(c, ties);
    for (size_t k = 0; k < ties.size(); ++k) {
      const CzTie &t = ties[k];
      if (t.kind == 0) continue;
      const CzPos &p = czpos[k];
      if (p.horiz ? c->ngen_h[p.edge] : c->ngen_v[p.edge]) continue;  // bit not addressable
      (p.horiz ? L.fix_h[p.edge] : L.fix_v[p.edge]) |= 1u << p.bit;
      const uint32_t v0 = (uint32_t)t.flip, v1 = t.kind == 2 ? (uint32_t)(t.flip ^ 1) : v0;
      (p.horiz ? hv0_h[p.edge] : hv0_v[p.edge]) |= v0 << p.bit;
      (p.horiz ? hv1_h[p.edge] : hv1_v[p.edge]) |= v1 << p.bit;
      if (t.kind == 2) (p.horiz ? hq_h[p.edge] : hq_v[p.edge]) = t.q;
      if (t.kind == 3) {
        const CzPos &ps = czpos[t.src];
        if (ps.horiz != p.horiz || ps.edge != p.edge)
          return fail(PEPS_EINVAL, "internal: linked CZ bits on different edges");
        Links &lk = p.horiz ? lk_h[p.edge] : lk_v[p.edge];
        if ((int)lk.size() >= kMaxLinks)
          return fail(PEPS_EUNSUPPORTED, "more than %d linked bits on one edge", kMaxLinks);
        lk.push_back({ps.bit, p.bit});
      }
    }
  }
  // Qubits other than the block's own sites whose output bits select a
  // block's operand: the projector qubits of held bits on the sites' legs.
  auto set_variant_qubits = [&](StepShape &sh) -> int {
    sh.nx = 0;
    if (!hold || sh.nq < 1) return PEPS_OK;
    int sites[2] = {sh.q, sh.q + sh.qs};
    for (int j = 0; j < sh.nq; ++j) {
      const int q = sites[j], r = q / C, col = q % C;
      int cand[4] = {-1, -1, -1, -1};
      if (col > 0) cand[0] = hq_h[edge_h(c, r, col - 1)];
      if (col < C - 1) cand[1] = hq_h[edge_h(c, r, col)];
      if (r > 0) cand[2] = hq_v[edge_v(c, r - 1, col)];
      if (r < R - 1) cand[3] = hq_v[edge_v(c, r, col)];
      for (int a = 0; a < 4; ++a) {
        const int x = cand[a];
        if (x < 0) continue;
        bool have = false;
        for (int i = 0; i < sh.nq; ++i) have |= sites[i] == x;
        for (int i = 0; i < sh.nx; ++i) have |= sh.xq[i] == x;
        if (have) continue;
        if (sh.nx == 4) return fail(PEPS_EINVAL, "internal: too many operand variant bits");
        sh.xq[sh.nx++] = x;
      }
    }
    return PEPS_OK;
  };
  P.slice_list.clear();
  if (o.n_sliced > 0) {
    if (o.slice_ids) {
      for (int64_t i = 0; i < o.n_slice_ids; ++i) {
        if (o.n_sliced < 64 && (o.slice_ids[i] >> o.n_sliced) != 0)
          return fail(PEPS_EINVAL, "slice id %llu has bits beyond n_sliced",
                      (unsigned long long)o.slice_ids[i]);
        P.slice_list.push_back((int64_t)o.slice_ids[i]);
      }
      P.slice_ids.assign(o.slice_ids, o.slice_ids + o.n_slice_ids);
    } else {
      if (o.n_sliced > 24) return fail(PEPS_EINVAL, "pass slice_ids when n_sliced > 24");
      for (int64_t s = 0; s < ((int64_t)1 << o.n_sliced); ++s) P.slice_list.push_back(s);
    }
  } else {
    P.slice_list.push_back(0);
  }
  P.lower_mask = 0;
  P.lower_skip = odd && n == 1 && o.n_sliced > 0;
  if (P.lower_skip) {
    // the lower half holds rows R/2+1 .. R-1; a CZ touches it if either site does
    const int m = R / 2;
    for (int j = 0; j < o.n_sliced; ++j) {
      const CzPos &p = czpos[o.sliced_cz[j]];
      const int r0 = p.horiz ? p.edge / (C - 1) : p.edge / C;
      const int r1 = p.horiz ? r0 : r0 + 1;
      if (r0 > m || r1 > m) P.lower_mask |= 1ull << j;
    }
    // slices with equal lower bits next to one another (the sum's order only)
    const uint64_t lm = P.lower_mask;
    std::stable_sort(P.slice_list.begin(), P.slice_list.end(), [lm](int64_t a, int64_t b) {
      return ((uint64_t)a & lm) < ((uint64_t)b & lm);
    });
  }

  auto rdim_h = [&](int r, int col) -> int64_t {
    if (col < 0 || col >= C - 1) return 1;
    const int e = edge_h(c, r, col);
    const int64_t d = (int64_t)L.dim_h[e] >> popcount32(L.fix_h[e]);
    return dl ? d * d : d;
  };
  auto rdim_v = [&](int r, int col) -> int64_t {
    if (r < 0 || r >= R - 1) return 1;
    const int e = edge_v(c, r, col);
    const int64_t d = (int64_t)L.dim_v[e] >> popcount32(L.fix_v[e]);
    return dl ? d * d : d;
  };
  auto fdim_h = [&](int r, int col) -> int {
    return (col < 0 || col >= C - 1) ? 1 : L.dim_h[edge_h(c, r, col)];
  };
  auto fdim_v = [&](int r, int col) -> int {
    return (r < 0 || r >= R - 1) ? 1 : L.dim_v[edge_v(c, r, col)];
  };

  struct Block { int col, r0, nq; };
  std::vector<Block> blocks;
  struct Leg { int id; int64_t dim; };
  P.steps.clear();
  P.step_site.clear();
  P.step_opbase.clear();
  P.step_roles.clear();
  P.scheme = o.scheme;
  int64_t cap = 1;
  double flops = 0, bytes = 0;
  int n_ops_total = 0;
  if (!quad) {
    // ---- blocks: the sites each step absorbs ----
    // One site per step, except that (with fuse_rows == 0) the two top rows and
    // the two bottom rows of a column are absorbed together when that costs no
    // more multiply-adds and leaves the step enough output tiles (or no longer
    // a K) to fill the GPU: the top pair has no incoming vertical leg and the
    // bottom pair no outgoing one, so the pair's operand is no larger than the
    // largest single step's and the running tensor between the two rows is never
    // written.
    for (int col = 0; col < C; ++col) {
      const bool fuse = o.fuse_rows == 0 && R >= 4 && !dl;
      int r = 0;
      while (r < R) {
        int nq = 1;
        if (fuse && (r == 0 || r == R - 2)) {
          // cost of the pair vs its two single steps (dims at this column)
          const int64_t hl0 = rdim_h(r, col - 1), hl1 = rdim_h(r + 1, col - 1);
          const int64_t hr0 = rdim_h(r, col), hr1 = rdim_h(r + 1, col);
          const int64_t vin = rdim_v(r - 1, col), vmid = rdim_v(r, col), vout = rdim_v(r + 1, col);
          const double pair = (double)hl0 * hl1 * vin * hr0 * hr1 * vout;
          const double single = (double)hl0 * vin * hr0 * vmid * hl1 + (double)hr0 * hl1 * vmid * hr1 * vout;
          // a pair with few output tiles runs its whole K on a few CTAs: take
          // it only if its K is no longer than the two single steps' together
          double Mrest = 1;
          for (int rr = 0; rr < R; ++rr)
            if (rr < r) Mrest *= (double)rdim_h(rr, col);
            else if (rr > r + 1) Mrest *= (double)rdim_h(rr, col - 1);
          const double tiles = std::ceil(Mrest / 128.0) * std::ceil((double)(hr0 * hr1 * vout) / 64.0);
          const bool shallow = hl0 * hl1 * vin <= hl0 * vin + hl1 * vmid;
          if (pair <= single && (tiles >= 152 || shallow) && vmid <= kMaxMid) nq = 2;
        }
        blocks.push_back({col, r, nq});
        r += nq;
      }
    }

    // ---- step list of the column sweep (legs tracked by identity) ----
    // Before a block of rows r .. r+k-1 the running tensor's legs are, slowest
    // first, [h_{r+k} .. h_{R-1}, h'_0 .. h'_{r-1}, h_r .. h_{r+k-1}, v]; the
    // block's store moves the next block's k' legs (the slowest M legs) next to
    // v', which restores that form.  Leg ids: h-edge (r, col) -> 1000 + r*64 +
    // col + 1; v-leg -> 2 at the column ends (the bottom leg of column c and the
    // top leg of column c+1 are both of dim 1 and share the id).
    std::vector<Leg> legs;
    auto hid = [&](int r, int col) { return 1000 + r * 64 + (col + 1); };
    {
      const int k0 = blocks.empty() ? 1 : blocks[0].nq;
      for (int j = k0; j < R; ++j) legs.push_back({hid(j, -1), 1});
      for (int j = 0; j < k0; ++j) legs.push_back({hid(j, -1), 1});
      legs.push_back({2, 1});
    }
    for (size_t bi = 0; bi < blocks.size(); ++bi) {
      const Block &bk = blocks[bi];
      const int col = bk.col, r0 = bk.r0, k = bk.nq;
      const int knext = bi + 1 < blocks.size() ? blocks[bi + 1].nq : 0;
      const size_t nl = legs.size();
      for (int j = 0; j < k; ++j)
        if (legs[nl - 1 - k + j].id != hid(r0 + j, col - 1))
          return fail(PEPS_EINVAL, "internal: leg order broken at (%d,%d)", r0 + j, col);
      int64_t K = legs[nl - 1].dim;
      for (int j = 0; j < k; ++j) K *= legs[nl - 1 - k + j].dim;
      const size_t nM = nl - 1 - k;  // M legs: legs[0 .. nM)
      int64_t M = 1;
      for (size_t i = 0; i < nM; ++i) M *= legs[i].dim;
      int64_t dh = 1;
      for (int j = 0; j < k; ++j) dh *= rdim_h(r0 + j, col);
      const int64_t dv = rdim_v(r0 + k - 1, col);
      const int64_t N = dh * dv;
      const size_t kmove = std::min<size_t>((size_t)knext, nM);
      int64_t Pdim = 1;
      for (size_t i = 0; i < kmove; ++i) Pdim *= legs[i].dim;
      if (K > (1 << 20) || N > (1 << 20))
        return fail(PEPS_EUNSUPPORTED, "site operand too large at (%d,%d)", r0, col);
      StepShape sh{};
      sh.M = M;
      sh.K = (int)K;
      sh.N = (int)N;
      sh.P = Pdim;
      sh.dv_out = (int)dv;
      sh.dh_out = (int)dh;
      sh.q = r0 * C + col;
      sh.nq = k;
      sh.qs = C;
      sh.fmt = fmt;
      sh.target = scale_target(fmt);
      sh.Mr = M;
      if (int rc = set_variant_qubits(sh)) return rc;
      P.steps.push_back(sh);
      P.step_roles.push_back({0, 1, 2, 3});
      P.step_site.push_back(r0 * C + col);
      P.step_opbase.push_back(n_ops_total);
      n_ops_total += step_variants(sh);
      cap = std::max(cap, std::max(M * K, M * N));
      flops += 8.0 * (double)M * K * N;
      bytes += (double)bpe * (double)(M * K + M * N);
      std::vector<Leg> nlgs;
      for (size_t i = kmove; i < nM; ++i) nlgs.push_back(legs[i]);
      for (int j = 0; j < k; ++j) nlgs.push_back({hid(r0 + j, col), rdim_h(r0 + j, col)});
      for (size_t i = 0; i < kmove; ++i) nlgs.push_back(legs[i]);
      nlgs.push_back({r0 + k == R ? 2 : 3000 + r0 + k - 1, dv});
      legs.swap(nlgs);
    }

  } else {
    // ---- square partition (supplementary Fig. S2(b)) ----
    // Each quarter is swept column by column in its own coordinates (i, j),
    // starting from its lattice corner: ul transposed, bl transposed and
    // flipped in rows, ur flipped in columns, br flipped in both.  A site's
    // roles (l, r, u, d in the sweep) map to physical legs.  The open legs
    // toward the neighbouring quarters are: the d legs of the sweep's last
    // row (they join the batch, slowest, in sweep-column order) and the r legs
    // of its last column (the rest, in sweep-row order); a quarter tensor is
    // stored [batch][rest].  With these orientations
    //   F_ul = [row cut, rows 0..h-1][column cut, columns 0..w-1]
    //   F_bl = [row cut, rows R-1..h][column cut, columns 0..w-1]
    //   F_ur = [column cut, columns C-1..w][row cut, rows 0..h-1]
    //   F_br = [column cut, columns C-1..w][row cut, rows R-1..h]
    // so F_l = F_ul F_bl^T is [rows 0..h-1][rows R-1..h], Y = F_br F_l^T is
    // laid out as F_ur, and the amplitude is sum Y * F_ur.
    struct Orient { int t, fr, fc; };
    auto to_lattice = [&](const Orient &w, int i, int j, int &r, int &col) {
      const int r0 = w.t ? j : i, c0 = w.t ? i : j;
      r = w.fr ? R - 1 - r0 : r0;
      col = w.fc ? C - 1 - c0 : c0;
    };
    auto phys_leg = [](int r, int col, int r2, int c2) -> int {
      if (r2 == r && c2 == col - 1) return 0;
      if (r2 == r && c2 == col + 1) return 1;
      if (c2 == col && r2 == r - 1) return 2;
      return 3;
    };
    auto leg_rdim = [&](int r, int col, int a) -> int64_t {
      switch (a) {
        case 0: return rdim_h(r, col - 1);
        case 1: return rdim_h(r, col);
        case 2: return rdim_v(r - 1, col);
        default: return rdim_v(r, col);
      }
    };
    const int h = R / 2, w = C / 2;
    auto plan_quarter = [&](int qi, Orient ori, int Hs, int Ws) -> int {
      Plan::Quarter &Q = P.quarter[qi];
      Q.first = (int)P.steps.size();
      Q.span = 1;
      auto hs = [](int i, int j) { return 1000 + i * 64 + (j + 1); };
      const int VID = 2;
      static const int di[4] = {0, 0, -1, 1}, dj[4] = {-1, 1, 0, 0};
      // per sweep site: lattice index, roles, restricted dims by role
      struct SiteInfo { int q; std::array<int, 4> roles; int64_t rd[4]; };
      auto info = [&](int i, int j) {
        SiteInfo f{};
        int r, col;
        to_lattice(ori, i, j, r, col);
        f.q = r * C + col;
        for (int ro = 0; ro < 4; ++ro) {
          int r2, c2;
          to_lattice(ori, i + di[ro], j + dj[ro], r2, c2);
          f.roles[ro] = phys_leg(r, col, r2, c2);
          f.rd[ro] = leg_rdim(r, col, f.roles[ro]);
        }
        return f;
      };
      // blocks: the top two rows of a sweep column in one step where that costs
      // no more multiply-adds and stays parallel (the rule of the column
      // sweep); the last row (its open bottom leg joins the batch) stays single
      struct QBlock { int j, i0, k; };
      std::vector<QBlock> qb;
      {
        int64_t B = 1;
        for (int j = 0; j < Ws; ++j) {
          int i = 0;
          while (i < Hs) {
            int k = 1;
            if (o.fuse_rows == 0 && i == 0 && Hs >= 3 && !dl) {
              const SiteInfo a0 = info(0, j), a1 = info(1, j);
              const double hl0 = a0.rd[0], hl1 = a1.rd[0], hr0 = a0.rd[1], hr1 = a1.rd[1];
              const double vin = a0.rd[2], vmid = a0.rd[3], vout = a1.rd[3];
              double Mrest = (double)B;
              for (int ii = 2; ii < Hs; ++ii) Mrest *= (double)info(ii, j).rd[0];
              const double pair = hl0 * hl1 * vin * hr0 * hr1 * vout;
              const double single = hl0 * vin * hr0 * vmid * hl1 + hr0 * hl1 * vmid * hr1 * vout;
              const double tiles = std::ceil(Mrest / 128.0) * std::ceil(hr0 * hr1 * vout / 64.0);
              const bool shallow = hl0 * hl1 * vin <= hl0 * vin + hl1 * vmid;
              if (pair <= single && (tiles >= 152 || shallow) && vmid <= kMaxMid) k = 2;
            }
            qb.push_back({j, i, k});
            i += k;
          }
          B *= info(Hs - 1, j).rd[3];
        }
      }
      std::vector<Leg> legs;
      {
        const int k0 = qb[0].k;
        for (int k = k0; k < Hs; ++k) legs.push_back({hs(k, -1), 1});
        for (int k = 0; k < k0; ++k) legs.push_back({hs(k, -1), 1});
        legs.push_back({VID, 1});
      }
      int64_t B = 1;
      for (size_t bi = 0; bi < qb.size(); ++bi) {
        const int j = qb[bi].j, i0 = qb[bi].i0, k = qb[bi].k;
        const int knext = bi + 1 < qb.size() ? qb[bi + 1].k : 0;
        SiteInfo f[2];
        for (int t = 0; t < k; ++t) f[t] = info(i0 + t, j);
        const size_t nl = legs.size();
        for (int t = 0; t < k; ++t)
          if (legs[nl - 1 - k + t].id != hs(i0 + t, j - 1))
            return fail(PEPS_EINVAL, "internal: quarter %d leg order broken at (%d,%d)", qi, i0 + t, j);
        int64_t K = legs[nl - 1].dim, Kc = f[0].rd[2];
        for (int t = 0; t < k; ++t) {
          K *= legs[nl - 1 - k + t].dim;
          Kc *= f[t].rd[0];
        }
        if (K != Kc)
          return fail(PEPS_EINVAL, "internal: quarter %d leg dims disagree at (%d,%d)", qi, i0, j);
        const size_t nM = nl - 1 - k;
        int64_t Mr = 1;
        for (size_t t = 0; t < nM; ++t) Mr *= legs[t].dim;
        int64_t dh = 1;
        for (int t = 0; t < k; ++t) dh *= f[t].rd[1];
        const int64_t dv = f[k - 1].rd[3];
        const bool last = i0 + k == Hs;
        const size_t kmove = std::min<size_t>((size_t)knext, nM);
        int64_t Pd = 1;
        for (size_t t = 0; t < kmove; ++t) Pd *= legs[t].dim;
        if (K > (1 << 20) || dh * dv > (1 << 20))
          return fail(PEPS_EUNSUPPORTED, "site operand too large at site %d", f[0].q);
        StepShape sh{};
        sh.M = B * Mr;
        sh.K = (int)K;
        sh.N = (int)(dh * dv);
        sh.P = Pd;
        sh.dv_out = (int)dv;
        sh.dh_out = (int)dh;
        sh.q = f[0].q;
        sh.nq = k;
        sh.qs = k == 2 ? f[1].q - f[0].q : 0;   // lattice offset of the block's second site
        sh.fmt = fmt;
        sh.target = scale_target(fmt);
        sh.vb = last ? 1 : 0;
        // the open leg's store is contiguous in h' when nothing moves (P = 1):
        // order the operand's N with v' slowest there
        sh.nvs = (last && Pd == 1 && k == 1 && dh > 1) ? 1 : 0;
        sh.Mr = Mr;
        if (int rc = set_variant_qubits(sh)) return rc;
        P.steps.push_back(sh);
        P.step_roles.push_back(f[0].roles);   // one orientation: the same for both sites
        P.step_site.push_back(f[0].q);
        P.step_opbase.push_back(n_ops_total);
        n_ops_total += step_variants(sh);
        cap = std::max(cap, std::max(sh.M * K, sh.M * (int64_t)sh.N));
        Q.span = std::max(Q.span, std::max(sh.M * K, sh.M * (int64_t)sh.N));
        flops += 8.0 * (double)sh.M * K * sh.N;
        bytes += (double)bpe * (double)(sh.M * K + sh.M * (int64_t)sh.N);
        std::vector<Leg> nlgs;
        for (size_t t = kmove; t < nM; ++t) nlgs.push_back(legs[t]);
        for (int t = 0; t < k; ++t) nlgs.push_back({hs(i0 + t, j), f[t].rd[1]});
        for (size_t t = 0; t < kmove; ++t) nlgs.push_back(legs[t]);
        if (last) {
          B *= dv;
          nlgs.push_back({VID, 1});
        } else {
          nlgs.push_back({3000 + (i0 + k - 1) * 64 + j, dv});
        }
        legs.swap(nlgs);
      }
      // the rest legs are the last sweep column's r legs, in sweep-row order
      if (legs.size() != (size_t)Hs + 1)
        return fail(PEPS_EINVAL, "internal: quarter %d ends with %zu legs", qi, legs.size());
      Q.rest = 1;
      for (int i = 0; i < Hs; ++i) {
        if (legs[i].id != hs(i, Ws - 1))
          return fail(PEPS_EINVAL, "internal: quarter %d final leg order", qi);
        Q.rest *= legs[i].dim;
      }
      Q.rest_last = legs[Hs - 1].dim;
      Q.batch = B;
      Q.batch_last = info(Hs - 1, Ws - 1).rd[3];
      Q.count = (int)P.steps.size() - Q.first;
      return PEPS_OK;
    };
    auto merge_shape = [&](int64_t M, int64_t K, int64_t N) {
      StepShape sh{};
      sh.M = M;
      sh.K = (int)K;
      sh.N = (int)N;
      sh.P = 1;
      sh.dv_out = N % 8 == 0 ? 8 : 1;   // row-major store: dest = m N + n
      sh.dh_out = (int)(N / sh.dv_out);
      sh.q = 0;
      sh.nq = 0;
      sh.qs = 0;
      sh.fmt = fmt;
      sh.target = scale_target(fmt);
      sh.vb = 0;
      sh.Mr = M;
      return sh;
    };
    auto add_merge = [&](const StepShape &sh) {
      if (sh.K > (1 << 20) || sh.N > (1 << 20))
        return fail(PEPS_EUNSUPPORTED, "quarter merge operand too large (%d x %d)", sh.K, sh.N);
      P.steps.push_back(sh);
      P.step_roles.push_back({0, 1, 2, 3});
      P.step_site.push_back(-1);
      P.step_opbase.push_back(-1);  // set once the site operands are numbered
      cap = std::max(cap, std::max(sh.M * (int64_t)sh.K, sh.M * (int64_t)sh.N));
      flops += 8.0 * (double)sh.M * sh.K * sh.N;
      bytes += (double)bpe * (double)(sh.M * (int64_t)sh.K + sh.M * (int64_t)sh.N);
      P.max_kn_merge = std::max<int64_t>(P.max_kn_merge, (int64_t)sh.K * sh.N);
      return (int)PEPS_OK;
    };
    int rc;
    P.odd = odd;
    if (!odd) {
      if ((rc = plan_quarter(0, {1, 0, 0}, w, h))) return rc;   // ul
      if ((rc = plan_quarter(1, {1, 1, 0}, w, h))) return rc;   // bl
      const Plan::Quarter &ul = P.quarter[0], &bl = P.quarter[1];
      if (ul.rest != bl.rest) return fail(PEPS_EINVAL, "internal: ul / bl cut dims differ");
      P.s_m1 = (int)P.steps.size();
      if ((rc = add_merge(merge_shape(ul.batch, ul.rest, bl.batch)))) return rc;
      if ((rc = plan_quarter(2, {0, 0, 1}, h, w))) return rc;   // ur
      if ((rc = plan_quarter(3, {0, 1, 1}, h, w))) return rc;   // br
      const Plan::Quarter &ur = P.quarter[2], &br = P.quarter[3];
      if (br.rest != bl.batch || br.batch != ur.batch || ul.batch != ur.rest)
        return fail(PEPS_EINVAL, "internal: quarter cut dims differ");
      P.s_m2 = (int)P.steps.size();
      if ((rc = add_merge(merge_shape(br.batch, br.rest, ul.batch)))) return rc;
    } else {
      // odd side L = 2m+1 (Fig. S2(c)): ul = rows 0..m x cols 0..m-1, ur =
      // rows 0..m x cols m..2m (holds the centre site), bl = rows m+1..2m x
      // cols 0..m, br = rows m+1..2m x cols m+1..2m, each swept column by
      // column from its lattice corner, so that the horizontal cut is every
      // quarter's batch (its legs appear one per sweep column, from the first
      // column on: a sliced bit there shrinks the rest of the sweep):
      //   F_ul = [horizontal cut, cols 0..m-1][upper vertical cut, rows 0..m]
      //   F_ur = [horizontal cut, cols 2m..m][upper vertical cut, rows 0..m]
      //   F_bl = [horizontal cut, cols 0..m][lower vertical cut, rows 2m..m+1]
      //   F_br = [horizontal cut, cols 2m..m+1][lower vertical cut, rows 2m..m+1]
      // The larger quarter of each half (ur: 8 open legs, bl: 2m+1) is its
      // merge's A operand as stored, the other one the (transposed) B operand:
      //   F_u^T = F_ur F_ul^T,  F_b = F_bl F_br^T,
      // both written as [col m][cols 0..m-1][cols 2m..m+1], and the amplitude
      // is their dot product: the paper's order (upper-left with upper-right,
      // bottom-left with bottom-right, then the halves).
      const int m = R / 2;
      if ((rc = plan_quarter(0, {0, 0, 0}, m + 1, m))) return rc;       // ul
      if ((rc = plan_quarter(2, {0, 0, 1}, m + 1, m + 1))) return rc;   // ur
      const Plan::Quarter &ul = P.quarter[0], &ur = P.quarter[2];
      if (ul.rest != ur.rest) return fail(PEPS_EINVAL, "internal: ul / ur cut dims differ");
      // F_u^T rows are (cols 2m..m+1, col m), its columns cols 0..m-1; stored
      // [col m][cols 0..m-1][cols 2m..m+1] by the epilogue's permuted store
      // (m_lo = col m, m_hi = cols 2m..m+1, h' = the whole N)
      P.s_m1 = (int)P.steps.size();
      {
        StepShape sh = merge_shape(ur.batch, ur.rest, ul.batch);
        sh.P = ur.batch / ur.batch_last;
        sh.dh_out = (int)ul.batch;
        sh.dv_out = 1;
        if ((rc = add_merge(sh))) return rc;
      }
      if ((rc = plan_quarter(1, {0, 1, 0}, m, m + 1))) return rc;       // bl
      if ((rc = plan_quarter(3, {0, 1, 1}, m, m))) return rc;           // br
      const Plan::Quarter &bl = P.quarter[1], &br = P.quarter[3];
      if (bl.rest != br.rest) return fail(PEPS_EINVAL, "internal: bl / br cut dims differ");
      if (ul.batch * ur.batch != bl.batch * br.batch || ur.batch_last != bl.batch_last)
        return fail(PEPS_EINVAL, "internal: the halves' cut dims differ");
      // F_b = F_bl F_br^T: rows (cols 0..m-1, col m), columns cols 2m..m+1;
      // the same order (m_lo = col m, m_hi = cols 0..m-1, v' = the whole N)
      P.s_m2 = (int)P.steps.size();
      {
        StepShape sh = merge_shape(bl.batch, bl.rest, br.batch);
        sh.P = bl.batch / bl.batch_last;
        sh.dh_out = 1;
        sh.dv_out = (int)br.batch;
        if ((rc = add_merge(sh))) return rc;
      }
    }
    P.n_site_ops = n_ops_total;   // merge operands: placed once glanes is known
  }
  if (!quad) P.n_site_ops = n_ops_total;
  // tensor-core accumulation.  An FP32 accumulator that the tensor core adds
  // into loses about an ulp of its own magnitude per MMA, so adding the split
  // form's small correction products (hi*lo, lo*hi, 2^-11 of the main ones)
  // into the main accumulator costs twice the error of the main products
  // themselves.  Automatic (0): steps with K >= 2048 real (the merges, the
  // fused bottom pairs) give the corrections an accumulator of their own, and
  // so does every step of a chain longer than 32 steps (the error adds up
  // along the chain; a short-K step then keeps its epilogue overlap with half
  // the tile width).  tc_ksplit = k >= 1 forces k K segments on every step and
  // no separate corrections; -1 separates them on every step (measurement).
  const bool long_chain = P.steps.size() > 32;
  for (auto &sh : P.steps) {
    if (o.tc_ksplit == 0 || o.tc_ksplit == -1) {
      sh.ksplit = 1;
      sh.csep = (o.tc_ksplit == -1 || long_chain || 2LL * sh.K >= 2048) ? 1 : 0;
    } else {
      sh.ksplit = o.tc_ksplit;
      sh.csep = 0;
    }
  }
  if (cap > ((int64_t)1 << 36) && !(o.flags & PEPS_FLAG_ESTIMATE))
    return fail(PEPS_EUNSUPPORTED, "running tensor too large (%lld entries)", (long long)cap);
  if (ws && (o.flags & PEPS_FLAG_ESTIMATE))
    return fail(PEPS_EINVAL, "PEPS_FLAG_ESTIMATE is for planning queries only");
  P.cap = cap;
  P.n_steps = (int)P.steps.size();
  P.flops_per_slice = flops;
  P.bytes_per_slice = bytes;
  // two-plane formats: the lo plane starts 1 KiB-aligned after the hi plane
  if (fmt == FMT_BF16X2 || fmt == FMT_FP16X2) {
    const size_t plane_bytes = align_up((size_t)cap * 4, 1024);
    P.plane = (int64_t)plane_bytes / 2;
    P.gbuf_bytes = 2 * plane_bytes;
  } else {
    P.plane = 0;
    P.gbuf_bytes = align_up((size_t)cap * bpe, 1024);
  }
  P.odd_bytes = 0;
  if (quad && P.odd) {
    // odd side: one bitstring at a time, so each sweep pair gets its own
    // size.  The lower half (bl, br -> F_b) runs first; only F_b, in a buffer
    // of its own, outlives it, so the upper half's pairs (ul, which also
    // holds F_u^T, and ur) reuse the lower half's memory.  All hi planes
    // first, every lo plane at the same offset behind them.
    const bool two = fmt == FMT_BF16X2 || fmt == FMT_FP16X2;
    const size_t pe = two ? 4 : (size_t)bpe;
    const StepShape &m1 = P.steps[P.s_m1], &m2 = P.steps[P.s_m2];
    const int64_t span[4] = {std::max(P.quarter[0].span, m1.M * (int64_t)m1.N), P.quarter[2].span,
                             P.quarter[1].span, P.quarter[3].span};
    size_t top = 0, bot = 0;
    for (int b = 0; b < 4; ++b) {
      P.obuf_off[b] = top;
      top = align_up(top + pe * (size_t)span[b / 2], 1024);
      P.obuf_off[4 + b] = bot;
      bot = align_up(bot + pe * (size_t)span[2 + b / 2], 1024);
    }
    P.obuf_fb = std::max(top, bot);
    const size_t o2 = align_up(P.obuf_fb + pe * (size_t)(m2.M * (int64_t)m2.N), 1024);
    P.plane = two ? (int64_t)o2 / 2 : 0;
    P.odd_bytes = two ? 2 * o2 : o2;
  }
  for (auto &s : P.steps) s.plane = P.plane;

  // ---- lanes ----
  const int pc = o.prefix_cols;
  // steps of the shared prefix: the blocks of columns 0 .. pc-1
  int pre_steps = 0;
  for (const auto &bk : blocks)
    if (bk.col < pc) ++pre_steps;
  // square partition: a group shares the left half (F_l); without prefix
  // reuse every bitstring is a group of one
  int64_t gs = pc > 0 ? o.prefix_group : (quad ? 1 : std::max<int64_t>(n, 1));
  P.n_groups = ((pc > 0 || quad) && n > 0) ? (int)(n / gs) : 0;
  P.bufs_per_lane = quad ? 4 : 2;
  // one launch for the sweeps of a small lattice: every running tensor and
  // operand fits one block's shared memory (FP32 arithmetic: the FP32 form
  // and the split forms, whose results it matches)
  P.small = false;
  if (!quad && pc == 0 && !(o.flags & PEPS_FLAG_STEPWISE) &&
      (fmt == FMT_F32 || fmt == FMT_FP16X2 || fmt == FMT_BF16X2)) {
    int64_t cg = 1, ce = 1;
    for (auto &sh : P.steps) {
      cg = std::max(cg, std::max(sh.M * sh.K, sh.M * (int64_t)sh.N));
      ce = std::max(ce, (int64_t)sh.K * sh.N);
    }
    if ((2 * cg + ce) * (int64_t)sizeof(float2) <= (int64_t)kSmallSweepMaxSmem) {
      P.small = true;
      P.small_cap_g = (int)cg;
      P.small_cap_e = (int)ce;
    }
  }
  int lanes = o.max_lanes > 0 ? o.max_lanes : 16;
  // square partition: the left quarters of up to this many groups share a
  // launch, and the members of those groups may share their lanes' launches
  P.glanes = (int)std::min<int64_t>(lanes, std::max<int64_t>(P.n_groups, 1));
  if (quad) {
    // the merge operands: one slot per group of a chunk (even side), one
    // otherwise
    P.merge_slots = (!odd && P.n_groups > 0) ? P.glanes : 1;
    P.op_m1 = n_ops_total;
    P.op_m2 = n_ops_total + P.merge_slots;
    n_ops_total += 2 * P.merge_slots;
    P.step_opbase[P.s_m1] = P.op_m1;
    P.step_opbase[P.s_m2] = P.op_m2;
  }
  const int64_t span = (quad && !odd) ? gs * P.glanes : gs;
  lanes = (int)std::min<int64_t>(lanes, std::max<int64_t>(std::min<int64_t>(n, span), 1));
  P.lanes = lanes;

  // ---- site tensors ----
  std::vector<int> sd(4 * NQ);
  P.site_elems.assign(NQ, 0);
  for (int q = 0; q < NQ; ++q) {
    const int r = q / C, col = q % C;
    sd[4 * q + 0] = fdim_h(r, col - 1);
    sd[4 * q + 1] = fdim_h(r, col);
    sd[4 * q + 2] = fdim_v(r - 1, col);
    sd[4 * q + 3] = fdim_v(r, col);
    P.site_elems[q] = 2LL * sd[4 * q] * sd[4 * q + 1] * sd[4 * q + 2] * sd[4 * q + 3];
  }

  // ---- workspace layout ----
  size_t off = 0;
  P.off_status = off; off = align_up(off + sizeof(DeviceStatus));
  for (int b = 0; b < 2; ++b) P.site_buf_off[b].assign(NQ, 0);
  for (int q = 0; q < NQ; ++q)
    for (int b = 0; b < 2; ++b) {
      P.site_buf_off[b][q] = off;  // hi plane, then lo plane (float-float)
      off = align_up(off + 2 * (size_t)P.site_elems[q] * sizeof(float2));
    }
  P.off_site_ptrs = off; off = align_up(off + NQ * sizeof(float2 *));
  P.off_site_lo = off; off = align_up(off + NQ * sizeof(int64_t));

  // evolution schedule (needs only offsets)
  std::vector<Gate1Entry> g1;
  std::vector<CzEntry> cz;
  std::vector<Gate2Entry> g2e;
  P.evo.clear();
  std::vector<std::vector<EvoRef>> site_refs(NQ);
  std::vector<std::vector<int>> site_ref_batch(NQ);   // the batch of each reference
  {
    std::vector<int> cur(NQ, 0);
    std::vector<int> dims(4 * NQ, 1);
    std::vector<int> in_batch(NQ, -1);
    int batch_id = -1, batch_kind = -1;
    auto site_ptr = [&](int q, int b) -> float2 * {
      return (float2 *)((char *)ws + P.site_buf_off[b][q]);
    };
    auto start_batch = [&](int kind) {
      Plan::EvoBatch eb{};
      eb.kind = kind;
      eb.off = kind == 0 ? (int64_t)g1.size() : kind == 1 ? (int64_t)cz.size() : (int64_t)g2e.size();
      eb.n = 0;
      eb.max_work = 0;
      P.evo.push_back(eb);
      batch_id = (int)P.evo.size() - 1;
      batch_kind = kind;
    };
    for (auto &g : c->gates) {
      const int kind = g.kind;
      bool clash = batch_kind != kind;
      if (!clash) {
        if (in_batch[g.q0] == batch_id) clash = true;
        if (kind != 0 && in_batch[g.q1] == batch_id) clash = true;
      }
      if (clash || batch_id < 0) start_batch(kind);
      Plan::EvoBatch &eb = P.evo[batch_id];
      if (kind == 0) {
        const int q = g.q0;
        Gate1Entry e{};
        e.A = site_ptr(q, cur[q]);
        e.half = (int64_t)dims[4 * q] * dims[4 * q + 1] * dims[4 * q + 2] * dims[4 * q + 3];
        e.lo_off = P.site_elems[q];
        for (int i = 0; i < 4; ++i) {
          const float hr = (float)g.U[2 * i], hi_ = (float)g.U[2 * i + 1];
          e.U_hi[i] = make_float2(hr, hi_);
          e.U_lo[i] = make_float2((float)(g.U[2 * i] - (double)hr),
                                  (float)(g.U[2 * i + 1] - (double)hi_));
        }
        site_refs[q].push_back(EvoRef{0, (int32_t)g1.size()});
        site_ref_batch[q].push_back(batch_id);
        g1.push_back(e);
        eb.n++;
        eb.max_work = std::max(eb.max_work, e.half);
        in_batch[q] = batch_id;
      } else if (kind == 2) {
        // general two-qubit gate: W0 on the lower site, W1 on the other; the
        // shared leg grows by the rank (s fastest)
        const bool horiz = g.horiz != 0;
        const int qs[2] = {g.q0, g.q1};
        const int axes[2] = {horiz ? 1 : 3, horiz ? 0 : 2};
        for (int side = 0; side < 2; ++side) {
          const int q = qs[side];
          Gate2Entry e{};
          e.in = site_ptr(q, cur[q]);
          e.out = site_ptr(q, cur[q] ^ 1);
          e.lo_off = P.site_elems[q];
          for (int a = 0; a < 4; ++a) e.dims[a] = dims[4 * q + a];
          e.axis = axes[side];
          e.chi = g.chi;
          for (int k = 0; k < g.chi; ++k)
            for (int i = 0; i < 4; ++i) {
              const std::complex<double> w = side ? g.W1[k][i] : g.W0[k][i];
              const float hr = (float)w.real(), hi_ = (float)w.imag();
              e.W_hi[k][i] = make_float2(hr, hi_);
              e.W_lo[k][i] = make_float2((float)(w.real() - (double)hr), (float)(w.imag() - (double)hi_));
            }
          dims[4 * q + e.axis] *= g.chi;
          const int64_t out_n =
              2LL * dims[4 * q] * dims[4 * q + 1] * dims[4 * q + 2] * dims[4 * q + 3];
          cur[q] ^= 1;
          site_refs[q].push_back(EvoRef{2, (int32_t)g2e.size()});
          site_ref_batch[q].push_back(batch_id);
          g2e.push_back(e);
          eb.n++;
          eb.max_work = std::max(eb.max_work, out_n);
          in_batch[q] = batch_id;
        }
      } else {
        const bool horiz = g.horiz != 0;
        const int qs[2] = {g.q0, g.q1};
        const int axes[2] = {horiz ? 1 : 3, horiz ? 0 : 2};
        for (int side = 0; side < 2; ++side) {
          const int q = qs[side];
          CzEntry e{};
          e.in = site_ptr(q, cur[q]);
          e.out = site_ptr(q, cur[q] ^ 1);
          e.lo_off = P.site_elems[q];
          for (int a = 0; a < 4; ++a) e.dims[a] = dims[4 * q + a];
          e.axis = axes[side];
          e.kind = side;  // projector on the lower q, phase on the other
          e.fixed_s = -1;
          e.pad_ = 0;
          dims[4 * q + e.axis] *= 2;
          const int64_t out_n =
              2LL * dims[4 * q] * dims[4 * q + 1] * dims[4 * q + 2] * dims[4 * q + 3];
          cur[q] ^= 1;
          site_refs[q].push_back(EvoRef{1, (int32_t)cz.size()});
          site_ref_batch[q].push_back(batch_id);
          cz.push_back(e);
          eb.n++;
          eb.max_work = std::max(eb.max_work, out_n);
          in_batch[q] = batch_id;
        }
      }
    }
    P.final_buf = cur;
    for (int q = 0; q < NQ; ++q)
      for (int a = 0; a < 4; ++a)
        if (dims[4 * q + a] != sd[4 * q + a])
          return fail(PEPS_EINVAL, "internal: evolution dims mismatch at site %d", q);
  }
  P.off_g1 = off; off = align_up(off + std::max<size_t>(g1.size(), 1) * sizeof(Gate1Entry));
  P.off_cz = off; off = align_up(off + std::max<size_t>(cz.size(), 1) * sizeof(CzEntry));
  P.off_g2 = off; off = align_up(off + std::max<size_t>(g2e.size(), 1) * sizeof(Gate2Entry));
  // The evolution's leading gate batches, while every site tensor they touch
  // is small enough for one block (16384 entries), run as one launch with a
  // block per site (each site evolves through its own gate halves only); the
  // rest one launch per batch.  All of it in that launch when every site
  // tensor stays small.
  P.evo_prefix = 0;
  if (!(o.flags & PEPS_FLAG_STEPWISE))
    while (P.evo_prefix < (int)P.evo.size() && P.evo[P.evo_prefix].max_work <= 16384)
      ++P.evo_prefix;
  P.evo_sites = P.evo_prefix == (int)P.evo.size();
  std::vector<EvoRef> evo_refs;
  std::vector<int32_t> evo_first(NQ + 1, 0);
  for (int q = 0; q < NQ; ++q) {
    evo_first[q] = (int32_t)evo_refs.size();
    for (size_t i = 0; i < site_refs[q].size(); ++i)
      if (site_ref_batch[q][i] < P.evo_prefix) evo_refs.push_back(site_refs[q][i]);
  }
  evo_first[NQ] = (int32_t)evo_refs.size();
  P.off_evo_refs = off; off = align_up(off + std::max<size_t>(evo_refs.size(), 1) * sizeof(EvoRef));
  P.off_evo_first = off; off = align_up(off + (size_t)(NQ + 1) * sizeof(int32_t));
  P.off_ops_begin = off;

  // operands (restricted dims): 2^nq variants per step
  const int n_ops = n_ops_total;
  if (n_ops > 65535) return fail(PEPS_EUNSUPPORTED, "too many site operands (%d)", n_ops);
  P.n_ops = n_ops;
  P.ec_off.assign(n_ops, 0);
  P.bt_off[0].assign(n_ops, 0);
  P.bt_off[1].assign(n_ops, 0);
  P.max_kn = 1;
  P.max_kn2 = 1;
  const bool want_tc = o.precision != PEPS_FP32_SIMT && !(o.flags & PEPS_FLAG_NO_TC);
  int64_t n1 = 0, n2 = 0;
  for (int s = 0; s < P.n_steps; ++s) {
    const StepShape &sh = P.steps[s];
    if (sh.nq == 1) {
      P.max_kn = std::max<int>(P.max_kn, sh.K * sh.N);
      n1 += step_variants(sh);
    } else if (sh.nq == 2) {
      P.max_kn2 = std::max<int>(P.max_kn2, sh.K * sh.N);
      n2 += step_variants(sh);
    }  // nq == 0: a merge operand, built from a stored tensor during the call
    // a tensor-core merge builds its planes straight from the stored tensor
    const bool merge_tc = sh.nq == 0 && want_tc && tc_supports(sh, fmt);
    for (int t = 0; t < op_slots(P, s); ++t) {
      const int op = P.step_opbase[s] + t;
      P.ec_off[op] = 0;
      if (!merge_tc) {
        P.ec_off[op] = off;
        off = align_up(off + (size_t)sh.K * (size_t)sh.N * sizeof(float2), 1024);
      }
      if (want_tc && tc_supports(sh, fmt)) {
        const size_t planes = (fmt == FMT_BF16X2 || fmt == FMT_FP16X2) ? 2 : 1;
        const size_t esz = (fmt == FMT_TF32) ? 4 : 2;
        const size_t pb = (size_t)tc_Kr_pad(sh.K) * tc_Nr_pad(sh.N) * esz;
        for (size_t p = 0; p < planes; ++p) {
          P.bt_off[p][op] = off;
          off = align_up(off + pb, 1024);
        }
      }
    }
  }
  P.off_opdesc = off; off = align_up(off + n_ops * sizeof(OpDesc));
  P.n_opbuild_per_slice = n1;
  P.n_obe2_per_slice = n2;
  P.off_opbuild = off;
  off = align_up(off + (size_t)std::max<int64_t>(n1, 1) * P.slice_list.size() * sizeof(OpBuildEntry));
  P.off_opbuild2 = off;
  off = align_up(off + (size_t)std::max<int64_t>(n2, 1) * P.slice_list.size() * sizeof(OpBuild2Entry));

  // records: chains = groups + bitstrings
  P.n_recs = (int)((P.n_groups + n) * P.n_steps);
  P.off_recs = off; off = align_up(off + std::max<size_t>(P.n_recs, 1) * sizeof(Rec));

  // launches + items
  std::vector<StepItem> items;
  std::vector<FinalEntry> fins;
  P.launches.clear();
  const size_t lane_off_rel = 0;  // filled below
  (void)lane_off_rel;
  // buffers are placed after all tables; compute their offsets after sizing
  // the item arrays, using relative positions first.
  struct Pending { int64_t first_item; };
  const int64_t NS = P.n_steps;
  // Relative buffer addresses, resolved once the table sizes are known.
  const int BPL = P.bufs_per_lane;
  auto lane_buf = [&](int lane, int b) -> size_t {
    return (size_t)(BPL * lane + b) * P.gbuf_bytes;
  };
  auto pre_buf = [&](int b) -> size_t { return (size_t)(BPL * P.lanes + b) * P.gbuf_bytes; };
  // square partition: group g's buffers, laid out like a lane's after the lanes'
  auto grp_buf = [&](int g, int b) -> size_t {
    return (size_t)(BPL * (P.lanes + g) + b) * P.gbuf_bytes;
  };
  const size_t REL = (size_t)1 << 62;  // marker: relative to the buffer area
  struct RelItem { size_t a, d; bool a_unit; int64_t bit; };
  std::vector<RelItem> rel;
  auto add_step_launch = [&](int s, std::vector<StepItem> its, const std::vector<RelItem> &rs,
                             int a_lanes) {
    Launch ln{};
    ln.kind = 0;
    ln.step = s;
    ln.shape = P.steps[s];
    ln.tc = want_tc && tc_supports(P.steps[s], fmt);
    ln.a_base_rel = rs[0].a;
    ln.a_lanes = a_lanes;
    ln.op_base = P.step_opbase[s];
    for (size_t i = 0; i < its.size(); ++i) its[i].a_lane = a_lanes > 1 ? (int)i : 0;
    ln.items_off = (int64_t)items.size();
    ln.n_items = (int)its.size();
    ln.flops = 8.0 * (double)ln.shape.M * ln.shape.K * ln.shape.N * ln.n_items;
    ln.bytes = (double)bpe * (double)(ln.shape.M * ln.shape.K + ln.shape.M * ln.shape.N) * ln.n_items;
    items.insert(items.end(), its.begin(), its.end());
    rel.insert(rel.end(), rs.begin(), rs.end());
    P.launches.push_back(ln);
  };
  std::vector<TensorOpEntry> tops;
  std::vector<DotEntry> dots;
  if (quad) {
    // per group: ul and bl sweeps, F_bl -> operand, F_l = F_ul F_bl^T, F_l ->
    // operand; per chunk of member lanes: ur and br sweeps, Y = F_br F_l^T,
    // amplitude += sum Y * F_ur.  Group buffers 0-1 hold the ul sweep, 2-3 the
    // bl sweep and then F_l; lane buffers 0-1 the ur sweep, 2-3 the br sweep
    // and then Y.
    const Plan::Quarter &ul = P.quarter[0], &bl = P.quarter[1], &ur = P.quarter[2],
                        &br = P.quarter[3];
    // steps of one sweep on `nl` lanes: chains ch(l), bitstrings bit(l), buffers
    // buf(l, 0..1) (ping-pong); returns the buffer index (0/1) of the result
    auto sweep = [&](const Plan::Quarter &Q, int nl, auto chain_of, auto bit_of, auto buf_of) {
      for (int k = 0; k < Q.count; ++k) {
        const int s = Q.first + k;
        std::vector<StepItem> its;
        std::vector<RelItem> rs;
        for (int l = 0; l < nl; ++l) {
          const int64_t ch = chain_of(l);
          StepItem it{};
          it.op_base = P.step_opbase[s];
          it.in_rec = k == 0 ? -1 : (int)(ch * NS + s - 1);
          it.out_rec = (int)(ch * NS + s);
          RelItem ri{k == 0 ? 0 : buf_of(l, (k - 1) % 2), buf_of(l, k % 2), k == 0, bit_of(l)};
          its.push_back(it);
          rs.push_back(ri);
        }
        add_step_launch(s, its, rs, k == 0 ? 1 : nl);
      }
      return (Q.count - 1) % 2;
    };
    auto tensor_op = [&](size_t g_rel, int64_t K, int64_t N, int64_t ns, int rec, int op,
                         int consumer) {
      TensorOpEntry t{};
      t.G = (const void *)(REL + g_rel);
      t.ks = 1;
      t.ns = ns;
      t.ns_hi = 0;
      t.Nlo = N;
      t.K = (int)K;
      t.N = (int)N;
      t.rec = rec;
      t.op = op;
      t.target = scale_target(fmt);
      // operands of the same merge step for consecutive slots, one after the
      // other, share a launch
      if (!P.launches.empty()) {
        Launch &pl = P.launches.back();
        if (pl.kind == 2 && pl.step == consumer && pl.op + pl.n_aux == op &&
            pl.aux_off + pl.n_aux == (int64_t)tops.size() && pl.kn == K * N) {
          tops.push_back(t);
          ++pl.n_aux;
          return;
        }
      }
      Launch ln{};
      ln.kind = 2;
      ln.step = consumer;
      ln.aux_off = (int64_t)tops.size();
      ln.n_aux = 1;
      ln.op = op;
      ln.kn = K * N;
      ln.shape = P.steps[consumer];
      ln.tc = want_tc && tc_supports(P.steps[consumer], fmt);
      ln.flops = ln.bytes = 0;
      tops.push_back(t);
      P.launches.push_back(ln);
    };
    if (P.odd) {
      // per bitstring: bl, br -> F_b; ul, ur -> F_u^T; amplitude = F_u^T . F_b.
      // One bitstring at a time in sized buffers: ul 0-1 (then F_u^T), ur 2-3,
      // bl 4-5, br 6-7 (the lower half's, under the upper half's), F_b.
      auto ob = [&](int b) -> size_t { return P.obuf_off[b]; };
      for (int64_t i = 0; i < n; ++i) {
        const int64_t chain = i;
        auto ch = [&](int) { return chain; };
        auto bit = [&](int) { return i; };
        const size_t lower_first = P.launches.size();
        const int bbl = sweep(bl, 1, ch, bit, [&](int, int b) { return ob(4 + b); });
        const int bbr = sweep(br, 1, ch, bit, [&](int, int b) { return ob(6 + b); });
        const int rec_bl = (int)(chain * NS + bl.first + bl.count - 1);
        const int rec_br = (int)(chain * NS + br.first + br.count - 1);
        const int rec_b = (int)(chain * NS + P.s_m2);
        // Ec[k][n] = F_br[n K + k]
        tensor_op(ob(6 + bbr), br.rest, br.batch, br.rest, rec_br, P.op_m2, P.s_m2);
        {
          StepItem it{};
          it.op_base = P.op_m2;
          it.in_rec = rec_bl;
          it.out_rec = rec_b;
          RelItem ri{ob(4 + bbl), P.obuf_fb, false, i};
          add_step_launch(P.s_m2, {it}, {ri}, 1);
        }
        for (size_t li = lower_first; li < P.launches.size(); ++li) {
          P.launches[li].lower = true;
          if (P.launches[li].kind == 0) P.flops_lower += P.launches[li].flops;
        }
        const int bul = sweep(ul, 1, ch, bit, [&](int, int b) { return ob(b); });
        const int bur = sweep(ur, 1, ch, bit, [&](int, int b) { return ob(2 + b); });
        const int rec_ul = (int)(chain * NS + ul.first + ul.count - 1);
        const int rec_ur = (int)(chain * NS + ur.first + ur.count - 1);
        const int rec_u = (int)(chain * NS + P.s_m1);
        // Ec[k][n] = F_ul[n K + k]
        tensor_op(ob(bul), ul.rest, ul.batch, ul.rest, rec_ul, P.op_m1, P.s_m1);
        {
          StepItem it{};
          it.op_base = P.op_m1;
          it.in_rec = rec_ur;
          it.out_rec = rec_u;
          RelItem ri{ob(2 + bur), ob(bul ^ 1), false, i};
          add_step_launch(P.s_m1, {it}, {ri}, 1);
        }
        Launch dl{};
        dl.kind = 3;
        dl.aux_off = (int64_t)dots.size();
        dl.n_aux = 1;
        dl.flops = dl.bytes = 0;
        DotEntry d{};
        d.Y = (const void *)(REL + ob(bul ^ 1));
        d.F = (const void *)(REL + P.obuf_fb);
        d.n = ur.batch * ul.batch;
        d.rec_y = rec_u;
        d.rec_f = rec_b;
        d.out_index = (int)i;
        d.nslots = kDotBlocks;
        dots.push_back(d);
        P.launches.push_back(dl);
      }
    }
    // Groups in chunks of glanes (a lane per group; group slot j's four
    // buffers sit after the member lanes' with the same per-lane layout):
    // their left quarters swept together; F_bl of every group turned into its
    // merge operand (slot op_m1 + j); the groups' left halves
    // F_l = F_ul F_bl^T merged in one launch and kept in the groups' buffers,
    // each then turned into the group's operand of the last merge (slot
    // op_m2 + j).  Then the chunk's members in chunks of `lanes` bitstrings
    // (which may span groups): their right quarters swept together, and one
    // launch of the merges Y = F_br F_l^T of all of them, each against its
    // group's operand, with the dot product against F_ur.
    const int G = P.odd ? 0 : P.n_groups;
    for (int g0 = 0; g0 < G; g0 += P.glanes) {
      const int gc = std::min(P.glanes, G - g0);
      auto gch = [&](int l) { return (int64_t)(g0 + l); };
      auto gbit = [&](int l) { return (int64_t)(g0 + l) * gs; };
      const int bul = sweep(ul, gc, gch, gbit, [&](int l, int b) { return grp_buf(l, b); });
      const int bbl = sweep(bl, gc, gch, gbit, [&](int l, int b) { return grp_buf(l, 2 + b); });
      std::vector<StepItem> mits;
      std::vector<RelItem> mrs;
      for (int j = 0; j < gc; ++j) {
        const int64_t chain = g0 + j, first = chain * gs;
        const int rec_ul = (int)(chain * NS + ul.first + ul.count - 1);
        const int rec_bl = (int)(chain * NS + bl.first + bl.count - 1);
        const int rec_l = (int)(chain * NS + P.s_m1);
        tensor_op(grp_buf(j, 2 + bbl), bl.rest, bl.batch, bl.rest, rec_bl, P.op_m1 + j, P.s_m1);
        StepItem it{};
        it.op_base = P.op_m1 + j;
        it.b_slot = j;
        it.in_rec = rec_ul;
        it.out_rec = rec_l;
        mits.push_back(it);
        mrs.push_back(RelItem{grp_buf(j, bul), grp_buf(j, 2 + (bbl ^ 1)), false, first});
      }
      add_step_launch(P.s_m1, mits, mrs, gc);
      for (int j = 0; j < gc; ++j) {
        // F_l = [a][b] (N of the first merge = bl.batch per row); operand Ec[b][a]
        const int rec_l = (int)((g0 + j) * NS + P.s_m1);
        tensor_op(grp_buf(j, 2 + (bbl ^ 1)), bl.batch, ul.batch, bl.batch, rec_l, P.op_m2 + j,
                  P.s_m2);
      }
      const int64_t m0 = (int64_t)g0 * gs, mcount = (int64_t)gc * gs;
      // on the tensor cores the merge's epilogue forms the dot product with
      // F_ur itself (Y is never stored): its items point at F_ur
      const bool fuse = want_tc && tc_supports(P.steps[P.s_m2], fmt);
      for (int64_t base = 0; base < mcount; base += P.lanes) {
        const int nl = (int)std::min<int64_t>(P.lanes, mcount - base);
        auto mch = [&](int l) { return (int64_t)P.n_groups + m0 + base + l; };
        auto mbit = [&](int l) { return m0 + base + l; };
        const int bur = sweep(ur, nl, mch, mbit, [&](int l, int b) { return lane_buf(l, b); });
        const int bbr = sweep(br, nl, mch, mbit, [&](int l, int b) { return lane_buf(l, 2 + b); });
        std::vector<StepItem> its;
        std::vector<RelItem> rs;
        for (int l = 0; l < nl; ++l) {
          const int64_t ch = mch(l);
          const int j = (int)((m0 + base + l) / gs - g0);
          StepItem it{};
          it.op_base = P.op_m2 + j;
          it.b_slot = j;
          it.in_rec = (int)(ch * NS + br.first + br.count - 1);
          it.out_rec = (int)(ch * NS + P.s_m2);
          its.push_back(it);
          rs.push_back(RelItem{lane_buf(l, 2 + bbr),
                               fuse ? lane_buf(l, bur) : lane_buf(l, 2 + (bbr ^ 1)), false,
                               mbit(l)});
        }
        add_step_launch(P.s_m2, its, rs, nl);
        if (fuse) P.launches.back().shape.dot = 1;
        Launch dl{};
        dl.kind = 3;
        dl.aux_off = (int64_t)dots.size();
        dl.n_aux = nl;
        dl.flops = dl.bytes = 0;
        if (P.launches.back().shape.dot) dl.fused_merge = (int)P.launches.size() - 1;
        for (int l = 0; l < nl; ++l) {
          const int64_t ch = mch(l);
          DotEntry d{};
          d.Y = (const void *)(REL + lane_buf(l, 2 + (bbr ^ 1)));
          d.F = (const void *)(REL + lane_buf(l, bur));
          d.n = ur.batch * ur.rest;
          d.rec_y = (int)(ch * NS + P.s_m2);
          d.rec_f = (int)(ch * NS + ur.first + ur.count - 1);
          d.out_index = (int)mbit(l);
          d.nslots = kDotBlocks;   // fused: set once the merge's tiles are known
          dots.push_back(d);
        }
        P.launches.push_back(dl);
      }
    }
  } else if (pc > 0) {
    for (int g = 0; g < P.n_groups; ++g) {
      const int chain = g;
      for (int s = 0; s < pre_steps; ++s) {
        StepItem it{};
        it.op_base = P.step_opbase[s];
        it.in_rec = s == 0 ? -1 : (int)(chain * NS + s - 1);
        it.out_rec = (int)(chain * NS + s);
        RelItem ri{s == 0 ? 0 : pre_buf((s - 1) % 2), pre_buf(s % 2), s == 0, (int64_t)g * gs};
        add_step_launch(s, {it}, {ri}, 1);
      }
      const size_t pre_out = pre_buf((pre_steps - 1) % 2);
      for (int64_t base = 0; base < gs; base += P.lanes) {
        const int nl = (int)std::min<int64_t>(P.lanes, gs - base);
        for (int s = pre_steps; s < NS; ++s) {
          std::vector<StepItem> its;
          std::vector<RelItem> rs;
          for (int l = 0; l < nl; ++l) {
            const int64_t i = (int64_t)g * gs + base + l;
            const int64_t ch = P.n_groups + i;
            StepItem it{};
            it.op_base = P.step_opbase[s];
            it.in_rec = s == pre_steps ? (int)(chain * NS + pre_steps - 1) : (int)(ch * NS + s - 1);
            it.out_rec = (int)(ch * NS + s);
            RelItem ri{s == pre_steps ? pre_out : lane_buf(l, (s - 1 - pre_steps) % 2),
                       lane_buf(l, (s - pre_steps) % 2), false, i};
            its.push_back(it);
            rs.push_back(ri);
          }
          add_step_launch(s, its, rs, s == pre_steps ? 1 : nl);
        }
        Launch fl{};
        fl.kind = 1;
        fl.fin_off = (int64_t)fins.size();
        fl.n_fin = nl;
        for (int l = 0; l < nl; ++l) {
          const int64_t i = (int64_t)g * gs + base + l;
          FinalEntry f{};
          f.G = (const void *)(REL + lane_buf(l, (NS - 1 - pre_steps) % 2));
          f.rec = (int)((P.n_groups + i) * NS + NS - 1);
          f.out_index = (int)i;
          fins.push_back(f);
        }
        P.launches.push_back(fl);
      }
    }
  } else if (P.small) {
    Launch ln{};
    ln.kind = 0;
    ln.small = true;
    ln.shape = P.steps[0];
    ln.tc = false;
    ln.items_off = 0;
    ln.n_items = 0;
    ln.flops = P.flops_per_slice * (double)n;
    ln.bytes = P.bytes_per_slice * (double)n;
    P.launches.push_back(ln);
  } else {
    for (int64_t base = 0; base < n; base += P.lanes) {
      const int nl = (int)std::min<int64_t>(P.lanes, n - base);
      for (int s = 0; s < NS; ++s) {
        std::vector<StepItem> its;
        std::vector<RelItem> rs;
        for (int l = 0; l < nl; ++l) {
          const int64_t i = base + l;
          StepItem it{};
          it.op_base = P.step_opbase[s];
          it.in_rec = s == 0 ? -1 : (int)(i * NS + s - 1);
          it.out_rec = (int)(i * NS + s);
          RelItem ri{s == 0 ? 0 : lane_buf(l, (s - 1) % 2), lane_buf(l, s % 2), s == 0, i};
          its.push_back(it);
          rs.push_back(ri);
        }
        add_step_launch(s, its, rs, nl);
      }
      Launch fl{};
      fl.kind = 1;
      fl.fin_off = (int64_t)fins.size();
      fl.n_fin = nl;
      for (int l = 0; l < nl; ++l) {
        const int64_t i = base + l;
        FinalEntry f{};
        f.G = (const void *)(REL + lane_buf(l, (NS - 1) % 2));
        f.rec = (int)(i * NS + NS - 1);
        f.out_index = (int)i;
        fins.push_back(f);
      }
      P.launches.push_back(fl);
    }
  }
  P.off_items = off; off = align_up(off + std::max<size_t>(items.size(), 1) * sizeof(StepItem));
  P.off_fin = off; off = align_up(off + std::max<size_t>(fins.size(), 1) * sizeof(FinalEntry));
  P.off_tops = off; off = align_up(off + std::max<size_t>(tops.size(), 1) * sizeof(TensorOpEntry));
  P.off_dots = off; off = align_up(off + std::max<size_t>(dots.size(), 1) * sizeof(DotEntry));
  P.off_partials = off;
  {
    // per lane: the separate dot kernel's blocks, or a fused merge's slots
    // (at most ceil(M / 128) x (2N / 16) tiles x 4 warps)
    size_t per_lane = kDotBlocks;
    if (quad && !P.odd) {
      const StepShape &m2 = P.steps[P.s_m2];
      per_lane = std::max(per_lane, (size_t)((m2.M + 127) / 128) * (size_t)(2 * m2.N / 16) * 4);
    }
    off = align_up(off + (quad ? per_lane * P.lanes * sizeof(double2) : 16));
  }
  P.off_small_steps = off; off = align_up(off + (size_t)std::max(NS, (int64_t)1) * sizeof(StepShape));
  P.off_small_opbase = off; off = align_up(off + (size_t)std::max(NS, (int64_t)1) * sizeof(int32_t));
  P.off_acc = off; off = align_up(off + std::max<int64_t>(n, 1) * sizeof(double2));
  P.off_bits = off; off = align_up(off + std::max<int64_t>(n, 1) * sizeof(uint64_t));
  P.off_out = off; off = align_up(off + std::max<int64_t>(n, 1) * sizeof(peps_c128));
  P.off_tables_end = off;
  off = align_up(off, 4096);
  P.lane_off = off;
  const int n_gbufs = P.small ? 0
                      : quad ? 4 * P.lanes + 4 * P.glanes
                             : 2 * P.lanes + (pc > 0 ? 2 : 0);
  off += (quad && P.odd) ? P.odd_bytes : (size_t)n_gbufs * P.gbuf_bytes;
  P.need = off;
  if (!ws) return PEPS_OK;
  if (ws_bytes < P.need)
    return fail(PEPS_ENOMEM, "workspace too small: %zu bytes given, %zu needed", ws_bytes, P.need);

  // ---- resolve addresses and assemble the table blob ----
  char *base = (char *)ws;
  const uint64_t *bsrc = host_bits ? (const uint64_t *)(base + P.off_bits) : bits_dev;
  P.small_bits = bsrc;
  for (size_t i = 0; i < items.size(); ++i) {
    items[i].bits = bsrc + rel[i].bit;
    items[i].A = rel[i].a_unit ? nullptr : (const void *)(base + P.lane_off + rel[i].a);
    items[i].D = (void *)(base + P.lane_off + rel[i].d);
  }
  for (auto &f : fins) f.G = (const void *)(base + P.lane_off + ((size_t)f.G - REL));
  for (auto &t : tops) t.G = (const void *)(base + P.lane_off + ((size_t)t.G - REL));
  for (auto &d : dots) {
    d.Y = (const void *)(base + P.lane_off + ((size_t)d.Y - REL));
    d.F = (const void *)(base + P.lane_off + ((size_t)d.F - REL));
  }
  for (auto &l : P.launches) {
    if (l.kind != 0 || !l.tc) continue;
    const int q = l.shape.q;
    const int ob = l.op_base;
    // the variants' planes are equally spaced (allocated one after another
    // with the same padded size)
    const int nv = op_slots(P, l.step);
    const void *bb[2];
    for (int pl = 0; pl < 2; ++pl)
      bb[pl] = P.bt_off[pl][ob] ? (const void *)(base + P.bt_off[pl][ob])
                                : (const void *)(base + P.bt_off[0][ob]);
    const int64_t vst = nv > 1 ? (int64_t)(P.bt_off[0][ob + 1] - P.bt_off[0][ob]) : 0;
    for (int t = 1; t < nv; ++t)
      for (int pl = 0; pl < 2; ++pl)
        if (P.bt_off[pl][ob] &&
            (int64_t)(P.bt_off[pl][ob + t] - P.bt_off[pl][ob]) != (int64_t)t * vst)
          return fail(PEPS_EINVAL, "internal: operand variants not equally spaced at site %d", q);
    int rc = tc_prepare(l.shape, fmt, base + P.lane_off + l.a_base_rel, l.a_lanes,
                        (int64_t)(BPL * P.gbuf_bytes), P.plane * 2, bb, nv, vst, o.tc_kchunk,
                        o.tc_cluster, o.tc_epi, &l.tc_handle);
    if (rc != 0)
      return fail(PEPS_ECUDA, "tensor-map encoding failed (%d) for the step at site %d", rc, q);
  }
  // fused dots: the merge's partial-sum slots per item
  for (auto &l : P.launches) {
    if (l.kind != 3 || l.fused_merge < 0) continue;
    const int slots = tc_dot_slots(P.launches[l.fused_merge].tc_handle);
    for (int k = 0; k < l.n_aux; ++k) dots[l.aux_off + k].nslots = slots;
  }

  std::vector<OpDesc> ops(n_ops);
  for (int s = 0; s < P.n_steps; ++s) {
    const StepShape &sh = P.steps[s];
    for (int t = 0; t < op_slots(P, s); ++t) {
      const int op = P.step_opbase[s] + t;
      OpDesc d{};
      d.Ec = P.ec_off[op] ? (const float2 *)(base + P.ec_off[op]) : nullptr;
      d.Bt[0] = P.bt_off[0][op] ? (const void *)(base + P.bt_off[0][op]) : nullptr;
      d.Bt[1] = P.bt_off[1][op] ? (const void *)(base + P.bt_off[1][op]) : nullptr;
      d.b_t = operand_scale_exp(fmt);
      d.K = sh.K;
      d.N = sh.N;
      ops[op] = d;
    }
  }
  // operand build entries per slice: one per (step, variant)
  std::vector<OpBuildEntry> obe;
  std::vector<OpBuild2Entry> obe2;
  for (int64_t sid : P.slice_list) {
    // fixed values of every edge for this slice
    std::vector<uint32_t> val_h = fixval_h, val_v = fixval_v;
    for (int j = 0; j < o.n_sliced; ++j) {
      const CzPos &p = czpos[o.sliced_cz[j]];
      if ((sid >> j) & 1) (p.horiz ? val_h[p.edge] : val_v[p.edge]) |= 1u << p.bit;
    }
    // the projected tensor of site q for bit t, legs restricted to the slice
    // roles[ro] = physical leg (0..3 = l, r, u, d) that plays role ro of the
    // absorbing sweep (identity for the column sweep)
    // xv: output bits of the operand variant (bit qq = output bit of qubit
    // qq; only the variant's qubits are set), which select the held values
    auto site_entry = [&](int q, int t, int op, const std::array<int, 4> &roles, uint64_t xv) {
      const int r = q / C, col = q % C;
      OpBuildEntry e;
      std::memset(&e, 0, sizeof e);   // padding too: entries are compared bytewise
      const int fb = P.final_buf[q];
      e.A = (const float2 *)(base + P.site_buf_off[fb][q]);
      e.lo_off = P.site_elems[q];
      // physical legs: l = h(r, col-1), r = h(r, col), u = v(r-1, col), d = v(r, col)
      int32_t pd[4], prd[4];
      uint32_t pfm[4], pfv[4];
      const Links *plk[4] = {nullptr, nullptr, nullptr, nullptr};
      auto leg = [&](int a, bool horiz, int rr, int cc) {
        bool inside = horiz ? (cc >= 0 && cc < C - 1) : (rr >= 0 && rr < R - 1);
        uint32_t fm = 0, fv = 0;
        if (inside) {
          const int eidx = horiz ? edge_h(c, rr, cc) : edge_v(c, rr, cc);
          fm = horiz ? L.fix_h[eidx] : L.fix_v[eidx];
          fv = horiz ? val_h[eidx] : val_v[eidx];
          if (hold) {
            const int hq = horiz ? hq_h[eidx] : hq_v[eidx];
            const bool one = hq >= 0 && ((xv >> hq) & 1ull);
            fv |= one ? (horiz ? hv1_h[eidx] : hv1_v[eidx]) : (horiz ? hv0_h[eidx] : hv0_v[eidx]);
            plk[a] = horiz ? &lk_h[eidx] : &lk_v[eidx];
          }
        }
        pd[a] = sd[4 * q + a];
        // nothing fixed on this leg: the restricted index is the index
        pfm[a] = fm ? (uint32_t)(pd[a] - 1) & ~fm : 0xFFFFFFFFu;
        pfv[a] = fv;
        prd[a] = pd[a] >> popcount32(fm);
      };
      leg(0, true, r, col - 1);
      leg(1, true, r, col);
      leg(2, false, r - 1, col);
      leg(3, false, r, col);
      // element strides of the physical layout [sigma][l][r][u][d]
      const int64_t pst[4] = {(int64_t)pd[1] * pd[2] * pd[3], (int64_t)pd[2] * pd[3], pd[3], 1};
      for (int ro = 0; ro < 4; ++ro) {
        const int a = roles[ro];
        e.dims[ro] = pd[a];
        e.rdims[ro] = prd[a];
        e.free_mask[ro] = pfm[a];
        e.fixed_val[ro] = pfv[a];
        e.stride[ro] = pst[a];
        e.n_links[ro] = 0;
        if (plk[a])
          for (const auto &pr : *plk[a]) {
            e.link_src[ro][e.n_links[ro]] = (uint8_t)pr.first;
            e.link_dst[ro][e.n_links[ro]] = (uint8_t)pr.second;
            ++e.n_links[ro];
          }
      }
      e.tau_stride = (int64_t)pd[0] * pd[1] * pd[2] * pd[3];
      e.tau = t;
      e.op = op;
      if (dl) {
        // double layer: sigma fixed to tau on a measured qubit, summed otherwise
        e.dl = ((o.measured_mask >> q) & 1ull) ? 1 : 2;
        for (int ro = 0; ro < 4; ++ro) e.rdims[ro] = e.dims[ro] * e.dims[ro];
      }
      return e;
    };
    for (int s = 0; s < P.n_steps; ++s) {
      const StepShape &sh = P.steps[s];
      const int ob = P.step_opbase[s];
      // output bits of variant v (the inverse of block_variant)
      auto variant_bits = [&](int v) {
        uint64_t xv = 0;
        for (int j = 0; j < sh.nq; ++j)
          if ((v >> j) & 1) xv |= 1ull << (sh.q + j * sh.qs);
        for (int i = 0; i < sh.nx; ++i)
          if ((v >> (sh.nq + i)) & 1) xv |= 1ull << sh.xq[i];
        return xv;
      };
      if (sh.nq == 1) {
        for (int v = 0; v < step_variants(sh); ++v) {
          OpBuildEntry e = site_entry(sh.q, v & 1, ob + v, P.step_roles[s], variant_bits(v));
          e.nvs = sh.nvs;
          obe.push_back(e);
        }
      } else if (sh.nq == 2) {
        // the block's sites are q and q + qs (qs = C for the column sweep; a
        // quarter's orientation can make it -C or +-1), same roles for both
        for (int v = 0; v < step_variants(sh); ++v) {
          OpBuild2Entry e2{};
          const uint64_t xv = variant_bits(v);
          e2.a = site_entry(sh.q, v & 1, ob + v, P.step_roles[s], xv);
          e2.b = site_entry(sh.q + sh.qs, (v >> 1) & 1, ob + v, P.step_roles[s], xv);
          e2.op = ob + v;
          obe2.push_back(e2);
        }
      }
    }
  }
  // keep, for each slice after the first, only the entries that change
  {
    const size_t n1 = (size_t)P.n_opbuild_per_slice, n2 = (size_t)P.n_obe2_per_slice;
    const size_t ns = P.slice_list.size();
    std::vector<OpBuildEntry> c1;
    std::vector<OpBuild2Entry> c2;
    P.obe_first.assign(ns, 0);
    P.obe_count.assign(ns, 0);
    P.obe2_first.assign(ns, 0);
    P.obe2_count.assign(ns, 0);
    for (size_t si = 0; si < ns; ++si) {
      P.obe_first[si] = (int64_t)c1.size();
      for (size_t j = 0; j < n1; ++j) {
        const OpBuildEntry &e = obe[si * n1 + j];
        if (si == 0 || std::memcmp(&e, &obe[(si - 1) * n1 + j], sizeof(OpBuildEntry)) != 0)
          c1.push_back(e);
      }
      P.obe_count[si] = (int64_t)c1.size() - P.obe_first[si];
      P.obe2_first[si] = (int64_t)c2.size();
      for (size_t j = 0; j < n2; ++j) {
        const OpBuild2Entry &e = obe2[si * n2 + j];
        if (si == 0 || std::memcmp(&e, &obe2[(si - 1) * n2 + j], sizeof(OpBuild2Entry)) != 0)
          c2.push_back(e);
      }
      P.obe2_count[si] = (int64_t)c2.size() - P.obe2_first[si];
    }
    obe.swap(c1);
    obe2.swap(c2);
  }

  std::vector<float2 *> site_ptrs(NQ);
  for (int q = 0; q < NQ; ++q) site_ptrs[q] = (float2 *)(base + P.site_buf_off[0][q]);

  const size_t part_a = P.off_ops_begin - P.off_site_ptrs;
  P.blob.assign(part_a + (P.off_tables_end - P.off_opdesc), 0);
  auto put = [&](size_t off_abs, const void *src, size_t nbytes) {
    if (!nbytes) return;
    const size_t at = off_abs < P.off_ops_begin ? off_abs - P.off_site_ptrs
                                                : part_a + (off_abs - P.off_opdesc);
    std::memcpy(P.blob.data() + at, src, nbytes);
  };
  put(P.off_site_ptrs, site_ptrs.data(), NQ * sizeof(float2 *));
  put(P.off_site_lo, P.site_elems.data(), NQ * sizeof(int64_t));
  put(P.off_g1, g1.data(), g1.size() * sizeof(Gate1Entry));
  put(P.off_cz, cz.data(), cz.size() * sizeof(CzEntry));
  put(P.off_g2, g2e.data(), g2e.size() * sizeof(Gate2Entry));
  put(P.off_evo_refs, evo_refs.data(), evo_refs.size() * sizeof(EvoRef));
  put(P.off_evo_first, evo_first.data(), evo_first.size() * sizeof(int32_t));
  put(P.off_small_steps, P.steps.data(), P.steps.size() * sizeof(StepShape));
  put(P.off_small_opbase, P.step_opbase.data(), P.step_opbase.size() * sizeof(int32_t));
  put(P.off_opdesc, ops.data(), ops.size() * sizeof(OpDesc));
  put(P.off_opbuild, obe.data(), obe.size() * sizeof(OpBuildEntry));
  put(P.off_opbuild2, obe2.data(), obe2.size() * sizeof(OpBuild2Entry));
  put(P.off_items, items.data(), items.size() * sizeof(StepItem));
  put(P.off_fin, fins.data(), fins.size() * sizeof(FinalEntry));
  put(P.off_tops, tops.data(), tops.size() * sizeof(TensorOpEntry));
  put(P.off_dots, dots.data(), dots.size() * sizeof(DotEntry));
  return PEPS_OK;
}

// Slices of the call that run the lower half (odd side): the first, and every
// one whose lower bits differ from the slice before it.
static int64_t lower_runs(const Plan &P) {
  const int64_t ns = (int64_t)P.slice_list.size();
  if (!P.lower_skip) return ns;
  int64_t k = ns > 0 ? 1 : 0;
  for (int64_t si = 1; si < ns; ++si)
    if ((((uint64_t)P.slice_list[si] ^ (uint64_t)P.slice_list[si - 1]) & P.lower_mask) != 0) ++k;
  return k;
}

extern "C" int peps_workspace_bytes(const peps_ctx *c, int64_t n, const peps_opts *opts,
                                    size_t *bytes) {
  if (!c || !bytes) return fail(PEPS_EINVAL, "peps_workspace_bytes: NULL argument");
  peps_opts o{};
  if (opts) o = *opts;
  Plan P;
  int rc = build_plan(const_cast<peps_ctx *>(c), n, o, nullptr, 0, nullptr, false, P);
  if (rc) return rc;
  *bytes = P.need;
  return PEPS_OK;
}

extern "C" int peps_plan_info_get(const peps_ctx *c, int64_t n, const peps_opts *opts,
                                  peps_plan_info *info) {
  if (!c || !info) return fail(PEPS_EINVAL, "peps_plan_info_get: NULL argument");
  peps_opts o{};
  if (opts) o = *opts;
  Plan P;
  int rc = build_plan(const_cast<peps_ctx *>(c), n, o, nullptr, 0, nullptr, false, P);
  if (rc) return rc;
  peps_plan_info I{};
  I.n_steps = P.n_steps;
  I.max_entries = P.cap;
  I.flops_per_chain = P.flops_per_slice;
  I.bytes_per_chain = P.bytes_per_slice;
  I.n_slices = (int64_t)P.slice_list.size();
  const int64_t nl = lower_runs(P);
  for (auto &l : P.launches) {
    if (l.kind != 0) continue;
    const int64_t k = l.lower ? nl : I.n_slices;
    I.flops_call += (double)k * l.flops;
    I.bytes_call += (double)k * l.bytes;
    I.n_launches += k;
    I.n_tc_launches += l.tc ? k : 0;
  }
  I.lanes = P.lanes;
  I.flops_lower = P.flops_lower;
  I.n_lower_bits = P.lower_skip ? popcount64(P.lower_mask) : o.n_sliced;
  *info = I;
  return PEPS_OK;
}

extern "C" int peps_plan_steps(const peps_ctx *c, int64_t n, const peps_opts *opts,
                               peps_step_info *steps, int64_t cap, int64_t *n_out) {
  if (!c || !n_out) return fail(PEPS_EINVAL, "peps_plan_steps: NULL argument");
  if (cap < 0 || (cap > 0 && !steps)) return fail(PEPS_EINVAL, "peps_plan_steps: bad output array");
  peps_opts o{};
  if (opts) o = *opts;
  Plan P;
  int rc = build_plan(const_cast<peps_ctx *>(c), n, o, nullptr, 0, nullptr, false, P);
  if (rc) return rc;
  const bool want_tc = o.precision != PEPS_FP32_SIMT && !(o.flags & PEPS_FLAG_NO_TC);
  const int64_t ns = (int64_t)P.slice_list.size(), nl = lower_runs(P);
  std::vector<peps_step_info> out(P.n_steps);
  for (int s = 0; s < P.n_steps; ++s) {
    const StepShape &sh = P.steps[s];
    peps_step_info &i = out[s];
    i.M = sh.M;
    i.K = sh.K;
    i.N = sh.N;
    i.sites = sh.nq;
    i.variants = step_variants(sh);
    i.P = sh.P;
    i.Mr = sh.Mr > 0 ? sh.Mr : sh.M;
    i.dv = sh.dv_out;
    i.dh = sh.dh_out;
    i.open_leg = sh.vb;
    i.fused_dot = sh.dot;
    i.tensor_cores = (!P.small && want_tc && tc_supports(sh, P.fmt)) ? 1 : 0;
    i.part = -1;
    if (P.scheme == PEPS_SCHEME_QUADRANTS) {
      i.part = 4;
      for (int qi = 0; qi < 4; ++qi)
        if (s >= P.quarter[qi].first && s < P.quarter[qi].first + P.quarter[qi].count) i.part = qi;
    }
  }
  // launches and flops per step (a whole-sweep launch counts for no step's
  // launches but carries every step's flops)
  for (auto &l : P.launches) {
    if (l.kind != 0) continue;
    const int64_t k = l.lower ? nl : ns;
    if (l.small) {
      for (int s = 0; s < P.n_steps; ++s)
        out[s].flops += (double)k * 8.0 * (double)P.steps[s].M * P.steps[s].K * P.steps[s].N *
                        (double)P.n;
      continue;
    }
    if (l.step >= 0 && l.step < P.n_steps) {
      out[l.step].launches += k;
      out[l.step].flops += (double)k * l.flops;
      if (l.shape.dot) out[l.step].fused_dot = 1;
    }
  }
  for (int64_t s = 0; s < std::min<int64_t>(cap, P.n_steps); ++s) steps[s] = out[s];
  *n_out = P.n_steps;
  return PEPS_OK;
}

// ---------------------------------------------------------------------------
// Execution
// ---------------------------------------------------------------------------
static int ensure_events(peps_ctx *c, size_t n) {
  while (c->ev.size() < n) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  return PEPS_OK;
}

// Launch counters of one graph replay (the same sequence as an eager call
// with the evolution included).
static int enqueue_sequence_stats_only(Plan &P, peps_stats &S) {
  S.launches_evolve = 1 + (int64_t)P.evo.size() - P.evo_prefix;
  if (P.opts.prefix_cols > 0 && P.n > 0) S.launches_finalize++;
  bool any_tc = false;
  for (auto &l : P.launches) any_tc |= (l.kind == 0 && l.tc);
  const int64_t ns = (int64_t)P.slice_list.size();
  S.launches_operand = ns * (1 + (any_tc ? 1 : 0));
  for (int64_t si = 0; si < ns; ++si)
    S.launches_operand += (P.obe_count[si] > 0 ? 1 : 0) + (P.obe2_count[si] > 0 ? 1 : 0);
  const int64_t nl = lower_runs(P);
  for (auto &l : P.launches) {
    const int64_t k = l.lower ? nl : ns;
    if (l.kind == 0) {
      S.launches_contract += k;
      S.contract_flops += k * l.flops;
      S.contract_bytes += k * l.bytes;
      if (l.tc) {
        S.launches_contract_tc += k;
        S.contract_tc_flops += k * l.flops;
        S.contract_tc_bytes += k * l.bytes;
      }
    } else if (l.kind == 2) {
      S.launches_operand += k * (l.tc ? 3 : 2);
    } else if (l.kind == 3) {
      S.launches_finalize += (l.fused_merge >= 0 ? 1 : 2) * k;
    } else {
      S.launches_finalize += k;
    }
  }
  S.launches_total = S.launches_evolve + S.launches_operand + S.launches_contract + S.launches_finalize;
  return PEPS_OK;
}

// Enqueue the whole call on `s`: status reset, evolution (if `rebuild`), the
// prefix-group check, and per slice the operand build, the absorption steps
// and the final reduction.  With `timing`, CUDA events bracket every
// contraction launch (their count goes to *n_timed, the index of each timed
// launch in P.launches to timed_idx).
static int enqueue_sequence(peps_ctx *c, Plan &P, const uint64_t *d_bits_in, cudaStream_t s,
                            bool rebuild, bool timing, peps_stats &S, size_t *n_timed,
                            std::vector<int> *timed_idx, bool capturing = false) {
  // inside a stream capture an event record becomes a graph node only when
  // recorded as an external event (a plain record orders streams)
  auto record = [&](cudaEvent_t e) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                     : cudaEventRecord(e, s);
  };
  char *base = (char *)P.ws;
  DeviceStatus *st = (DeviceStatus *)(base + P.off_status);
  const int64_t wd_ns = P.opts.watchdog_ns > 0 ? P.opts.watchdog_ns : 2000000000LL;
  CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DeviceStatus), s));
  if (rebuild) {
    // the leading batches (sites initialised there too), then the rest
    if (P.evo_prefix > 0)
      CUDA_TRY(launch_evolve_sites((const Gate1Entry *)(base + P.off_g1),
                                   (const CzEntry *)(base + P.off_cz),
                                   (const Gate2Entry *)(base + P.off_g2),
                                   (const EvoRef *)(base + P.off_evo_refs),
                                   (const int32_t *)(base + P.off_evo_first),
                                   (float2 *const *)(base + P.off_site_ptrs),
                                   (const int64_t *)(base + P.off_site_lo), c->n, st, s));
    else
      CUDA_TRY(launch_init_sites((float2 *const *)(base + P.off_site_ptrs),
                                 (const int64_t *)(base + P.off_site_lo), c->n, st, s));
    S.launches_evolve++;
    for (size_t bi = (size_t)P.evo_prefix; bi < P.evo.size(); ++bi) {
      const Plan::EvoBatch &eb = P.evo[bi];
      if (eb.kind == 0)
        CUDA_TRY(launch_gate1((const Gate1Entry *)(base + P.off_g1) + eb.off, eb.n, eb.max_work, s));
      else if (eb.kind == 1)
        CUDA_TRY(launch_cz((const CzEntry *)(base + P.off_cz) + eb.off, eb.n, eb.max_work, s));
      else
        CUDA_TRY(launch_gate2((const Gate2Entry *)(base + P.off_g2) + eb.off, eb.n, eb.max_work, s));
      S.launches_evolve++;
    }
  } else {
    // status block still needs its unit scalars
    CUDA_TRY(launch_init_sites((float2 *const *)(base + P.off_site_ptrs),
                               (const int64_t *)(base + P.off_site_lo), 0, st, s));
    S.launches_evolve++;
  }
  if (P.opts.prefix_cols > 0 && P.n > 0) {
    uint64_t mask = 0;
    for (int q = 0; q < c->n; ++q)
      if (q % c->C < P.opts.prefix_cols) mask |= 1ull << q;
    CUDA_TRY(launch_check_groups(d_bits_in, P.n, P.opts.prefix_group, mask, st, s));
    S.launches_finalize++;
  }
  double2 *acc = (double2 *)(base + P.off_acc);
  CUDA_TRY(cudaMemsetAsync(acc, 0, std::max<int64_t>(P.n, 1) * sizeof(double2), s));
  Rec *recs = (Rec *)(base + P.off_recs);
  OpDesc *ops = (OpDesc *)(base + P.off_opdesc);
  const StepItem *items = (const StepItem *)(base + P.off_items);
  const FinalEntry *fins = (const FinalEntry *)(base + P.off_fin);
  const OpBuildEntry *obe = (const OpBuildEntry *)(base + P.off_opbuild);
  const OpBuild2Entry *obe2 = (const OpBuild2Entry *)(base + P.off_opbuild2);
  const TensorOpEntry *tops = (const TensorOpEntry *)(base + P.off_tops);
  const DotEntry *dots = (const DotEntry *)(base + P.off_dots);
  double2 *partials = (double2 *)(base + P.off_partials);
  bool any_tc = false;
  for (auto &l : P.launches) any_tc |= (l.kind == 0 && l.tc);
  for (size_t si = 0; si < P.slice_list.size(); ++si) {
    // odd side: the lower half (and F_b's records, the steps after s_m1) stays
    // when this slice's lower bits equal the previous slice's
    const bool skip_lower = P.lower_skip && si > 0 &&
                            (((uint64_t)P.slice_list[si] ^ (uint64_t)P.slice_list[si - 1]) &
                             P.lower_mask) == 0;
    const int64_t n_clear = skip_lower ? (int64_t)P.s_m1 + 1 : P.n_recs;
    if (n_clear > 0) CUDA_TRY(cudaMemsetAsync(recs, 0, n_clear * sizeof(Rec), s));
    // operands whose restriction is unchanged since the previous slice stay
    const OpBuildEntry *e = obe + P.obe_first[si];
    const OpBuild2Entry *e2 = obe2 + P.obe2_first[si];
    if (P.obe_count[si] > 0) {
      CUDA_TRY(launch_build_operands(e, (int)P.obe_count[si], P.max_kn, ops, s));
      S.launches_operand++;
    }
    if (P.obe2_count[si] > 0) {
      CUDA_TRY(launch_build_operands2(e2, (int)P.obe2_count[si], P.max_kn2, ops, s));
      S.launches_operand++;
    }
    CUDA_TRY(launch_operand_bounds(P.n_site_ops, ops, s));
    S.launches_operand++;
    if (any_tc) {
      CUDA_TRY(launch_build_tc_operands(P.n_site_ops, std::max(P.max_kn, P.max_kn2), ops, P.fmt, s));
      S.launches_operand++;
    }
    for (auto &l : P.launches) {
      if (skip_lower && l.lower) continue;
      if (l.kind == 0) {
        if (timing) CUDA_TRY(record(c->ev[2 * *n_timed]));
        if (l.small) {
          SmallSweep sw{};
          sw.steps = (const StepShape *)(base + P.off_small_steps);
          sw.op_base = (const int32_t *)(base + P.off_small_opbase);
          sw.ops = ops;
          sw.bits = P.small_bits;
          sw.acc = acc;
          sw.n = P.n;
          sw.n_steps = P.n_steps;
          sw.cap_g = P.small_cap_g;
          sw.cap_e = P.small_cap_e;
          CUDA_TRY(launch_sweep_small(sw, c->sm_count, s));
        } else if (l.tc) {
          CUDA_TRY(launch_contract_tc(l.tc_handle, items + l.items_off, l.n_items, ops, recs,
                                      st, wd_ns, c->sm_count, s, l.shape.dot ? partials : nullptr));
          S.launches_contract_tc++;
          S.contract_tc_flops += l.flops;
          S.contract_tc_bytes += l.bytes;
        } else {
          CUDA_TRY(launch_contract_simt(l.shape, items + l.items_off, l.n_items, ops, recs, st, s));
        }
        if (timing) {
          CUDA_TRY(record(c->ev[2 * *n_timed + 1]));
          timed_idx->push_back((int)(&l - P.launches.data()));
          ++*n_timed;
        }
        S.launches_contract++;
        S.contract_flops += l.flops;
        S.contract_bytes += l.bytes;
      } else if (l.kind == 2) {
        // a merge operand from a stored tensor: for the tensor cores its bound
        // and planes straight from the tensor, else Ec and its bound
        if (l.tc) {
          CUDA_TRY(launch_tensor_operand_tc(tops + l.aux_off, l.n_aux, l.shape.K, l.shape.N, P.fmt,
                                            P.plane, ops, recs, s));
          S.launches_operand += 3;
        } else {
          CUDA_TRY(launch_tensor_operand(tops + l.aux_off, l.n_aux, l.kn, P.fmt, P.plane, ops, recs,
                                         s));
          CUDA_TRY(launch_operand_bounds(l.n_aux, ops + l.op, s, l.shape.N));
          S.launches_operand += 2;
        }
      } else if (l.kind == 3 && l.fused_merge >= 0) {
        CUDA_TRY(launch_dot_final(dots + l.aux_off, l.n_aux, recs, partials, acc, s));
        S.launches_finalize += 1;
      } else if (l.kind == 3) {
        CUDA_TRY(launch_dot(dots + l.aux_off, l.n_aux, P.fmt, P.plane, recs, partials, acc, s));
        S.launches_finalize += 2;
      } else {
        CUDA_TRY(launch_finalize(fins + l.fin_off, l.n_fin, P.fmt, P.plane, recs, acc, s));
        S.launches_finalize++;
      }
    }
  }
  S.launches_total = S.launches_evolve + S.launches_operand + S.launches_contract + S.launches_finalize;
  return PEPS_OK;
}

// After a timed call (its stream synchronised): the event time of every
// contraction launch, summed into S and kept per launch in the context's log.
static int read_launch_times(peps_ctx *c, Plan &P, size_t n_timed, const std::vector<int> &idx,
                             peps_stats &S) {
  c->launch_log.clear();
  for (size_t i = 0; i < n_timed; ++i) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
    const Launch &l = P.launches[idx[i]];
    S.contract_ms += ms;
    if (l.tc) S.contract_tc_ms += ms;
    peps_launch_info li{};
    li.flops = l.flops;
    li.bytes = l.bytes;
    li.ms = ms;
    li.tensor_cores = l.tc ? 1 : 0;
    li.step = l.step;
    c->launch_log.push_back(li);
  }
  return PEPS_OK;
}

static int run_plan(peps_ctx *c, Plan &P, const uint64_t *d_bits_in, cudaStream_t s) {
  const bool timing = (P.opts.flags & PEPS_FLAG_TIMING) != 0;
  const bool graph = (P.opts.flags & PEPS_FLAG_GRAPH) != 0;
  peps_stats S{};
  S.n_steps = P.n_steps;
  S.n_lanes = P.lanes;

  if (c->sm_count == 0) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
  }

  if (graph) {
    // the graph always contains the evolution, so a replay never depends on
    // what an earlier call left in the site tensors.  With TIMING the replay
    // is of a second graph whose capture also recorded the events around
    // every contraction launch (event-record nodes), so that it times its
    // own launches; the plain graph carries no events.
    cudaGraphExec_t &gx = P.graph_exec[timing ? 1 : 0];
    if (!gx) {
      for (auto &l : P.launches)
        if (l.kind == 0 && l.tc) CUDA_TRY(tc_warm(l.tc_handle));
      if (timing) {
        size_t nl = 0;
        for (auto &l : P.launches) nl += l.kind == 0;
        int rc = ensure_events(c, 2 * nl * P.slice_list.size());
        if (rc) return rc;
      }
      if (!c->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      cudaStream_t cs = c->cap_stream;
      CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      peps_stats S2{};
      size_t n_t = 0;
      std::vector<int> t_idx;
      int rc = enqueue_sequence(c, P, d_bits_in, cs, true, timing, S2, &n_t, &t_idx, true);
      if (timing) {
        P.graph_n_timed = n_t;
        P.graph_timed_idx = t_idx;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      CUDA_TRY(e);
      e = cudaGraphInstantiate(&gx, g, 0);
      cudaGraphDestroy(g);
      CUDA_TRY(e);
    }
    CUDA_TRY(cudaGraphLaunch(gx, s));
    int rc = enqueue_sequence_stats_only(P, S);
    if (rc) return rc;
    if (timing) {
      CUDA_TRY(cudaStreamSynchronize(s));
      int rc2 = read_launch_times(c, P, P.graph_n_timed, P.graph_timed_idx, S);
      if (rc2) return rc2;
    }
    c->built_generation = c->generation;
    c->built_ws = P.ws;
    c->stats = S;
    return PEPS_OK;
  }

  const bool rebuild = (P.opts.flags & PEPS_FLAG_REBUILD) || c->built_generation != c->generation ||
                       c->built_ws != P.ws;
  size_t n_timed = 0;
  std::vector<int> timed_idx;
  if (timing) {
    size_t nl = 0;
    for (auto &l : P.launches) nl += l.kind == 0;
    int rc = ensure_events(c, 2 * nl * P.slice_list.size());
    if (rc) return rc;
  }
  int rc = enqueue_sequence(c, P, d_bits_in, s, rebuild, timing, S, &n_timed, &timed_idx);
  if (rc) return rc;
  if (rebuild) {
    c->built_generation = c->generation;
    c->built_ws = P.ws;
  }
  if (timing) {
    CUDA_TRY(cudaStreamSynchronize(s));
    rc = read_launch_times(c, P, n_timed, timed_idx, S);
    if (rc) return rc;
  }
  c->stats = S;
  return PEPS_OK;
}

static int check_status(peps_ctx *c, Plan &P, cudaStream_t s) {
  DeviceStatus h{};
  CUDA_TRY(cudaMemcpyAsync(&h, (char *)P.ws + P.off_status, sizeof h, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h.timeout) {
    c->broken = true;
    return fail(PEPS_ETIMEOUT, "a device wait exceeded the watchdog budget (site step %d)", h.error_info);
  }
  if (h.error)
    return fail(PEPS_EINVAL, "prefix group check failed at bitstring %d: bits of the first %d "
                "columns differ inside a group", h.error_info, P.opts.prefix_cols);
  return PEPS_OK;
}

// Plan the call (or reuse the context's plan) and upload the plan's tables
// into the workspace.  The upload is ordered on the call's stream `s`, after
// whatever the caller enqueued there before (an earlier call's kernels may
// still be reading the tables of the same workspace).
static int prepare(peps_ctx *c, int64_t n, const peps_opts *opts, void *ws, size_t ws_bytes,
                   const uint64_t *bits_dev, bool host_bits, cudaStream_t s) {
  peps_opts o{};
  if (opts) o = *opts;
  Plan *P = c->plan.get();
  bool reuse = P && P->generation == c->generation && P->n == n && opts_equal(P->opts, o) &&
               P->ws == ws && P->ws_bytes == ws_bytes && P->bits == bits_dev &&
               P->host_bits == host_bits;
  if (reuse && o.n_fixed > 0)
    reuse = P->fixed == std::vector<uint32_t>(o.fixed_cz, o.fixed_cz + o.n_fixed) &&
            P->fixed_s == std::vector<uint8_t>(o.fixed_s, o.fixed_s + o.n_fixed);
  if (reuse && o.n_sliced > 0) {
    reuse = P->sliced == std::vector<uint32_t>(o.sliced_cz, o.sliced_cz + o.n_sliced);
    if (reuse && o.slice_ids)
      reuse = P->slice_ids == std::vector<uint64_t>(o.slice_ids, o.slice_ids + o.n_slice_ids);
  }
  if (reuse) {
    P->opts.flags = o.flags;
    P->opts.watchdog_ns = o.watchdog_ns;
    return PEPS_OK;
  }
  auto NP = std::make_unique<Plan>();
  int rc = build_plan(c, n, o, ws, ws_bytes, bits_dev, host_bits, *NP);
  if (rc) return rc;
  {
    const size_t part_a = NP->off_ops_begin - NP->off_site_ptrs;
    // pageable source: the copy is staged before the call returns, so the
    // blob may be replaced by a later plan at any time
    CUDA_TRY(cudaMemcpyAsync((char *)ws + NP->off_site_ptrs, NP->blob.data(), part_a,
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync((char *)ws + NP->off_opdesc, NP->blob.data() + part_a,
                             NP->blob.size() - part_a, cudaMemcpyHostToDevice, s));
  }
  c->plan = std::move(NP);
  c->built_generation = 0;  // site buffers may have moved: re-evolve
  return PEPS_OK;
}

extern "C" int peps_amplitudes_device(peps_ctx *c, const uint64_t *d_bits, int64_t n,
                                      peps_c128 *d_out, const peps_opts *opts, void *ws,
                                      size_t ws_bytes, void *stream) {
  if (!c) return fail(PEPS_EINVAL, "peps_amplitudes_device: NULL context");
  if (c->broken) return fail(PEPS_ESTATE, "context unusable after an earlier device failure");
  if (n < 0 || (n > 0 && (!d_bits || !d_out)) || !ws)
    return fail(PEPS_EINVAL, "peps_amplitudes_device: bad arguments");
  if (n == 0) return PEPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare(c, n, opts, ws, ws_bytes, d_bits, false, s);
  if (rc) return rc;
  Plan &P = *c->plan;
  rc = run_plan(c, P, d_bits, s);
  if (rc) return rc;
  CUDA_TRY(launch_store_out((const double2 *)((char *)ws + P.off_acc), d_out, n, s));
  c->stats.launches_finalize++;
  c->stats.launches_total++;
  const bool needs_check = (P.opts.flags & PEPS_FLAG_TIMING) || P.opts.prefix_cols > 0;
  if (needs_check) return check_status(c, P, s);
  return PEPS_OK;
}

extern "C" int peps_amplitudes(peps_ctx *c, const uint64_t *bits, int64_t n, peps_c128 *out,
                               const peps_opts *opts, void *ws, size_t ws_bytes, void *stream) {
  if (!c) return fail(PEPS_EINVAL, "peps_amplitudes: NULL context");
  if (c->broken) return fail(PEPS_ESTATE, "context unusable after an earlier device failure");
  if (n < 0 || (n > 0 && (!bits || !out)) || !ws)
    return fail(PEPS_EINVAL, "peps_amplitudes: bad arguments");
  if (n == 0) return PEPS_OK;
  for (int64_t i = 0; i < n; ++i)
    if (c->n < 64 && (bits[i] >> c->n) != 0)
      return fail(PEPS_EINVAL, "bitstring %lld has bits beyond qubit %d", (long long)i, c->n - 1);
  cudaStream_t s = (cudaStream_t)stream;
  // The staging area sits at a fixed place in the workspace; the plan's items
  // point there.
  int rc = prepare(c, n, opts, ws, ws_bytes, nullptr, true, s);
  if (rc) return rc;
  Plan &P = *c->plan;
  uint64_t *d_bits = (uint64_t *)((char *)ws + P.off_bits);
  peps_c128 *d_out = (peps_c128 *)((char *)ws + P.off_out);
  CUDA_TRY(cudaMemcpyAsync(d_bits, bits, n * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  rc = run_plan(c, P, d_bits, s);
  if (rc) return rc;
  CUDA_TRY(launch_store_out((const double2 *)((char *)ws + P.off_acc), d_out, n, s));
  c->stats.launches_finalize++;
  c->stats.launches_total++;
  rc = check_status(c, P, s);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(out, d_out, n * sizeof(peps_c128), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return PEPS_OK;
}

// ---------------------------------------------------------------------------
// Helpers for the allocation-free entry point (noalloc.cu)
// ---------------------------------------------------------------------------
int peps::internal_fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void peps::internal_forget_workspace(peps_ctx *c) {
  c->plan.reset();
  c->built_generation = 0;
  c->built_ws = nullptr;
}
