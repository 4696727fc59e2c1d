// Shared definitions of libhfmm: context, device buffers, multi-index helpers,
// packed list entries and the integer cell geometry used by the traversal.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hfmm.h"

namespace hfmm {

constexpr int kDepth = 21;           // finest octree level (2^21 cells per side)
constexpr int kPMax = 8;             // highest supported expansion order
constexpr int kNCMax = 165;          // ncoef(kPMax)
constexpr int kMlpWeights = 5512;    // learned-acceptance network parameters (BF16)
constexpr int64_t kHalfBox = 1ll << 22;  // box side in half units (L / 2^22)

__host__ __device__ constexpr int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Graded multi-index order: k = |n| ascending, nx descending, ny descending.
__host__ __device__ inline int midx(int nx, int ny, int nz) {
  int k = nx + ny + nz, j = k - nx;
  return k * (k + 1) * (k + 2) / 6 + j * (j + 1) / 2 + (j - ny);
}

// Inverse of midx.
__host__ __device__ inline void mdecode(int c, int &nx, int &ny, int &nz) {
  int k = 0;
  while (ncoef(k) <= c) ++k;
  int r = c - (k ? ncoef(k - 1) : 0);
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= r) ++j;
  nx = k - j;
  ny = j - (r - j * (j + 1) / 2);
  nz = k - nx - ny;
}

// ---------------------------------------------------------------- lists
// Packed (sink node, source node, shift, order) entry:
//   bits 61..63  expansion order - 1 of an M2L entry (0 for P2P and frontier entries)
//   bits 34..60  sink node (27 bits)
//   bit  33      M2L entries: 1 = the operator is evaluated per pair, 0 = it is read
//                from the (level, offset) table (sorting on bits 33.. puts a sink's
//                table pairs first)
//   bits  5..32  source node (28 bits)
//   bits  0..4   periodic shift index 0..26
constexpr int kSinkShift = 34;
constexpr int kSinkBits = 27;
constexpr int kOrderShift = 61;
__host__ __device__ inline uint64_t pack_pair(uint32_t sink, uint32_t src, uint32_t s, uint32_t order_m1 = 0) {
  return ((uint64_t)order_m1 << kOrderShift) | ((uint64_t)sink << kSinkShift) | ((uint64_t)src << 5) | (uint64_t)s;
}
__host__ __device__ inline uint32_t pair_sink(uint64_t e) { return (uint32_t)((e >> kSinkShift) & 0x7ffffffull); }
__host__ __device__ inline uint32_t pair_src(uint64_t e) { return (uint32_t)((e >> 5) & 0xfffffffull); }
constexpr int kGenericBit = 33;
__host__ __device__ inline bool pair_generic(uint64_t e) { return (e >> kGenericBit) & 1ull; }
__host__ __device__ inline uint32_t pair_shift(uint64_t e) { return (uint32_t)(e & 31ull); }
__host__ __device__ inline uint32_t pair_order(uint64_t e) { return (uint32_t)(e >> kOrderShift) + 1u; }
__host__ __device__ inline uint64_t with_order(uint64_t e, uint32_t order) {
  return (e & ~(7ull << kOrderShift)) | ((uint64_t)(order - 1u) << kOrderShift);
}

// ---------------------------------------------------------------- cells
// cell = {ix, iy, iz, level}; half-unit centre 2*ix*w + w with w = 2^(21-level).
__host__ __device__ inline int64_t half_width(uint32_t level) { return (int64_t)1 << (kDepth - level); }
__host__ __device__ inline int64_t half_centre(uint32_t i, uint32_t level) {
  int64_t w = half_width(level);
  return 2 * (int64_t)i * w + w;
}
__host__ __device__ inline int shift_component(uint32_t s, int d) {
  return d == 0 ? (int)(s / 9) - 1 : d == 1 ? (int)((s / 3) % 3) - 1 : (int)(s % 3) - 1;
}
// Source centre (displaced by the periodic shift) minus sink centre, half units.
__host__ __device__ inline void half_delta(uint4 sink, uint4 src, uint32_t s, int64_t *dd) {
  dd[0] = half_centre(src.x, src.w) + shift_component(s, 0) * kHalfBox - half_centre(sink.x, sink.w);
  dd[1] = half_centre(src.y, src.w) + shift_component(s, 1) * kHalfBox - half_centre(sink.y, sink.w);
  dd[2] = half_centre(src.z, src.w) + shift_component(s, 2) * kHalfBox - half_centre(sink.z, sink.w);
}

// Source centre (with the periodic shift) minus sink centre in half units; every
// quantity fits 32 bits: centres are below 2^22, the shift is +-2^22.
__host__ __device__ inline void half_delta32(uint4 sink, uint4 src, uint32_t s, int (&dd)[3]) {
  const uint32_t la = kDepth - sink.w, lb = kDepth - src.w;  // log2 of the half widths
  dd[0] = (int)(((2u * src.x + 1u) << lb) - ((2u * sink.x + 1u) << la)) + shift_component(s, 0) * (int)kHalfBox;
  dd[1] = (int)(((2u * src.y + 1u) << lb) - ((2u * sink.y + 1u) << la)) + shift_component(s, 1) * (int)kHalfBox;
  dd[2] = (int)(((2u * src.z + 1u) << lb) - ((2u * sink.z + 1u) << la)) + shift_component(s, 2) * (int)kHalfBox;
}

// ---------------------------------------------------------------- Morton keys
// Periodic wrap and 63-bit Morton key of one position (shared by the octree
// build and the allocation-free sort, so both give the same keys).
// x / L: when L is a power of two, x * (1/L) is the same correctly rounded
// quotient (1/L exact), without an FP64 division.
__device__ __forceinline__ double div_box(double x, double box, double inv_pow2) {
  return inv_pow2 != 0.0 ? __dmul_rn(x, inv_pow2) : __ddiv_rn(x, box);
}

// x - L floor(x / L), each operation rounded separately (no FMA contraction).
__device__ __forceinline__ double wrap_box(double x, double box, double inv_pow2) {
  double q = floor(div_box(x, box, inv_pow2));
  return __dsub_rn(x, __dmul_rn(box, q));
}

// Cell index of a wrapped coordinate on the 2^21 grid per side.
__device__ __forceinline__ uint32_t grid_coord(double w, double box, double inv_pow2) {
  double t = floor(__dmul_rn(div_box(w, box, inv_pow2), 2097152.0));
  t = fmax(0.0, fmin(t, 2097151.0));
  return (uint32_t)t;
}

// Spread the low 21 bits of v to every third bit.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// The cell index grid_coord(wrap_box(x)) for a power-of-two L and x already in
// [0, L), read from the bits of x: x = 1.f 2^(e - 1023), L = 2^(eL - 1023), so
// floor(x 2^21 / L) is the 53-bit significand shifted right by 52 - (e - eL + 21)
// (zero when that is negative) -- the same value with no FP64 arithmetic (this
// GPU's FP64 rate is low).  False, with nothing computed, for x outside [0, L),
// a denormal x, or NaN; the caller then takes the FP64 route.
__device__ __forceinline__ bool grid_coord_bits(double x, double box, uint32_t &k) {
  const long long b = __double_as_longlong(x), lb = __double_as_longlong(box);
  if (b < 0 || b >= lb) return false;  // positive doubles order like their bit patterns
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) {
    if (b != 0) return false;
    k = 0;
    return true;
  }
  const int s = e - (int)((lb >> 52) & 0x7ff) + 21;  // <= 20, since x < L
  if (s < 0) {
    k = 0;
    return true;
  }
  const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | (1ull << 52);
  k = (uint32_t)(m >> (52 - s));
  return true;
}

// wrap_box, with the bits of x checked first: a coordinate already in [0, L)
// of a power-of-two L is its own wrap (no FP64 arithmetic).
__device__ __forceinline__ double wrap_box_fast(double x, double box, double inv_pow2) {
  const long long b = __double_as_longlong(x);
  if (inv_pow2 != 0.0 && b >= 0 && b < __double_as_longlong(box)) return x;
  return wrap_box(x, box, inv_pow2);
}

__device__ __forceinline__ uint32_t cell_coord(double x, double box, double inv_pow2) {
  uint32_t k;
  if (inv_pow2 != 0.0 && grid_coord_bits(x, box, k)) return k;
  return grid_coord(wrap_box(x, box, inv_pow2), box, inv_pow2);
}

// Key of the (unwrapped) position (x, y, z): x bits above y bits above z bits.
__device__ __forceinline__ uint64_t morton_key(double x, double y, double z, double box, double inv_pow2) {
  const uint32_t k0 = cell_coord(x, box, inv_pow2);
  const uint32_t k1 = cell_coord(y, box, inv_pow2);
  const uint32_t k2 = cell_coord(z, box, inv_pow2);
  return (spread3(k0) << 2) | (spread3(k1) << 1) | spread3(k2);
}

// Mutual P2P: which of the mirror pairs (a, b, s) and (b, a, 26 - s) evaluates
// both directions.  The deeper (smaller) leaf owns, so that a large leaf beside
// a dense region does not take all of that region's pairs on one warp; leaves
// of one level alternate by the parity of a + b; a leaf against its own
// periodic images keeps s <= 13 (13 = itself, evaluated one-sided).
__host__ __device__ inline bool p2p_owner(uint32_t a, uint32_t b, uint32_t s, uint32_t lev_a, uint32_t lev_b) {
  if (a == b) return s <= 13u;
  if (lev_a != lev_b) return lev_a > lev_b;
  return ((a ^ b) & 1u) ? a < b : a > b;
}

// ---------------------------------------------------------------- tree sizes on the device
// The octree build's sizes as its cooperative kernel leaves them (node count,
// leaf count, levels, first node of each level, capacity overflow).  In graph
// mode the kernels after the build read their sizes here instead of taking
// them from the host; an overflowed build reads as an empty tree.
struct TreeState {
  unsigned long long total, nleaves;
  int nlevels, overflow;
  unsigned long long level_start[kDepth + 3];
};
__host__ __device__ inline int64_t tree_nodes(const TreeState *t, int64_t host) {
  return t ? (t->overflow ? 0 : (int64_t)t->total) : host;
}
__host__ __device__ inline int64_t tree_leaves(const TreeState *t, int64_t host) {
  return t ? (t->overflow ? 0 : (int64_t)t->nleaves) : host;
}
// nodes [lo, lo + cnt) of level l (cnt = 0 beyond the last level or after an overflow)
__host__ __device__ inline void tree_level(const TreeState *t, int l, int64_t &lo, int64_t &cnt) {
  if (!t) return;
  if (t->overflow || l + 1 >= t->nlevels) {
    lo = 0;
    cnt = 0;
    return;
  }
  lo = (int64_t)t->level_start[l];
  cnt = (int64_t)t->level_start[l + 1] - lo;
}

// ---------------------------------------------------------------- buffers
struct DBuf {
  void *p = nullptr;
  size_t cap = 0;
};

// Grow b to at least `bytes` (contents not kept).  While *g_deferred_free is set
// (a stream capture is in progress) the old allocation is queued there instead of freed.
cudaError_t ensure(DBuf &b, size_t bytes);
extern thread_local std::vector<void *> *g_deferred_free;
// Grow b to at least `bytes`, keeping the first `keep` bytes (stream-ordered copy).
cudaError_t ensure_keep(DBuf &b, size_t bytes, size_t keep, cudaStream_t st);
void release(DBuf &b);

template <class T>
inline T *P(DBuf &b) {
  return static_cast<T *>(b.p);
}

// ---------------------------------------------------------------- scan / sort
// Exclusive prefix sum of n uint32 values; *total (device, uint64) receives the sum.
// `tmp` is scratch grown as needed.
cudaError_t scan_u32(const uint32_t *in, uint32_t *out, uint64_t *total, size_t n, DBuf &tmp, cudaStream_t st);

// Stable LSD radix sort of uint64 keys on bits [bit_lo, bit_hi), optionally
// carrying uint32 values.  Ping-pongs between (keys, vals) and (keys_alt,
// vals_alt); returns in *in_alt whether the result ended in the alt buffers.
cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, size_t n,
                           int bit_lo, int bit_hi, bool *in_alt, DBuf &tmp, cudaStream_t st);

// The same sort with all scratch in a caller-provided region (no allocation);
// radix_sort_scratch_bytes(n) is the size that region needs.
size_t radix_sort_scratch_bytes(size_t n);
cudaError_t radix_sort_u64_into(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, size_t n,
                                int bit_lo, int bit_hi, bool *in_alt, void *scratch, size_t scratch_bytes,
                                cudaStream_t st);

// ---------------------------------------------------------------- pair force
// S(x) = erfc(x/2) + x e^(-x^2/4) / sqrt(pi) = exp2(r^2 kexp) Q(r / R_c),
// Q(t) = sum_j c[j] t^j (degree 9), kexp = -log2(e) / (4 r_s^2).
// 1/L when the box side L is a power of two (then exact), else 0
inline double box_inverse_if_pow2(double box) {
  int e = 0;
  return std::frexp(box, &e) == 0.5 ? 1.0 / box : 0.0;
}

struct PairFit {
  float c[10];  // Q = sum_i c[i] u^i, u = r - rmid
  float rmid, rc2, kexp;
};
// Chebyshev interpolation (10 nodes on [0, R_c]) of e^(x^2/4) erfc(x/2) + x/sqrt(pi),
// x = r / r_s, in FP64, expanded in powers of u = r - R_c / 2 and rounded to FP32.
PairFit fit_pair_factor(double rs, double rc);
struct Ctx;
void mac_integer_thresholds(Ctx &c);

// ---------------------------------------------------------------- context
// ORB / k-d tree of tree = 1 (kdtree.cu): binary nodes numbered breadth first.
struct KdTree {
  DBuf xw;                       // f64 [3][n] wrapped positions, input order
  DBuf ord[3], ord2[3];          // u32 [n] per axis: the particles of each node's range in (coordinate, index) order
  DBuf side;                     // u8 [n] per particle: 1 = in the second child of its node's split
  DBuf flag, scan;               // u32 [3][n]: side flags of the three orders and their scan
  DBuf pnode;                    // u32 [n] node of each position on the level being split (its leaf at the end)
  DBuf nflag, nscan;             // u32 [cap] split flags of a level's nodes and their scan
  DBuf first, count;             // u32 [cap] particle range
  DBuf child, parent, axis;      // i32 [cap] first child (-1 leaf), parent (-1 root), split axis (-1 leaf)
  DBuf box;                      // f64 [6][cap] lo xyz, hi xyz of the particles' bounding box
  DBuf geo;                      // f64 [7][cap] centre xyz, half extents xyz, side (largest extent)
  DBuf geof;                     // f32 [7][cap] the same rounded (the walk's FP32 filter)
  DBuf hs;                       // f32 [cap] expansion scale h: L 2^-j >= side, j <= 21
  DBuf ctr;                      // u64 [16]: the walk's counters, then the build's scan total
  DBuf lv;                       // u64 [2][levels]: each level's node extent [lo, hi) during the build
  std::vector<int64_t> level_start;
  int64_t cap = 0;
  uint64_t caps[3] = {0, 0, 0};  // frontier, M2L and P2P capacities of the last walk
};

struct Ctx {
  hfmm_params prm{};
  double rs = 0, rc = 0;        // split scale and cut-off radius
  double rc2h = 0, theta2 = 0;  // MAC thresholds (half units squared; theta^2)
  // The same tests on integer squared distances (decisions identical to the FP64 ones):
  //   (double)s > rc2h          <=>  s > rc2i = floor(rc2h)
  //   4 w_l^2 <= fl(theta2 * s)  <=>  s >= acc_thr[l]   (w_l = 2^(21-l) half units)
  int64_t rc2i = 0;
  int64_t acc_thr[kDepth + 1] = {};
  PairFit fit{};
  int p = 4, nc = 35;
  int ldm = 36;  // row stride of the expansion arrays: nc rounded up to a multiple of 4 (float4 rows)
  std::string err;

  // particles
  int64_t n = 0;
  bool have_tree = false;
  DBuf key, key_alt, idx, idx_alt;  // u64 keys, u32 input indices
  DBuf xs;                          // f64 [3][n] sorted wrapped positions
  DBuf pm4;                         // float4 [n] (offset from leaf centre, mass)
  DBuf perm;                        // u32 [n] input index per sorted particle (alias of idx result)

  // nodes (breadth-first)
  int64_t nnodes = 0, nleaves = 0;
  int nlevels = 0;
  int64_t level_start[kDepth + 3] = {0};
  DBuf cell;    // uint4 {ix, iy, iz, level}
  DBuf range;   // uint2 {first, count}
  DBuf kids;    // int2 {first child or -1, child count}
  DBuf leaves;  // u32 [nleaves] node index of each leaf
  DBuf bounds, nkids, koff, tstate;  // build scratch
  uint64_t cap_nodes = 0;

  // traversal
  DBuf front, front_next, cls, counts, offs;
  // sink-major walk: segment of each sink cell (per level), segment sinks and totals,
  // segment bases, runs of M2L / P2P entries per (sink, level)
  DBuf fseg, fseg_next, seg_a, seg_b, acc_a, acc_b, segbase, btot2, segpre, ctot;
  DBuf rm_key, rm_beg, rm_cnt, rp_key, rp_beg, rp_cnt;
  // runs per sink (counters during the walk) and each run's rank among its sink's runs
  DBuf rm_rank, rp_rank, rcnt_m, rcnt_p;
  uint64_t cap_seg = 0, cap_run = 0;
  int64_t nrun_m = 0, nrun_p = 0, frontier_items = 0;
  DBuf m2l, m2l_alt, p2p, p2p_alt;  // packed u64 entries
  int64_t nm2l = 0, np2p = 0;
  int traverse_iters = 0;
  int64_t traverse_walks = 0;  // walks of the last traversal (1 + repeats after an overflow)
  uint64_t cap_front = 0, cap_m2l = 0, cap_p2p = 0;  // traversal capacities (entries)
  int cap_levels = 0;  // graph mode: tree levels the level loops cover
  double walk_share = 1.0;  // sink batches: the share of the walk one batch takes (first list guesses)
  int last_batches = 1;     // sink batches of the last short-range call
  bool lists_split = false; // the last short-range call's lists were evaluated in parts (not kept)
  DBuf pacc;                // sink batches: P2P accelerations [3][n], added by L2P
  DBuf lpt_order, lpt_tmp;  // P2P: the sink leaves longest first, and its buckets and counters
  DBuf tf_pairs, tf_segs, tf_sst;  // sink batches: the frontier the top levels leave
  DBuf m2l_beg, m2l_end, p2p_beg, p2p_end;  // u32 [nnodes] CSR bounds by sink
  DBuf m2l_mid;  // u32 [nnodes]: [beg, mid) table pairs, [mid, end) per-pair operator

  // M2L operator table: T[level][ox][oy][oz][c], |o_d| <= tab_k, c < ncoef(p) padded to tab_ld
  DBuf tab;
  int tab_k = 0, tab_ld = 0;
  bool tab_ready = false;

  // expansions (scaled): M~ = M / h^|m|, L~ = L h^(|n|+1)
  DBuf M, L;

  // host-visible scratch
  DBuf tmp, tmp2;
  uint64_t *h_pinned = nullptr;  // small pinned host buffer for counters
  DBuf d_small;                  // small device buffer for counters

  // host-buffer entry point
  DBuf hpos, hmass, hacc;

  // learned acceptance: BF16 weights (5512 values); training-pair collection
  DBuf mlp_w;
  bool have_mlp = false;
  bool collect = false;
  // set for the duration of an interaction-count walk: 1 = hybrid acceptance
  // with geometric decisions, 2 = conventional acceptance (no cut-off rules,
  // primary box only)
  int count_walk = 0;
  DBuf cand;
  uint64_t cand_cap = 0;
  int64_t ncand_last = 0;  // candidates written by the last collection
  uint32_t sample_mod = 1;
  DBuf mlp_scratch;

  // PM long range (cuFFT plans made on first use; -1 = none) and the step
  DBuf pm_q, pm_rho, pm_mk, pm_ak, pm_a;
  // mutual P2P: per entry partial counts and offsets, sort keys and entry indices
  // (ping-pong), per leaf bounds of its entries as a source, partial sums [3][slots]
  DBuf mut_cnt, mut_poff, mut_key, mut_key_alt, mut_val, mut_val_alt, mut_bounds, mut_small, mut_part;
  DBuf mut_lkey, mut_lval;            // sink leaves sorted by descending work (keys, leaf ids; ping-pong)
  const uint32_t *mut_order = nullptr;  // the sorted leaf ids (inside mut_lval)
  // (level, offset) tensor-core M2L: node flags and ranks, tile meta, tile sinks,
  // tile pair counts and offsets, grouped pairs
  DBuf lo_flag, lo_rank, lo_meta, lo_sink, lo_tcnt, lo_toff, lo_scr;
  KdTree kd;  // tree = 1
  DBuf pm_gtab;          // polynomial split: long-range Green function per integer |k|^2
  size_t pm_gtab_n = 0;  // its length (0: not built)
  int pm_plan_r2c = -1, pm_plan_c2r = -1;
  const float *mass_ref = nullptr;  // the mass array of the last build_tree

  // graph mode: the post-traversal sequence captured on gstream, replayed on the caller's stream
  cudaStream_t gstream = nullptr;
  cudaEvent_t gready = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_updates = 0, graph_instantiations = 0;
  bool last_graph = false;  // the last short_range_forces ran as one graph
  bool graph_walk = false;  // while capturing: list sizes live on the device (capacities on the host)
  bool graph_tree = false;  // while capturing a step: tree sizes live on the device (c.tstate)
  cudaGraphExec_t gexec_step = nullptr;  // the KDK step as one graph (use_graph)
  std::vector<uint64_t> step_sig;         // the state the step graph's capture left
  long long step_kernels = 0;             // kernels in the step graph
  int64_t step_graphs = 0;                // steps launched as one graph
  bool last_step_graph = false;           // the last call was a step launched as one graph

  // stats
  int64_t p2p_particle_pairs = -1, p2p_useful_pairs = -1, nm2l_table = -1;
  cudaEvent_t ev[16] = {};
  bool ev_ready = false;
  float t_keys_sort = -1, t_tree = -1, t_upward = -1, t_traverse = -1, t_lists = -1, t_m2l = -1, t_l2l = -1,
        t_p2p = -1;
};

// Phase implementations (each returns a CUDA error; the ABI maps it).
cudaError_t build_tree(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st);
cudaError_t traverse(Ctx &c, cudaStream_t st);
cudaError_t sort_lists(Ctx &c, cudaStream_t st);
// particle pairs on the current P2P list (sum over entries of n_sink n_source); synchronises st
cudaError_t p2p_list_particle_pairs(Ctx &c, cudaStream_t st, int64_t *out);
cudaError_t upward(Ctx &c, cudaStream_t st);
// M2L of the list entries of order q (the CSR bounds m2l_beg/m2l_end cover
// exactly those entries); adds into L.
cudaError_t m2l_pass(Ctx &c, int q, cudaStream_t st);
// All M2L entries: one pass per order present in the list.
cudaError_t m2l_all(Ctx &c, cudaStream_t st);
// Table half-extent K for opening angle theta (0: no table).
int m2l_table_extent(const hfmm_params &p);
// Build the (level, offset) operator table once per context (FP64, rounded to FP32).
cudaError_t m2l_table_build(Ctx &c, cudaStream_t st);
// M2L of the table pairs [beg, mid) of order q; adds into L.
cudaError_t m2l_pass_table(Ctx &c, int q, cudaStream_t st);
// Split-precision (3xTF32) M2L on tcgen05 tensor cores; orders 1..6.  The
// kernel's status word (d_small[6]) is 1 after a timed-out wait.
bool m2l_tc_supported(int p);
cudaError_t m2l_pass_tc(Ctx &c, int q, cudaStream_t st);
// L2L top-down, then L2P writing the far-field accelerations in input order
// (plus add[3][n], input order, when given).
cudaError_t downward(Ctx &c, float *acc, cudaStream_t st, const float *add = nullptr);
// The short-range call in sink batches (upward pass done by the caller; L must
// be zero): the walk over the top levels, then per batch of sinks the rest of
// the walk, list grouping, M2L and P2P (into c.pacc), then L2L and L2P + P2P.
cudaError_t short_range_batched(Ctx &c, float *acc, int nbatch, cudaStream_t st);
// The batches the next short-range call takes (sink_batches, or the automatic count).
int sink_batches_for(const Ctx &c);
// Long-range PM accelerations added to acc (input order); mesh buffers and
// FFT plans are kept in the context (pm_release frees them).
cudaError_t pm_long_range(Ctx &c, float *acc, cudaStream_t st);
// Graph mode: the mesh buffers, FFT plans and Green-function table, made
// outside a capture (pm_long_range calls it too).
cudaError_t pm_prepare(Ctx &c);
void pm_release(Ctx &c);
// A step captured as one graph: the second kick runs only when the tree and the
// walk fitted their capacities (device flags; null pointers: always).
struct StepGuard {
  const int *tree_overflow = nullptr, *walk_overflow = nullptr;
  const unsigned long long *walk_left = nullptr;
};
StepGuard step_guard(Ctx &c);
cudaError_t kick_guarded(float *vel, const float *acc, int64_t n, double h, StepGuard g, cudaStream_t st);
// vel += h acc and pos += dt vel (wrapped), [3][n] arrays.
cudaError_t kick(float *vel, const float *acc, int64_t n, double h, cudaStream_t st);
cudaError_t drift(double *pos, const float *vel, int64_t n, double dt, double box, cudaStream_t st);
// Cut-off P2P, added to the accelerations written by downward().
cudaError_t p2p_pass(Ctx &c, float *acc, cudaStream_t st);
// Graph mode: the walk without its host read-back (sizes every buffer first; the
// read-back after the graph reports whether the lists fit), and the device
// address of the walk's run counts (0 M2L, 1 P2P).
cudaError_t traverse_graph_prepare(Ctx &c);
cudaError_t traverse_graph_launch(Ctx &c, cudaStream_t st);
cudaError_t traverse_graph_finish(Ctx &c, cudaStream_t st, bool *ok);
const unsigned long long *walk_run_counts(Ctx &c, int which);
cudaError_t sort_lists_prepare(Ctx &c);
// Graph mode for the step: the octree build without its read-back.
cudaError_t build_tree_prepare(Ctx &c, int64_t n);
cudaError_t build_tree_launch(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st);
bool build_tree_finish(Ctx &c, const TreeState &hs);
// M2L of order q with m2l_precision 3 / 4: table pairs as (level, offset) tensor-core contractions
// with the accumulators in tensor memory, the other pairs on the FP32 per-pair kernel.
bool m2l_lo_supported(int p);
cudaError_t m2l_pass_lo(Ctx &c, int q, cudaStream_t st);
// Mutual P2P (p2p_mutual = 1): one evaluation per particle pair, reactions through per-entry partials.
cudaError_t p2p_pass_mutual(Ctx &c, float *acc, cudaStream_t st);
// ORB / k-d tree (tree = 1): the build (fills xs, pm4, idx like the octree
// build, so the PM half and the step work unchanged), and the short-range call
// on it: upward pass, walk, lists grouped by sink, M2L, downward pass, P2P.
cudaError_t kd_build_tree(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st);
cudaError_t kd_short_range(Ctx &c, float *acc, cudaStream_t st);
// The walk alone (hybrid or conventional acceptance) and its counts: M2L pairs, P2P
// leaf pairs, particle pairs on the P2P list, pairs classified (Sec. 3).
cudaError_t kd_interaction_counts(Ctx &c, bool conventional, int64_t *out, cudaStream_t st);
cudaError_t kd_upward(Ctx &c, cudaStream_t st);                // expansions.cu
cudaError_t kd_downward(Ctx &c, float *acc, cudaStream_t st);  // expansions.cu: L2L, then L2P writing acc
cudaError_t kd_m2l(Ctx &c, cudaStream_t st);                   // m2l.cu

// Training pairs for the learned acceptance: features [n][12] and M2L errors
// at orders 2..8 [n][7] (device buffers of the caller); *count receives n.
cudaError_t collect_pairs(Ctx &c, int64_t max_pairs, uint32_t sample_mod, float *feat, float *err, int64_t *count,
                          cudaStream_t st);
// Network kernels (mlp.cu).
cudaError_t mlp_infer(const void *w_bf16, const float *x, int64_t n, float *logits, int *cls, cudaStream_t st);
size_t mlp_train_scratch_bytes();
cudaError_t mlp_grad(const float *wm, const float *x, const int *labels, const float *cw, int64_t n, float *grad,
                     float *loss, void *scratch, cudaStream_t st);
cudaError_t mlp_adam(float *wm, float *m1, float *m2, const float *grad, float lr, int step, void *w_bf16,
                     cudaStream_t st);

inline unsigned blocks_for(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

// Process-wide count of kernels launched by this library (reported in stats).
extern std::atomic<long long> g_launches;
inline void note_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace hfmm

struct hfmm_ctx {
  hfmm::Ctx c;
};
