// ORB / k-d tree variant of the short-range FMM (tree = 1): the tree of Sec. 2.1
// (Fig. 1), an ORB tree with a leaf limiter whose cells hand their particles to
// two children of almost equal count, which Sec. 4 keeps as a k-d tree inside
// every domain.
//
// Build, level by level on the device:
//   - positions wrapped (x - L floor(x / L), as for the octree); for each axis d
//     the particle indices sorted once by (coordinate d, input index) with the
//     stable radix sort of order-preserving 64-bit keys;
//   - a level's node reads its particles' bounding box from the first and last
//     entries of its range in the three orders; above leaf_max it splits on the
//     axis of largest extent (the lowest on a tie): the first floor(n / 2)
//     particles of that axis' order form the first child.  The other orders are
//     partitioned stably by the particles' side: an exclusive scan of the side
//     flags over all positions, less its value at the node's first position,
//     ranks a particle among the second child's particles.  So every order stays
//     sorted inside every node, and inside a leaf the x order is the particle
//     order (that of (x, input index)); the three orders are flagged, scanned
//     (one scan over the concatenated flags) and scattered together;
//   - the counts of a level differ by at most one, so the depth follows from N
//     and leaf_max on the host; each level's extent stays on the device (the
//     kernels read it) and is read back once, after the last level.
// Node geometry: the box centre c, half extents e, side (largest extent) in FP64,
// and the expansion scale h = L 2^-j >= side (j <= 21, the octree's deepest
// cell side): P2M offsets over h stay within [-1/2, 1/2] and the scale ratios of
// the translations are powers of two.
// Walk: one cooperative launch, level synchronous over the frontier of (sink,
// source, shift) pairs with grid-wide barriers between the levels, one thread per
// pair, the three rules of Sec. 2.3 on the boxes in FP64 with every operation
// rounded on its own (no contraction, so the decisions are those of any IEEE FP64
// evaluation in the same order), taken in FP32 wherever an error bound shows the
// FP32 comparison cannot differ; M2L and P2P entries and the next frontier are
// appended with warp-aggregated atomics, and when a list or the frontier outgrows
// its buffer the buffers are grown and the walk repeated.  The lists are then
// sorted by (sink, source, shift), so every sum after them runs in a fixed order.
// The same walk with the opening-angle test alone, from the root against itself,
// is the conventional FMM's of the interaction counts (Sec. 3).
// P2P: one warp per sink leaf, the leaves taken heaviest first from a counter,
// its sinks in lanes (a second sink per lane above 32); the list read in windows
// of 32 entries, each lane forming its entry's source-box offset from the sink
// box centre in FP64; each entry's sources loaded one entry ahead, kept only
// within R_c of the sink box, staged in shared memory and evaluated two at a
// time in packed FP32x2, with the Gaussian (Sec. 2.2) or polynomial (Sec. 5)
// pair force.
#include <algorithm>

#include <cooperative_groups.h>

#include "p2p_common.cuh"

namespace cg = cooperative_groups;

namespace hfmm {
namespace {

constexpr int kT = 256;
constexpr int kKdMaxLevels = 64;

__global__ void k_kd_wrap(const double *__restrict__ pos, int64_t n, double box, double inv_pow2,
                          double *__restrict__ xw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  xw[i] = wrap_box_fast(pos[i], box, inv_pow2);
}

// Order-preserving key of a double (negative values reversed below the positive ones).
__global__ void k_kd_keys(const double *__restrict__ x, int64_t n, uint64_t *__restrict__ key,
                          uint32_t *__restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t u = (uint64_t)__double_as_longlong(x[i]);
  key[i] = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  val[i] = (uint32_t)i;
}

__global__ void k_kd_root(int64_t n, uint32_t *first, uint32_t *count, int *parent, unsigned long long *lv) {
  first[0] = 0;
  count[0] = (uint32_t)n;
  parent[0] = -1;
  lv[0] = 0;
  lv[1] = 1;
}

// The extent [lo, hi) of tree level l on the device: lv[2 l], lv[2 l + 1].
__device__ __forceinline__ void level_extent(const unsigned long long *lv, int l, int64_t &lo, int64_t &hi) {
  lo = (int64_t)lv[2 * l];
  hi = (int64_t)lv[2 * l + 1];
}

// One level's nodes: bounding box and split decision (split flags zero up to `bound`
// nodes, the grid's size, so the scan of a level of unknown size on the host works).
__global__ void k_kd_level(const unsigned long long *__restrict__ lv, int level, int64_t bound, int leaf_max,
                           const double *__restrict__ xw, int64_t n,
                           const uint32_t *__restrict__ o0, const uint32_t *__restrict__ o1,
                           const uint32_t *__restrict__ o2, const uint32_t *__restrict__ first,
                           const uint32_t *__restrict__ count, double *__restrict__ box, int64_t cap,
                           int *__restrict__ axis, uint32_t *__restrict__ nflag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= bound) return;
  int64_t lo, hi;
  level_extent(lv, level, lo, hi);
  if (t >= hi - lo) {
    nflag[t] = 0u;
    return;
  }
  const int64_t k = lo + t;
  const uint32_t f = first[k], m = count[k];
  const uint32_t *ord[3] = {o0, o1, o2};
  double best = 0.0;
  int ax = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double a = xw[d * n + ord[d][f]], b = xw[d * n + ord[d][f + m - 1]];
    box[d * cap + k] = a;
    box[(3 + d) * cap + k] = b;
    const double ext = __dsub_rn(b, a);
    if (d == 0 || ext > best) {  // the lowest axis of the largest extent
      best = ext;
      ax = d;
    }
  }
  const bool split = (int64_t)m > leaf_max;
  axis[k] = split ? ax : -1;
  nflag[t] = split ? 1u : 0u;
}

__global__ void k_kd_children(const unsigned long long *__restrict__ lv, int level, const int *__restrict__ axis,
                              const uint32_t *__restrict__ nscan, uint32_t *__restrict__ first,
                              uint32_t *__restrict__ count, int *__restrict__ child, int *__restrict__ parent) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t lo, hi;
  level_extent(lv, level, lo, hi);
  if (t >= hi - lo) return;
  const int64_t k = lo + t;
  if (axis[k] < 0) {
    child[k] = -1;
    return;
  }
  const int64_t ch = hi + 2 * (int64_t)nscan[t];
  const uint32_t f = first[k], m = count[k];
  child[k] = (int)ch;
  first[ch] = f;
  count[ch] = m / 2;
  first[ch + 1] = f + m / 2;
  count[ch + 1] = m - m / 2;
  parent[ch] = parent[ch + 1] = (int)k;
}

// The next level's extent: [hi, hi + 2 splits).
__global__ void k_kd_next(unsigned long long *__restrict__ lv, int level, const uint64_t *__restrict__ nsplit) {
  lv[2 * level + 2] = lv[2 * level + 1];
  lv[2 * level + 3] = lv[2 * level + 1] + 2ull * nsplit[0];
}

// The side of every particle of a node split on this level (positions of earlier leaves: node < lo).
__global__ void k_kd_side(int64_t n, const unsigned long long *__restrict__ lv, int level,
                          const uint32_t *__restrict__ pnode, const uint32_t *__restrict__ first,
                          const uint32_t *__restrict__ count, const int *__restrict__ axis,
                          const uint32_t *__restrict__ o0, const uint32_t *__restrict__ o1,
                          const uint32_t *__restrict__ o2, uint8_t *__restrict__ side) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = (int64_t)lv[2 * level];
  const uint32_t k = pnode[i];
  if ((int64_t)k < lo) return;
  const int a = axis[k];
  if (a < 0) return;
  const uint32_t p = a == 0 ? o0[i] : a == 1 ? o1[i] : o2[i];
  side[p] = (uint32_t)i - first[k] >= count[k] / 2 ? 1 : 0;
}

// The side flags of the three orders, concatenated ([3][n]; zero outside the nodes
// split on this level), for one scan over all of them.
__global__ void k_kd_flag(int64_t n, const unsigned long long *__restrict__ lv, int level,
                          const uint32_t *__restrict__ pnode, const int *__restrict__ axis,
                          const uint32_t *__restrict__ o0, const uint32_t *__restrict__ o1,
                          const uint32_t *__restrict__ o2, const uint8_t *__restrict__ side,
                          uint32_t *__restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = (int64_t)lv[2 * level];
  const uint32_t k = pnode[i];
  const bool split = (int64_t)k >= lo && axis[k] >= 0;
  flag[i] = split ? side[o0[i]] : 0u;
  flag[n + i] = split ? side[o1[i]] : 0u;
  flag[2 * n + i] = split ? side[o2[i]] : 0u;
}

// Stable partition of the three orders inside every node split on this level:
// in order d a particle of the second child is preceded in it by scan[d n + i] -
// scan[d n + first] such particles (the scan runs over the concatenated flags).
__global__ void k_kd_scatter(int64_t n, const unsigned long long *__restrict__ lv, int level,
                             const uint32_t *__restrict__ pnode, const uint32_t *__restrict__ first,
                             const uint32_t *__restrict__ count, const int *__restrict__ axis,
                             const uint32_t *__restrict__ o0, const uint32_t *__restrict__ o1,
                             const uint32_t *__restrict__ o2, const uint8_t *__restrict__ side,
                             const uint32_t *__restrict__ scan, uint32_t *__restrict__ r0,
                             uint32_t *__restrict__ r1, uint32_t *__restrict__ r2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = (int64_t)lv[2 * level];
  const uint32_t k = pnode[i];
  const uint32_t *ord[3] = {o0, o1, o2};
  uint32_t *out[3] = {r0, r1, r2};
  if ((int64_t)k < lo || axis[k] < 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d][i] = ord[d][i];
    return;
  }
  const uint32_t f = first[k], nl = count[k] / 2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const uint32_t v = ord[d][i];
    const uint32_t r = scan[d * n + i] - scan[d * n + f];  // particles of the second child before position i
    out[d][side[v] ? f + nl + r : (uint32_t)i - r] = v;
  }
}

__global__ void k_kd_pnode(int64_t n, const unsigned long long *__restrict__ lv, int level,
                           uint32_t *__restrict__ pnode, const uint32_t *__restrict__ first,
                           const uint32_t *__restrict__ count, const int *__restrict__ child) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = (int64_t)lv[2 * level];
  const uint32_t k = pnode[i];
  if ((int64_t)k < lo || child[k] < 0) return;
  pnode[i] = (uint32_t)child[k] + ((uint32_t)i - first[k] >= count[k] / 2 ? 1u : 0u);
}

// Centre, half extents, side and expansion scale of every node.
__global__ void k_kd_geo(int64_t nn, int64_t cap, const double *__restrict__ box, double L, double *__restrict__ geo,
                         float *__restrict__ geof, float *__restrict__ hs, const int *__restrict__ child,
                         uint32_t *__restrict__ lflag) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  double side = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double a = box[d * cap + k], b = box[(3 + d) * cap + k];
    geo[d * cap + k] = __dmul_rn(0.5, __dadd_rn(a, b));
    geo[(3 + d) * cap + k] = __dmul_rn(0.5, __dsub_rn(b, a));
    const double e = __dsub_rn(b, a);
    side = d == 0 ? e : (e > side ? e : side);
  }
  geo[6 * cap + k] = side;
  // the walk's FP32 record of the node: (centre xyz, side), (half extents xyz, first child)
  reinterpret_cast<float4 *>(geof)[2 * k] = make_float4((float)geo[k], (float)geo[cap + k], (float)geo[2 * cap + k],
                                                         (float)side);
  reinterpret_cast<float4 *>(geof)[2 * k + 1] = make_float4((float)geo[3 * cap + k], (float)geo[4 * cap + k],
                                                             (float)geo[5 * cap + k], __int_as_float(child[k]));
  double h = L;
  for (int j = 0; j < kDepth && side <= 0.5 * h; ++j) h *= 0.5;
  hs[k] = (float)h;
  lflag[k] = child[k] < 0 ? 1u : 0u;
}

__global__ void k_kd_leaves(int64_t nn, const uint32_t *__restrict__ lflag, const uint32_t *__restrict__ lscan,
                            uint32_t *__restrict__ leaves) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn || !lflag[k]) return;
  leaves[lscan[k]] = (uint32_t)k;
}

// Particles in tree order: positions, input index, offset from the leaf's box centre and mass.
__global__ void k_kd_particles(int64_t n, const uint32_t *__restrict__ o0, const double *__restrict__ xw,
                               const float *__restrict__ mass, const uint32_t *__restrict__ pnode,
                               const double *__restrict__ geo, int64_t cap, double *__restrict__ xs,
                               uint32_t *__restrict__ perm, float4 *__restrict__ pm4) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t p = o0[i], k = pnode[i];
  float off[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double x = xw[d * n + p];
    xs[d * n + i] = x;
    off[d] = (float)__dsub_rn(x, geo[d * cap + k]);
  }
  perm[i] = p;
  pm4[i] = make_float4(off[0], off[1], off[2], mass[p]);
}

// ------------------------------------------------------------------ walk
struct KdGeo {
  const double *g;  // [7][cap]: centre xyz, half extents xyz, side
  const float *gf;  // [cap][8]: (centre xyz, side), (half extents xyz, first child) rounded to FP32
  int64_t cap;
  __device__ double c(int d, uint32_t k) const { return g[d * cap + k]; }
  __device__ double e(int d, uint32_t k) const { return g[(3 + d) * cap + k]; }
  __device__ double side(uint32_t k) const { return g[6 * cap + k]; }
  __device__ void rec(uint32_t k, float4 &p, float4 &q) const {
    const float4 *r = reinterpret_cast<const float4 *>(gf) + 2 * (size_t)k;
    p = __ldg(r);
    q = __ldg(r + 1);
  }
};

__device__ __forceinline__ float comp(const float4 &v, int d) { return d == 0 ? v.x : d == 1 ? v.y : v.z; }

struct WalkRule {
  double L, rc2, theta2;
  float Lf, rc2f, theta2f, dl;  // dl: 16 2^-24 L, the FP32 error bound of a shifted difference
  int rule, size_rule;
  int conventional;  // 1: the opening-angle test alone (a conventional FMM, Sec. 3), primary box
};

// 0 skip, 1 M2L, 2 open: the rules of Sec. 2.3 on the boxes (sink a, source b shifted by s L),
// in FP64 with every operation rounded on its own.
__device__ __forceinline__ int kd_classify64(const KdGeo &G, uint32_t a, uint32_t b, uint32_t s, const WalkRule &R) {
  double sc2 = 0.0, sm2 = 0.0, sx2 = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double dc = __dsub_rn(__dadd_rn(G.c(d, b), (double)shift_component(s, d) * R.L), G.c(d, a));
    const double ad = fabs(dc);
    const double w = __dadd_rn(G.e(d, a), G.e(d, b));
    double gap = __dsub_rn(ad, w);
    if (gap < 0.0) gap = 0.0;
    const double far = __dadd_rn(ad, w);
    sc2 = __dadd_rn(sc2, __dmul_rn(dc, dc));
    sm2 = __dadd_rn(sm2, __dmul_rn(gap, gap));
    sx2 = __dadd_rn(sx2, __dmul_rn(far, far));
  }
  if (!R.conventional && sm2 > R.rc2) return 0;
  const bool trans = R.conventional ? false : R.rule == 0 ? sc2 > R.rc2 : sx2 > R.rc2;
  const double sa = G.side(a), sb = G.side(b);
  const double wl = R.size_rule == 0 ? sb : (sa > sb ? sa : sb);
  const double lim = __dmul_rn(R.theta2, sc2);  // a pair with theta S_c = 0 is never accepted
  if (!trans && lim > 0.0 && __dmul_rn(wl, wl) <= lim) return 1;
  return 2;
}

// The same decisions, taken in FP32 where they are certain.  In FP32 the node
// geometry is off by at most 2^-24 L (centres) and 2^-25 L (half extents), so each
// shifted per-axis difference dc, gap and span (coordinates in [-L, 2L]) is within
// delta = 16 2^-24 L of its FP64 value, and a sum q of three squares x^2 within
//   E(q) = 2 (2 delta sum |x| + 3 delta^2 + 8 2^-24 q)
// (the factor 2 a margin above the rounding analysis); theta^2 S_c^2 within
// 2 (theta^2 E(S_c^2) + 3 2^-24 theta^2 S_c^2), the squared side within 6 2^-24 of
// itself, R_c^2 within 2^-23 of itself.  A comparison whose two sides' intervals
// overlap is taken again in FP64 (this GPU's FP64 rate is low), so the result is
// always the FP64 one.
__device__ __noinline__ int kd_classify64_call(const KdGeo &G, uint32_t a, uint32_t b, uint32_t s,
                                               const WalkRule &R) {
  return kd_classify64(G, a, b, s, R);
}

__device__ __forceinline__ int kd_classify(const KdGeo &G, uint32_t a, uint32_t b, uint32_t s, const WalkRule &R,
                                           const float4 &A0, const float4 &A1, const float4 &B0, const float4 &B1) {
  constexpr float u = 5.9604645e-8f;  // 2^-24
  float sc2 = 0.f, sm2 = 0.f, sx2 = 0.f, Sc = 0.f, Sm = 0.f, Sx = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float dc = __fsub_rn(__fadd_rn(comp(B0, d), (float)shift_component(s, d) * R.Lf), comp(A0, d));
    const float ad = fabsf(dc);
    const float w = __fadd_rn(comp(A1, d), comp(B1, d));
    const float gap = fmaxf(__fsub_rn(ad, w), 0.f);
    const float far = __fadd_rn(ad, w);
    sc2 = __fadd_rn(sc2, __fmul_rn(dc, dc));
    sm2 = __fadd_rn(sm2, __fmul_rn(gap, gap));
    sx2 = __fadd_rn(sx2, __fmul_rn(far, far));
    Sc += ad;
    Sm += gap;
    Sx += far;
  }
  const float dl = R.dl, d2 = 3.f * dl * dl;
  const float erc = 2.f * u * R.rc2f;
  const float ec = 2.f * (2.f * dl * Sc + d2 + 8.f * u * sc2);
  if (!R.conventional) {
    const float em = 2.f * (2.f * dl * Sm + d2 + 8.f * u * sm2);
    if (sm2 - em > R.rc2f + erc) return 0;
    if (sm2 + em >= R.rc2f - erc) return kd_classify64_call(G, a, b, s, R);
    const float tq = R.rule == 0 ? sc2 : sx2;
    const float et = R.rule == 0 ? ec : 2.f * (2.f * dl * Sx + d2 + 8.f * u * sx2);
    if (tq - et > R.rc2f + erc) return 2;
    if (tq + et >= R.rc2f - erc) return kd_classify64_call(G, a, b, s, R);
  }
  if (R.theta2 == 0.0) return 2;
  const float sa = A0.w, sb = B0.w;
  const float wl = R.size_rule == 0 ? sb : fmaxf(sa, sb);
  const float lim = __fmul_rn(R.theta2f, sc2), w2 = __fmul_rn(wl, wl);
  const float el = 2.f * (R.theta2f * ec + 3.f * u * lim), ew = 6.f * u * w2;
  if (lim - el > 0.f && w2 + ew < lim - el) return 1;
  if (w2 - ew > lim + el) return 2;
  return kd_classify64_call(G, a, b, s, R);
}

// Append the entries of the lanes with `take` at consecutive slots of a list
// (one atomic per warp); slots at or above cap are counted, not written.
__device__ __forceinline__ void warp_append(bool take, uint64_t e, unsigned long long *ctr, uint64_t *out,
                                            unsigned long long cap) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
  if (take && slot < cap) out[slot] = e;
}

// Walk counters (u64): [0] M2L entries, [1] P2P entries, [2] status (1: the frontier
// buffer outgrown), [3] levels walked, [4] pairs classified, [5..7] next-frontier counts
// of three consecutive levels (level l appends to [5 + l % 3]; the one of level
// l + 1 is cleared during level l, after every block has read it at level l - 2).
constexpr int kWalkCtr = 8;

// The whole walk in one cooperative launch: the 27 root pairs (root, root, s) as
// the first frontier (the conventional walk: the root against itself alone),
// then level after level with grid-wide barriers between
// them, until the frontier is empty or outgrows its buffer (the caller grows the
// buffers that were outgrown, the frontier's or a list's, and walks again).
__global__ void __launch_bounds__(kT, 4) k_kd_walk(uint64_t *__restrict__ fa, uint64_t *__restrict__ fb,
                                                unsigned long long cap_f, uint64_t *__restrict__ m2l,
                                                unsigned long long cap_m, uint64_t *__restrict__ p2p,
                                                unsigned long long cap_p, unsigned long long *__restrict__ ctr,
                                                KdGeo G, WalkRule R) {
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  // the root against its 27 nearest images (a conventional walk: against itself only)
  if (R.conventional ? gt == 0 : gt < 27) fa[gt] = pack_pair(0u, 0u, R.conventional ? 13u : (uint32_t)gt);
  unsigned long long nf = R.conventional ? 1 : 27, pairs = 0;
  grid.sync();
  for (int level = 0;; ++level) {
    uint64_t *cur = (level & 1) ? fb : fa, *next = (level & 1) ? fa : fb;
    unsigned long long *ncount = ctr + 5 + level % 3;
    if (gt == 0) ctr[5 + (level + 1) % 3] = 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < nf; base += stride) {
      const unsigned long long t = base + threadIdx.x;
      uint32_t a = 0, b = 0, s = 0;
      int cls = 0;
      uint64_t e = 0;
      float4 A0, A1, B0, B1;
      if (t < nf) {
        e = cur[t];
        a = pair_sink(e);
        b = pair_src(e);
        s = pair_shift(e);
        G.rec(a, A0, A1);
        G.rec(b, B0, B1);
        cls = kd_classify(G, a, b, s, R, A0, A1, B0, B1);
      }
      int ca = -1, cb = -1;
      bool opena = false, openb = false;
      if (cls == 2) {
        ca = __float_as_int(A1.w);
        cb = __float_as_int(B1.w);
        if (ca < 0 && cb < 0) {
          cls = 3;  // two leaves: P2P
        } else if (ca < 0) {
          openb = true;
        } else if (cb < 0) {
          opena = true;
        } else if (A0.w != B0.w) {  // rounding to FP32 keeps the order of unequal sides
          opena = A0.w > B0.w;
          openb = !opena;
        } else {
          const double sa = G.side(a), sb = G.side(b);
          opena = sa >= sb;
          openb = sb >= sa;
        }
      }
      warp_append(cls == 1, e, ctr + 0, m2l, cap_m);
      warp_append(cls == 3, e, ctr + 1, p2p, cap_p);
      // the children pairs: (opena ? 2 : 1) x (openb ? 2 : 1) of them
      const uint32_t nkid = cls == 2 ? (opena ? 2u : 1u) * (openb ? 2u : 1u) : 0u;
      uint32_t incl = nkid;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (tot == 0) continue;
      unsigned long long wb = 0;
      if (lane == 31) wb = atomicAdd(ncount, (unsigned long long)tot);
      wb = __shfl_sync(0xffffffffu, wb, 31);
      unsigned long long slot = wb + incl - nkid;
      if (nkid) {
        const uint32_t a0 = opena ? (uint32_t)ca : a, a1 = opena ? a0 + 2 : a + 1;
        const uint32_t b0 = openb ? (uint32_t)cb : b, b1 = openb ? b0 + 2 : b + 1;
        for (uint32_t x = a0; x < a1; ++x)
          for (uint32_t y = b0; y < b1; ++y, ++slot)
            if (slot < cap_f) next[slot] = pack_pair(x, y, s);
      }
    }
    pairs += nf;
    grid.sync();
    // Every block reads the same count (this level's counter takes no appends until
    // it is cleared two levels on), so every block takes the same decision.  The
    // M2L and P2P counters are not read here: blocks already in the next level
    // append to them.  An outgrown list only stops being written (the counts go on);
    // the caller compares the final counts with the capacities.
    const unsigned long long nn = *(volatile unsigned long long *)ncount;
    const bool over = nn > cap_f;
    if (over || nn == 0) {
      if (gt == 0) {
        ctr[2] = over ? 1ull : 0ull;
        ctr[3] = (unsigned long long)level + 1;
        ctr[4] = pairs;
      }
      return;
    }
    nf = nn;
  }
}

// CSR bounds of a list sorted by sink.
__global__ void k_kd_csr(const uint64_t *__restrict__ lst, int64_t n, uint32_t *__restrict__ beg,
                         uint32_t *__restrict__ end) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t k = pair_sink(lst[t]);
  if (t == 0 || pair_sink(lst[t - 1]) != k) beg[k] = (uint32_t)t;
  if (t == n - 1 || pair_sink(lst[t + 1]) != k) end[k] = (uint32_t)(t + 1);
}

// ------------------------------------------------------------------ P2P
// One warp per sink leaf (the leaves heaviest first, taken from a counter):
// sinks i = first + lane and first + lane + 32.  The list entries come in windows of 32, one per lane, each
// lane forming its entry's source-box offset from the sink box centre in FP64
// (once per entry: this GPU's FP64 rate is low); each entry's sources are held in
// registers one entry ahead; the sources within R_c of the sink box are staged in
// shared memory (SoA, padded to an even count with a far, massless source) and
// each lane evaluates two sources at a time with packed FP32x2 operations: the
// pair force of Sec. 2.2 (or of Sec. 5) with the hard cut-off, added to acc in
// input order.
constexpr int kKdStage = 64;

// kCount (statistics runs): also count the pairs inside (0, R_c) into *useful.
// kSplit: 0 the Gaussian pair force of Sec. 2.2, 1 the polynomial one of Sec. 5.
template <bool kCount, int kSplit>
__global__ void __launch_bounds__(kT) k_kd_p2p(const uint32_t *__restrict__ leaves, int64_t nl,
                                               const uint32_t *__restrict__ first, const uint32_t *__restrict__ count,
                                               KdGeo Gm, const uint32_t *__restrict__ beg,
                                               const uint32_t *__restrict__ end, const uint64_t *__restrict__ lst,
                                               const float4 *__restrict__ pm4, const uint32_t *__restrict__ perm,
                                               int64_t n, double L, PairFit2 fit, float G, float *__restrict__ acc,
                                               unsigned long long *__restrict__ useful,
                                               unsigned long long *__restrict__ next) {
  __shared__ __align__(16) float sx[kT / 32][kKdStage + 2], sy[kT / 32][kKdStage + 2], sz[kT / 32][kKdStage + 2],
      sw[kT / 32][kKdStage + 2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float *X = sx[wid], *Y = sy[wid], *Z = sz[wid], *Wm = sw[wid];
  const float rc2_cull = fit.rc2 * (1.f + 1.f / 4096.f);  // far above the FP32 rounding of either distance
  uint32_t n_in = 0;
  for (;;) {
    // the next leaf of the heaviest-first order (each leaf's sums stay its own warp's)
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(next, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= nl) break;
    const uint32_t k = leaves[t];
    const uint32_t f = first[k], m = count[k];
    const uint32_t tb = beg[k], te = end[k];
    const bool has0 = (uint32_t)lane < m, has1 = (uint32_t)lane + 32u < m;
    const bool two = m > 32;  // warp-uniform
    const float4 q0 = has0 ? pm4[f + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 q1 = has1 ? pm4[f + lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
    // the sink offsets, negated, as (x, x) pairs
    const float2 n0x = f2(-q0.x), n0y = f2(-q0.y), n0z = f2(-q0.z);
    const float2 n1x = f2(-q1.x), n1y = f2(-q1.y), n1z = f2(-q1.z);
    // the sink box's half extents (its particles' offsets lie within them, up to FP32 rounding)
    const float ex = (float)Gm.e(0, k), ey = (float)Gm.e(1, k), ez = (float)Gm.e(2, k);
    float2 a0x = f2(0.f), a0y = f2(0.f), a0z = f2(0.f), a1x = f2(0.f), a1y = f2(0.f), a1z = f2(0.f);
    // a window of 32 list entries, one per lane: source range and the source box's
    // offset from the sink box centre (FP64, then FP32)
    uint32_t wfb = 0, wmb = 0;
    float wox = 0.f, woy = 0.f, woz = 0.f;
    auto load_window = [&](uint32_t base) {
      wmb = 0;
      if (base + lane < te) {
        const uint64_t e = lst[base + lane];
        const uint32_t b = pair_src(e), s = pair_shift(e);
        wfb = first[b];
        wmb = count[b];
        wox = (float)__dsub_rn(__dadd_rn(Gm.c(0, b), (double)shift_component(s, 0) * L), Gm.c(0, k));
        woy = (float)__dsub_rn(__dadd_rn(Gm.c(1, b), (double)shift_component(s, 1) * L), Gm.c(1, k));
        woz = (float)__dsub_rn(__dadd_rn(Gm.c(2, b), (double)shift_component(s, 2) * L), Gm.c(2, k));
      }
    };
    // the sources of one entry in registers: lane j holds sources j and j + 32
    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
    uint32_t cmb = 0;
    float cox = 0.f, coy = 0.f, coz = 0.f;
    auto fetch = [&](uint32_t slot) {
      const uint32_t fb = __shfl_sync(0xffffffffu, wfb, slot);
      cmb = __shfl_sync(0xffffffffu, wmb, slot);
      cox = __shfl_sync(0xffffffffu, wox, slot);
      coy = __shfl_sync(0xffffffffu, woy, slot);
      coz = __shfl_sync(0xffffffffu, woz, slot);
      if ((uint32_t)lane < cmb) pa = pm4[fb + lane];
      if ((uint32_t)lane + 32u < cmb) pb = pm4[fb + lane + 32];
    };
    uint32_t wbase = tb;
    if (tb < te) {
      load_window(tb);
      fetch(0);
    }
    for (uint32_t q = tb; q < te; ++q) {
      // stage the sources of entry q within R_c of the sink box (R_c^2 (1 + 2^-12): far
      // above the FP32 rounding of either distance), compacted in their order
      const uint32_t mb = cmb;
      const float ox = cox, oy = coy, oz = coz;
      const float4 p0 = pa, p1 = pb;
      __syncwarp();
      uint32_t kept = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t j = (uint32_t)(32 * h + lane);
        float4 p = h ? p1 : p0;
        bool keep = false;
        if (j < mb) {
          p.x += ox;
          p.y += oy;
          p.z += oz;
          const float gx = fmaxf(fabsf(p.x) - ex, 0.f), gy = fmaxf(fabsf(p.y) - ey, 0.f),
                      gz = fmaxf(fabsf(p.z) - ez, 0.f);
          keep = gx * gx + gy * gy + gz * gz < rc2_cull;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const uint32_t w = kept + __popc(mask & ((1u << lane) - 1u));
          X[w] = p.x;
          Y[w] = p.y;
          Z[w] = p.z;
          Wm[w] = p.w;
        }
        kept += __popc(mask);
      }
      if (kept & 1u) {
        if (lane == 0) {  // a far, massless partner for the last source
          X[kept] = 1e18f;
          Y[kept] = 0.f;
          Z[kept] = 0.f;
          Wm[kept] = 0.f;
        }
        ++kept;
      }
      // the next entry's sources are loaded while this entry's pairs are evaluated
      if (q + 1 < te) {
        if (q + 1 - wbase == 32) {
          wbase = q + 1;
          load_window(wbase);
        }
        fetch(q + 1 - wbase);
      }
      __syncwarp();
      // (real: the lane holds this sink; the others evaluate a phantom sink whose result is dropped)
      auto pair2 = [&](float2 px, float2 py, float2 pz, float2 w, float2 nx, float2 ny, float2 nz, float2 &ax,
                       float2 &ay, float2 &az, bool real) {
        const float2 dx = __fadd2_rn(px, nx), dy = __fadd2_rn(py, ny), dz = __fadd2_rn(pz, nz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const bool in0 = r2.x < fit.rc2 && r2.x > 0.f, in1 = r2.y < fit.rc2 && r2.y > 0.f;
        if (kCount && real) n_in += (uint32_t)in0 + (uint32_t)in1;
        // outside (0, R_c) the values below may be inf / NaN; the selects discard them
        const float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        const float2 r3 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
        float2 fs;
        if constexpr (kSplit == 1) {
          // m (1/r^3 - 5 / (2 R_c^3) + 3 r^2 / (2 R_c^5))
          fs = __fmul2_rn(__fadd2_rn(r3, __ffma2_rn(r2, fit.pc1, fit.pc0)), w);
        } else {
          const float2 u = __ffma2_rn(r2, ri, fit.nrmid);  // r - R_c / 2
          float2 qv = fit.c[9];
#pragma unroll
          for (int i = 8; i >= 0; --i) qv = __ffma2_rn(qv, u, fit.c[i]);
          const float2 ea = __fmul2_rn(r2, fit.kexp);
          fs = __fmul2_rn(__fmul2_rn(__fmul2_rn(make_float2(exp2_mufu(ea.x), exp2_mufu(ea.y)), qv), r3), w);
        }
        fs.x = in0 ? fs.x : 0.f;
        fs.y = in1 ? fs.y : 0.f;
        ax = __ffma2_rn(fs, dx, ax);
        ay = __ffma2_rn(fs, dy, ay);
        az = __ffma2_rn(fs, dz, az);
      };
      if (two) {
#pragma unroll 2
        for (uint32_t j = 0; j < kept; j += 2) {
          const float2 px = *reinterpret_cast<const float2 *>(X + j), py = *reinterpret_cast<const float2 *>(Y + j);
          const float2 pz = *reinterpret_cast<const float2 *>(Z + j), w = *reinterpret_cast<const float2 *>(Wm + j);
          pair2(px, py, pz, w, n0x, n0y, n0z, a0x, a0y, a0z, has0);
          pair2(px, py, pz, w, n1x, n1y, n1z, a1x, a1y, a1z, has1);
        }
      } else {
#pragma unroll 4
        for (uint32_t j = 0; j < kept; j += 2) {
          const float2 px = *reinterpret_cast<const float2 *>(X + j), py = *reinterpret_cast<const float2 *>(Y + j);
          const float2 pz = *reinterpret_cast<const float2 *>(Z + j), w = *reinterpret_cast<const float2 *>(Wm + j);
          pair2(px, py, pz, w, n0x, n0y, n0z, a0x, a0y, a0z, has0);
        }
      }
    }
    if (has0) {
      const uint32_t o = perm[f + lane];
      acc[o] += G * (a0x.x + a0x.y);
      acc[n + o] += G * (a0y.x + a0y.y);
      acc[2 * n + o] += G * (a0z.x + a0z.y);
    }
    if (has1) {
      const uint32_t o = perm[f + lane + 32];
      acc[o] += G * (a1x.x + a1x.y);
      acc[n + o] += G * (a1y.x + a1y.y);
      acc[2 * n + o] += G * (a1z.x + a1z.y);
    }
  }
  if (kCount) {
    unsigned long long v = n_in;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(useful, v);
  }
}

// Sort keys of the sink leaves, heaviest first: the complement of entries x sinks (40 bits).
__global__ void k_kd_work(const uint32_t *__restrict__ leaves, int64_t nl, const uint32_t *__restrict__ count,
                          const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                          uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const uint32_t k = leaves[t];
  const uint64_t w = (uint64_t)(end[k] - beg[k]) * count[k];
  key[t] = (~w) & ((1ull << 40) - 1ull);
  val[t] = k;
}

// Particle pairs on the P2P list: sum over entries of n_sink n_source.
__global__ void k_kd_list_pairs(const uint64_t *__restrict__ lst, int64_t n, const uint32_t *__restrict__ count,
                                unsigned long long *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (t < n) v = (unsigned long long)count[pair_sink(lst[t])] * count[pair_src(lst[t])];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

#define TRY(x)                      \
  do {                              \
    cudaError_t e_ = (x);           \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// Read `count` device uint64 values into out (synchronises st).
cudaError_t read_u64(Ctx &c, const void *src, uint64_t *out, int count, cudaStream_t st) {
  TRY(cudaMemcpyAsync(c.h_pinned, src, 8 * (size_t)count, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  for (int q = 0; q < count; ++q) out[q] = c.h_pinned[q];
  return cudaSuccess;
}

KdGeo kd_geo(Ctx &c) { return KdGeo{P<double>(c.kd.geo), P<float>(c.kd.geof), c.kd.cap}; }

// The walk (one cooperative launch, repeated with grown buffers while one is outgrown).
cudaError_t kd_walk(Ctx &c, cudaStream_t st, bool conventional = false) {
  KdTree &kd = c.kd;
  const uint64_t nl = (uint64_t)std::max<int64_t>(c.nleaves, 1);
  uint64_t cap_f = std::max<uint64_t>(kd.caps[0], std::max<uint64_t>(1u << 16, 256 * nl));
  uint64_t cap_m = std::max<uint64_t>(kd.caps[1], std::max<uint64_t>(1u << 16, 32 * nl));
  uint64_t cap_p = std::max<uint64_t>(kd.caps[2], std::max<uint64_t>(1u << 16, 256 * nl));
  if (c.prm.list_init > 0 && kd.caps[0] == 0) cap_f = cap_m = cap_p = (uint64_t)c.prm.list_init;
  cap_f = std::max<uint64_t>(cap_f, 32);  // the 27 root pairs
  TRY(ensure(kd.ctr, 128));
  unsigned long long *ctr = P<unsigned long long>(kd.ctr);
  int dev = 0, nsm = 0, per_sm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kd_walk, kT, 0));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned nb = (unsigned)(nsm * std::min(per_sm, 4));
  WalkRule R;
  R.L = c.prm.box;
  R.rc2 = c.rc * c.rc;
  R.theta2 = c.prm.theta * c.prm.theta;
  R.Lf = (float)R.L;
  R.rc2f = (float)R.rc2;
  R.theta2f = (float)R.theta2;
  R.dl = (float)std::ldexp(16.0 * R.L, -24);
  R.rule = c.prm.transition_rule;
  R.size_rule = c.prm.size_rule;
  R.conventional = conventional ? 1 : 0;
  KdGeo G = kd_geo(c);
  int64_t walks = 0;
  uint64_t h[kWalkCtr];
  for (;;) {
    if (++walks > 16) return cudaErrorInvalidValue;
    TRY(ensure(c.front, cap_f * 8));
    TRY(ensure(c.front_next, cap_f * 8));
    TRY(ensure(c.m2l, cap_m * 8));
    TRY(ensure(c.p2p, cap_p * 8));
    TRY(cudaMemsetAsync(ctr, 0, kWalkCtr * 8, st));
    uint64_t *fa = P<uint64_t>(c.front), *fb = P<uint64_t>(c.front_next), *m2l = P<uint64_t>(c.m2l),
             *p2p = P<uint64_t>(c.p2p);
    unsigned long long cf = cap_f, cm = cap_m, cp = cap_p;
    void *args[] = {(void *)&fa, (void *)&fb, (void *)&cf, (void *)&m2l, (void *)&cm, (void *)&p2p, (void *)&cp,
                    (void *)&ctr, (void *)&G, (void *)&R};
    TRY(cudaLaunchCooperativeKernel((const void *)k_kd_walk, dim3(nb), dim3(kT), args, 0, st));
    note_launch();
    TRY(read_u64(c, ctr, h, kWalkCtr, st));
    if (!h[2] && h[0] <= cap_m && h[1] <= cap_p) break;
    // an outgrown buffer: grow what the counts ask for (the counts went on past the capacities)
    const uint64_t nn = std::max(std::max(h[5], h[6]), h[7]);
    if (nn > cap_f) cap_f = nn + nn / 2 + 4096;
    if (h[0] > cap_m) cap_m = h[0] + h[0] / 2 + 4096;
    if (h[1] > cap_p) cap_p = h[1] + h[1] / 2 + 4096;
  }
  kd.caps[0] = cap_f;
  kd.caps[1] = cap_m;
  kd.caps[2] = cap_p;
  c.nm2l = (int64_t)h[0];
  c.np2p = (int64_t)h[1];
  c.traverse_iters = (int)h[3];
  c.frontier_items = (int64_t)h[4];
  c.traverse_walks = walks;
  return cudaSuccess;
}

cudaError_t kd_group(Ctx &c, cudaStream_t st) {
  const size_t nn = (size_t)c.nnodes;
  TRY(ensure(c.m2l_beg, nn * 4));
  TRY(ensure(c.m2l_end, nn * 4));
  TRY(ensure(c.p2p_beg, nn * 4));
  TRY(ensure(c.p2p_end, nn * 4));
  // the sorts' scratch: the walk's frontier buffers, free once the walk is done, when
  // they are large enough (at 134M particles they hold tens of GB), else a buffer of its own
  DBuf *lst[2] = {&c.m2l, &c.p2p}, *alt[2] = {&c.front_next, &c.front};
  if (c.front_next.cap < (size_t)c.nm2l * 8) alt[0] = &c.m2l_alt;
  if (c.front.cap < (size_t)c.np2p * 8) alt[1] = &c.p2p_alt;
  DBuf *beg[2] = {&c.m2l_beg, &c.p2p_beg}, *end[2] = {&c.m2l_end, &c.p2p_end};
  const int64_t len[2] = {c.nm2l, c.np2p};
  for (int w = 0; w < 2; ++w) {
    TRY(cudaMemsetAsync(beg[w]->p, 0, nn * 4, st));
    TRY(cudaMemsetAsync(end[w]->p, 0, nn * 4, st));
    if (len[w] == 0) continue;
    TRY(ensure(*alt[w], (size_t)len[w] * 8));
    bool in_alt = false;
    TRY(radix_sort_u64(P<uint64_t>(*lst[w]), nullptr, P<uint64_t>(*alt[w]), nullptr, (size_t)len[w], 0,
                       kSinkShift + kSinkBits, &in_alt, c.tmp, st));
    if (in_alt) std::swap(*lst[w], *alt[w]);
    k_kd_csr<<<blocks_for((size_t)len[w], kT), kT, 0, st>>>(P<uint64_t>(*lst[w]), len[w], P<uint32_t>(*beg[w]),
                                                             P<uint32_t>(*end[w]));
    note_launch();
  }
  // statistics runs: the particle pairs on the P2P list
  c.p2p_particle_pairs = -1;
  if (c.prm.profile & 2) {
    unsigned long long *cnt = P<unsigned long long>(c.kd.ctr) + kWalkCtr + 1;
    TRY(cudaMemsetAsync(cnt, 0, 8, st));
    if (c.np2p > 0) {
      k_kd_list_pairs<<<blocks_for((size_t)c.np2p, kT), kT, 0, st>>>(P<uint64_t>(c.p2p), c.np2p,
                                                                      P<uint32_t>(c.kd.count), cnt);
      note_launch();
    }
    uint64_t pp = 0;
    TRY(read_u64(c, cnt, &pp, 1, st));
    c.p2p_particle_pairs = (int64_t)pp;
  }
  return cudaGetLastError();
}

cudaError_t kd_p2p(Ctx &c, float *acc, cudaStream_t st) {
  if (c.np2p == 0 || c.nleaves == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned g = (unsigned)std::min<int64_t>((c.nleaves + 7) / 8, (int64_t)nsm * 8);
  // the sink leaves heaviest first (stable: equal work keeps the leaf order), taken from a counter
  const size_t nl = (size_t)c.nleaves;
  TRY(ensure(c.lpt_tmp, nl * 24 + 64));
  uint64_t *key = P<uint64_t>(c.lpt_tmp), *key2 = key + nl;
  uint32_t *val = reinterpret_cast<uint32_t *>(key2 + nl), *val2 = val + nl;
  k_kd_work<<<blocks_for(nl, kT), kT, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint32_t>(c.kd.count),
                                               P<uint32_t>(c.p2p_beg), P<uint32_t>(c.p2p_end), key, val);
  note_launch();
  bool alt = false;
  TRY(radix_sort_u64(key, val, key2, val2, nl, 0, 40, &alt, c.tmp, st));
  const uint32_t *order = alt ? val2 : val;
  unsigned long long *next = P<unsigned long long>(c.kd.ctr) + kWalkCtr + 2;
  TRY(cudaMemsetAsync(next, 0, 8, st));
  unsigned long long *useful = P<unsigned long long>(c.d_small) + 4;  // the statistics counter of stats
  auto run = [&](auto kernel) {
    kernel<<<g, kT, 0, st>>>(order, c.nleaves, P<uint32_t>(c.kd.first), P<uint32_t>(c.kd.count), kd_geo(c),
                             P<uint32_t>(c.p2p_beg), P<uint32_t>(c.p2p_end), P<uint64_t>(c.p2p), P<float4>(c.pm4),
                             P<uint32_t>(c.idx), c.n, c.prm.box, pair_fit2(c), (float)c.prm.G, acc, useful, next);
  };
  const bool count_pairs = (c.prm.profile & 2) != 0, poly = c.prm.split == 1;
  if (count_pairs)
    poly ? run(k_kd_p2p<true, 1>) : run(k_kd_p2p<true, 0>);
  else
    poly ? run(k_kd_p2p<false, 1>) : run(k_kd_p2p<false, 0>);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t kd_build_tree(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st) {
  KdTree &kd = c.kd;
  c.n = n;
  c.nnodes = c.nleaves = 0;
  c.nlevels = 0;
  c.have_tree = false;
  kd.level_start.assign(1, 0);
  if (n == 0) {
    c.have_tree = true;
    return cudaSuccess;
  }
  // a leaf of a split node holds at least floor((leaf_max + 1) / 2) particles
  const int64_t lmin = std::max(1, (c.prm.leaf_max + 1) / 2);
  const int64_t cap = 2 * ((n + lmin - 1) / lmin) + 2;
  if (cap > ((int64_t)1 << kSinkBits)) return cudaErrorInvalidValue;  // mapped to HFMM_ERR_CAPACITY
  kd.cap = cap;
  if (c.prm.profile & 1) cudaEventRecord(c.ev[0], st);
  TRY(ensure(kd.xw, (size_t)n * 24));
  for (int d = 0; d < 3; ++d) {
    TRY(ensure(kd.ord[d], (size_t)n * 4));
    TRY(ensure(kd.ord2[d], (size_t)n * 4));
  }
  TRY(ensure(kd.side, (size_t)n));
  TRY(ensure(kd.flag, (size_t)n * 12));
  TRY(ensure(kd.scan, (size_t)n * 12));
  TRY(ensure(kd.pnode, (size_t)n * 4));
  TRY(ensure(kd.nflag, (size_t)cap * 4));
  TRY(ensure(kd.nscan, (size_t)cap * 4));
  TRY(ensure(kd.first, (size_t)cap * 4));
  TRY(ensure(kd.count, (size_t)cap * 4));
  TRY(ensure(kd.child, (size_t)cap * 4));
  TRY(ensure(kd.parent, (size_t)cap * 4));
  TRY(ensure(kd.axis, (size_t)cap * 4));
  TRY(ensure(kd.box, (size_t)cap * 48));
  TRY(ensure(kd.geo, (size_t)cap * 56));
  TRY(ensure(kd.geof, (size_t)cap * 32));
  TRY(ensure(kd.hs, (size_t)cap * 4));
  TRY(ensure(c.key, (size_t)n * 8));
  TRY(ensure(c.key_alt, (size_t)n * 8));
  TRY(ensure(c.idx, (size_t)n * 4));
  TRY(ensure(c.xs, (size_t)n * 24));
  TRY(ensure(c.pm4, (size_t)n * 16));
  TRY(ensure(c.leaves, (size_t)cap * 4));
  const double inv_pow2 = box_inverse_if_pow2(c.prm.box);
  double *xw = P<double>(kd.xw);
  k_kd_wrap<<<blocks_for((size_t)(3 * n), kT), kT, 0, st>>>(pos, n, c.prm.box, inv_pow2, xw);
  note_launch();
  for (int d = 0; d < 3; ++d) {
    k_kd_keys<<<blocks_for((size_t)n, kT), kT, 0, st>>>(xw + d * n, n, P<uint64_t>(c.key), P<uint32_t>(kd.ord[d]));
    note_launch();
    bool alt = false;
    TRY(radix_sort_u64(P<uint64_t>(c.key), P<uint32_t>(kd.ord[d]), P<uint64_t>(c.key_alt), P<uint32_t>(kd.ord2[d]),
                       (size_t)n, 0, 64, &alt, c.tmp, st));
    if (alt) std::swap(kd.ord[d], kd.ord2[d]);
  }
  if (c.prm.profile & 1) cudaEventRecord(c.ev[1], st);
  uint32_t *first = P<uint32_t>(kd.first), *count = P<uint32_t>(kd.count);
  int *child = P<int>(kd.child), *parent = P<int>(kd.parent), *axis = P<int>(kd.axis);
  TRY(ensure(kd.ctr, 128));
  uint64_t *total = P<uint64_t>(kd.ctr) + kWalkCtr;  // after the walk's counters
  // The depth from the counts alone: the counts of a level differ by at most one (a
  // split gives floor and ceil halves), so [qmin, qmax] bounds them level by level.
  int levels = 1;
  for (int64_t qmin = n, qmax = n; qmax > c.prm.leaf_max; ++levels) {
    qmin = std::max<int64_t>(qmin, c.prm.leaf_max + 1) / 2;
    qmax = (qmax + 1) / 2;
  }
  if (levels > kKdMaxLevels) return cudaErrorInvalidValue;
  TRY(ensure(kd.lv, sizeof(unsigned long long) * 2 * (kKdMaxLevels + 1)));
  unsigned long long *lv = P<unsigned long long>(kd.lv);
  k_kd_root<<<1, 1, 0, st>>>(n, first, count, parent, lv);
  note_launch();
  TRY(cudaMemsetAsync(kd.pnode.p, 0, (size_t)n * 4, st));
  const unsigned gn = blocks_for((size_t)n, kT);
  // every level on the device, its extent read by the kernels (no read-back per level)
  for (int level = 0; level < levels; ++level) {
    const int64_t bound = std::min<int64_t>(level < 62 ? (int64_t)1 << level : cap, cap);
    const unsigned gl = blocks_for((size_t)bound, kT);
    k_kd_level<<<gl, kT, 0, st>>>(lv, level, bound, c.prm.leaf_max, xw, n, P<uint32_t>(kd.ord[0]),
                                  P<uint32_t>(kd.ord[1]), P<uint32_t>(kd.ord[2]), first, count, P<double>(kd.box),
                                  cap, axis, P<uint32_t>(kd.nflag));
    note_launch();
    const bool last = level + 1 == levels;  // no node of the last level splits
    if (!last) TRY(scan_u32(P<uint32_t>(kd.nflag), P<uint32_t>(kd.nscan), total, (size_t)bound, c.tmp2, st));
    k_kd_children<<<gl, kT, 0, st>>>(lv, level, axis, P<uint32_t>(kd.nscan), first, count, child, parent);
    note_launch();
    if (last) break;
    k_kd_next<<<1, 1, 0, st>>>(lv, level, total);
    note_launch();
    k_kd_side<<<gn, kT, 0, st>>>(n, lv, level, P<uint32_t>(kd.pnode), first, count, axis, P<uint32_t>(kd.ord[0]),
                                 P<uint32_t>(kd.ord[1]), P<uint32_t>(kd.ord[2]), P<uint8_t>(kd.side));
    note_launch();
    k_kd_flag<<<gn, kT, 0, st>>>(n, lv, level, P<uint32_t>(kd.pnode), axis, P<uint32_t>(kd.ord[0]),
                                 P<uint32_t>(kd.ord[1]), P<uint32_t>(kd.ord[2]), P<uint8_t>(kd.side),
                                 P<uint32_t>(kd.flag));
    note_launch();
    TRY(scan_u32(P<uint32_t>(kd.flag), P<uint32_t>(kd.scan), total, (size_t)(3 * n), c.tmp2, st));
    k_kd_scatter<<<gn, kT, 0, st>>>(n, lv, level, P<uint32_t>(kd.pnode), first, count, axis, P<uint32_t>(kd.ord[0]),
                                    P<uint32_t>(kd.ord[1]), P<uint32_t>(kd.ord[2]), P<uint8_t>(kd.side),
                                    P<uint32_t>(kd.scan), P<uint32_t>(kd.ord2[0]), P<uint32_t>(kd.ord2[1]),
                                    P<uint32_t>(kd.ord2[2]));
    note_launch();
    for (int d = 0; d < 3; ++d) std::swap(kd.ord[d], kd.ord2[d]);
    k_kd_pnode<<<gn, kT, 0, st>>>(n, lv, level, P<uint32_t>(kd.pnode), first, count, child);
    note_launch();
  }
  // the level extents back (one read-back): nodes, levels, and a full binary tree's leaves
  uint64_t ext[2 * (kKdMaxLevels + 1)];
  TRY(read_u64(c, lv, ext, 2 * levels, st));
  int64_t hi = 0;
  for (int level = 0; level < levels; ++level) {
    if (ext[2 * level + 1] == ext[2 * level]) break;  // an empty level: the tree ended above
    kd.level_start.push_back((int64_t)ext[2 * level + 1]);
    hi = (int64_t)ext[2 * level + 1];
    c.nlevels = level + 1;
  }
  if (hi > cap) return cudaErrorInvalidValue;
  c.nnodes = hi;
  const unsigned gk = blocks_for((size_t)hi, kT);
  k_kd_geo<<<gk, kT, 0, st>>>(hi, cap, P<double>(kd.box), c.prm.box, P<double>(kd.geo), P<float>(kd.geof),
                              P<float>(kd.hs), child, P<uint32_t>(kd.nflag));
  note_launch();
  TRY(scan_u32(P<uint32_t>(kd.nflag), P<uint32_t>(kd.nscan), total, (size_t)hi, c.tmp2, st));
  k_kd_leaves<<<gk, kT, 0, st>>>(hi, P<uint32_t>(kd.nflag), P<uint32_t>(kd.nscan), P<uint32_t>(c.leaves));
  note_launch();
  k_kd_particles<<<gn, kT, 0, st>>>(n, P<uint32_t>(kd.ord[0]), xw, mass, P<uint32_t>(kd.pnode), P<double>(kd.geo),
                                    cap, P<double>(c.xs), P<uint32_t>(c.idx), P<float4>(c.pm4));
  note_launch();
  c.nleaves = (hi + 1) / 2;  // every split node has two children
  if (c.prm.profile & 1) cudaEventRecord(c.ev[2], st);
  c.have_tree = true;
  return cudaGetLastError();
}

cudaError_t kd_interaction_counts(Ctx &c, bool conventional, int64_t *out, cudaStream_t st) {
  TRY(kd_walk(c, st, conventional));
  out[0] = c.nm2l;
  out[1] = c.np2p;
  out[2] = 0;
  out[3] = c.frontier_items;
  if (c.np2p > 0) {
    unsigned long long *cnt = P<unsigned long long>(c.kd.ctr) + kWalkCtr + 1;
    TRY(cudaMemsetAsync(cnt, 0, 8, st));
    k_kd_list_pairs<<<blocks_for((size_t)c.np2p, kT), kT, 0, st>>>(P<uint64_t>(c.p2p), c.np2p,
                                                                    P<uint32_t>(c.kd.count), cnt);
    note_launch();
    uint64_t pp = 0;
    TRY(read_u64(c, cnt, &pp, 1, st));
    out[2] = (int64_t)pp;
  }
  return cudaSuccess;
}

cudaError_t kd_short_range(Ctx &c, float *acc, cudaStream_t st) {
  const bool prof = (c.prm.profile & 1) != 0;
  if (prof) cudaEventRecord(c.ev[3], st);
  TRY(kd_upward(c, st));
  if (prof) cudaEventRecord(c.ev[4], st);
  TRY(kd_walk(c, st));
  if (c.nm2l > (int64_t)UINT32_MAX || c.np2p > (int64_t)UINT32_MAX) return cudaErrorInvalidValue;
  if (prof) cudaEventRecord(c.ev[5], st);
  TRY(kd_group(c, st));
  if (prof) cudaEventRecord(c.ev[6], st);
  TRY(kd_m2l(c, st));
  if (prof) cudaEventRecord(c.ev[7], st);
  TRY(kd_downward(c, acc, st));
  if (prof) cudaEventRecord(c.ev[8], st);
  TRY(kd_p2p(c, acc, st));
  if (prof) cudaEventRecord(c.ev[9], st);
  return cudaSuccess;
}

#undef TRY

}  // namespace hfmm
