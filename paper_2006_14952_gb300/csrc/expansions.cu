// Upward and downward translation passes in scaled Cartesian form (Sec. 2.1,
// Eqs. p2m, m2m, l2l):
//   M~_m = M_m / h^|m|,   L~_n = L_n h^(|n|+1),   h = side of the cell.
// With this scaling the M2M and L2L operators are the same on every level.
// (M2L is in m2l.cu.)
#include "common.cuh"
#include "gen_bodies.cuh"

namespace hfmm {
namespace {

// Row of NC floats at a 16-byte aligned address (rows are padded to a multiple of 4).
template <int NC>
__device__ __forceinline__ void load_row(const float *__restrict__ src, float (&r)[NC]) {
  const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
  for (int q = 0; q < (NC + 3) / 4; ++q) {
    const float4 v = __ldg(s4 + q);
    if (4 * q + 0 < NC) r[4 * q + 0] = v.x;
    if (4 * q + 1 < NC) r[4 * q + 1] = v.y;
    if (4 * q + 2 < NC) r[4 * q + 2] = v.z;
    if (4 * q + 3 < NC) r[4 * q + 3] = v.w;
  }
}

template <int NC>
__device__ __forceinline__ void store_row(float *__restrict__ dst, const float (&r)[NC]) {
  float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
  for (int q = 0; q < NC / 4; ++q) d4[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
#pragma unroll
  for (int c = NC / 4 * 4; c < NC; ++c) dst[c] = r[c];
}

// P2M, one thread per leaf: M~_m = sum_a mu_a (-1)^|m| / m! (u_a)^m, u = (x - z) / h.
// tz (a step captured as one graph): the leaf count from the device tree state.
template <int P>
__global__ void k_p2m(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
                      const uint2 *__restrict__ range, const float4 *__restrict__ pm4, float box, int ldm,
                      float *__restrict__ M, const TreeState *tz) {
  constexpr int NC = ncoef(P);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tree_leaves(tz, nl)) return;
  const uint32_t k = leaves[t];
  const uint2 r = range[k];
  const float inv_h = (float)(1u << cell[k].w) / box;
  float acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.f;
  for (uint32_t i = r.x; i < r.x + r.y; ++i) {
    const float4 q = pm4[i];
    P2MBody<P>::run(q.x * inv_h, q.y * inv_h, q.z * inv_h, q.w, acc);
  }
  P2MBody<P>::finish(acc);
  store_row<NC>(M + (size_t)k * ldm, acc);
}

// M2M, one thread per (cell of one level, child slot): each thread translates
// one child's multipoles to the parent centre; the eight sibling threads are
// adjacent lanes and add their results with a fixed xor-shuffle tree (the same
// order on every run), and slot 0 stores the parent's row.  The loop is
// block-uniform (whole warps take each trip: the shuffles see all lanes); with
// tz (graph mode) the level's extent comes from the device tree state.
template <int P>
__global__ void k_m2m(int64_t lo, int64_t cnt, const uint4 *__restrict__ cell, const int2 *__restrict__ kids, int ldm,
                      float *__restrict__ M, const TreeState *tz, int level) {
  constexpr int NC = ncoef(P);
  tree_level(tz, level, lo, cnt);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < 8 * cnt; b += stride) {
    const int64_t t = b + threadIdx.x;
    const bool in_level = t < 8 * cnt;  // whole groups of 8: cnt * 8 threads, blocks of a multiple of 8
    const int64_t k = lo + t / 8;
    const int slot = (int)(t % 8);
    const int2 kd = in_level ? kids[k] : make_int2(0, 0);
    float o[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) o[c] = 0.f;
    if (slot < kd.y) {
      const int ch = kd.x + slot;
      const uint4 cc = cell[ch];
      // (z_P - z_C) / H = +1/4 for the lower half of an axis, -1/4 for the upper
      float ci[NC];
      load_row<NC>(M + (size_t)ch * ldm, ci);
      M2MBody<P>::run((cc.x & 1u) ? -1.f : 1.f, (cc.y & 1u) ? -1.f : 1.f, (cc.z & 1u) ? -1.f : 1.f, ci, o);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      o[c] += __shfl_xor_sync(0xffffffffu, o[c], 4);
      o[c] += __shfl_xor_sync(0xffffffffu, o[c], 2);
      o[c] += __shfl_xor_sync(0xffffffffu, o[c], 1);
    }
    if (in_level && slot == 0 && kd.y > 0) store_row<NC>(M + (size_t)k * ldm, o);
  }
}

// L2L, one thread per (cell of one level, child slot): the child's local
// expansion plus the parent's translated to the child's centre.  The eight
// siblings of a parent are neighbouring threads (one parent row load, shared).
template <int P>
__global__ void k_l2l(int64_t lo, int64_t cnt, const uint4 *__restrict__ cell, const int2 *__restrict__ kids, int ldm,
                      float *__restrict__ L, const TreeState *tz, int level) {
  constexpr int NC = ncoef(P);
  tree_level(tz, level, lo, cnt);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 8 * cnt; t += stride) {
    const int64_t k = lo + t / 8;
    const int2 kd = kids[k];
    const int slot = (int)(t % 8);
    if (slot >= kd.y) continue;
    const int ch = kd.x + slot;
    float pl[NC], cl[NC];
    load_row<NC>(L + (size_t)k * ldm, pl);
    float *dst = L + (size_t)ch * ldm;
    load_row<NC>(dst, cl);
    const uint4 cc = cell[ch];
    // (z_C - z_P) / H = -1/4 for the lower half of an axis, +1/4 for the upper
    L2LBody<P>::run((cc.x & 1u) ? 1.f : -1.f, (cc.y & 1u) ? 1.f : -1.f, (cc.z & 1u) ? 1.f : -1.f, pl, cl);
    store_row<NC>(dst, cl);
  }
}

// L2P, one thread per leaf: a = G h^-2 sum L~_{n+e_d} u^n / n!, written in input order.
template <int P>
__global__ void k_l2p(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
                      const uint2 *__restrict__ range, const float4 *__restrict__ pm4, const uint32_t *__restrict__ perm,
                      int64_t n, float box, float G, int ldm, const float *__restrict__ L, float *__restrict__ acc,
                      const TreeState *tz, const float *__restrict__ add) {
  constexpr int NC = ncoef(P);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tree_leaves(tz, nl)) return;
  const uint32_t k = leaves[t];
  const uint2 r = range[k];
  const float inv_h = (float)(1u << cell[k].w) / box;
  const float s = G * inv_h * inv_h;
  float l[NC];
  load_row<NC>(L + (size_t)k * ldm, l);
  for (uint32_t i = r.x; i < r.x + r.y; ++i) {
    const float4 q = pm4[i];
    float ax = 0.f, ay = 0.f, az = 0.f;
    L2PBody<P>::run(q.x * inv_h, q.y * inv_h, q.z * inv_h, l, ax, ay, az);
    const uint32_t o = perm[i];
    if (add) {  // sink batches: the P2P accelerations, added as P2P itself would add them
      acc[o] = s * ax + add[o];
      acc[n + o] = s * ay + add[n + o];
      acc[2 * n + o] = s * az + add[2 * n + o];
    } else {
      acc[o] = s * ax;
      acc[n + o] = s * ay;
      acc[2 * n + o] = s * az;
    }
  }
}

// Level loops: the tree's levels on the host, or (graph mode) the level
// capacity, each launch reading its level's extent from the device tree state
// on a grid sized for the node capacity (at most 16 blocks per SM; the kernels
// loop).
struct LevelLoop {
  const TreeState *tz;
  int levels;
  LevelLoop(Ctx &c) : tz(c.graph_tree ? hfmm::P<TreeState>(c.tstate) : nullptr),
                      levels(c.graph_tree ? c.cap_levels : c.nlevels) {}
  void extent(const Ctx &c, int l, int64_t &lo, int64_t &cnt) const {
    if (tz) {
      lo = 0;
      cnt = (int64_t)c.nnodes;  // a bound: the kernel reads the level's own extent
    } else {
      lo = c.level_start[l];
      cnt = c.level_start[l + 1] - lo;
    }
  }
  unsigned grid(int64_t cnt, int T) const {
    const unsigned g = blocks_for(8 * cnt, T);
    return tz && g > 152u * 16u ? 152u * 16u : g;
  }
};

template <int P>
cudaError_t upward_p(Ctx &c, cudaStream_t st) {
  const int T = 128;
  const float box = (float)c.prm.box;
  const LevelLoop lv(c);
  k_p2m<P><<<blocks_for(c.nleaves, T), T, 0, st>>>(hfmm::P<uint32_t>(c.leaves), c.nleaves, hfmm::P<uint4>(c.cell), hfmm::P<uint2>(c.range),
                                                   hfmm::P<float4>(c.pm4), box, c.ldm, hfmm::P<float>(c.M), lv.tz);
  note_launch();
  for (int l = lv.levels - 2; l >= 0; --l) {
    int64_t lo, cnt;
    lv.extent(c, l, lo, cnt);
    k_m2m<P><<<lv.grid(cnt, T), T, 0, st>>>(lo, cnt, hfmm::P<uint4>(c.cell), hfmm::P<int2>(c.kids), c.ldm,
                                            hfmm::P<float>(c.M), lv.tz, l);
    note_launch();
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t downward_p(Ctx &c, float *acc, cudaStream_t st, const float *add) {
  const int T = 128;
  const LevelLoop lv(c);
  for (int l = 0; l + 1 < lv.levels; ++l) {
    int64_t lo, cnt;
    lv.extent(c, l, lo, cnt);
    k_l2l<P><<<lv.grid(cnt, T), T, 0, st>>>(lo, cnt, hfmm::P<uint4>(c.cell), hfmm::P<int2>(c.kids), c.ldm,
                                            hfmm::P<float>(c.L), lv.tz, l);
    note_launch();
  }
  k_l2p<P><<<blocks_for(c.nleaves, T), T, 0, st>>>(hfmm::P<uint32_t>(c.leaves), c.nleaves, hfmm::P<uint4>(c.cell),
                                                   hfmm::P<uint2>(c.range), hfmm::P<float4>(c.pm4), hfmm::P<uint32_t>(c.idx), c.n,
                                                   (float)c.prm.box, (float)c.prm.G, c.ldm, hfmm::P<float>(c.L), acc,
                                                   lv.tz, add);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- k-d tree (tree = 1)
// The same scaled expansions with a node's scale h (a power of two >= its box
// side) in place of the octree cell side: P2M and L2P as above; the two children
// of a node translate with any offset d (in units of the parent's h) and scale
// ratio rho = h_child / h_parent (M2MGenBody, L2LGenBody); one thread per node,
// the children added in order (deterministic).

template <int P>
__global__ void k_kd_p2m(const uint32_t *__restrict__ leaves, int64_t nl, const uint32_t *__restrict__ first,
                         const uint32_t *__restrict__ count, const float *__restrict__ hs,
                         const float4 *__restrict__ pm4, int ldm, float *__restrict__ M) {
  constexpr int NC = ncoef(P);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const uint32_t k = leaves[t];
  const float inv_h = 1.f / hs[k];
  float acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = 0.f;
  for (uint32_t i = first[k]; i < first[k] + count[k]; ++i) {
    const float4 q = pm4[i];
    P2MBody<P>::run(q.x * inv_h, q.y * inv_h, q.z * inv_h, q.w, acc);
  }
  P2MBody<P>::finish(acc);
  store_row<NC>(M + (size_t)k * ldm, acc);
}

template <int P>
__global__ void k_kd_m2m(int64_t lo, int64_t cnt, const int *__restrict__ child, const double *__restrict__ geo,
                         int64_t cap, const float *__restrict__ hs, int ldm, float *__restrict__ M) {
  constexpr int NC = ncoef(P);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t k = lo + t;
  const int ch0 = child[k];
  if (ch0 < 0) return;
  const float inv_h = 1.f / hs[k];
  float o[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) o[q] = 0.f;
  for (int ch = ch0; ch < ch0 + 2; ++ch) {
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = (float)__dsub_rn(geo[a * cap + k], geo[a * cap + ch]) * inv_h;
    float ci[NC];
    load_row<NC>(M + (size_t)ch * ldm, ci);
    M2MGenBody<P>::run(d[0], d[1], d[2], hs[ch] * inv_h, ci, o);
  }
  store_row<NC>(M + (size_t)k * ldm, o);
}

template <int P>
__global__ void k_kd_l2l(int64_t lo, int64_t cnt, const int *__restrict__ parent, const double *__restrict__ geo,
                         int64_t cap, const float *__restrict__ hs, int ldm, float *__restrict__ L) {
  constexpr int NC = ncoef(P);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t k = lo + t;
  const int p = parent[k];
  const float inv_h = 1.f / hs[p];
  float d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = (float)__dsub_rn(geo[a * cap + k], geo[a * cap + p]) * inv_h;
  float pl[NC], cl[NC];
  load_row<NC>(L + (size_t)p * ldm, pl);
  float *dst = L + (size_t)k * ldm;
  load_row<NC>(dst, cl);
  L2LGenBody<P>::run(d[0], d[1], d[2], hs[k] * inv_h, pl, cl);
  store_row<NC>(dst, cl);
}

template <int P>
__global__ void k_kd_l2p(const uint32_t *__restrict__ leaves, int64_t nl, const uint32_t *__restrict__ first,
                         const uint32_t *__restrict__ count, const float *__restrict__ hs,
                         const float4 *__restrict__ pm4, const uint32_t *__restrict__ perm, int64_t n, float G,
                         int ldm, const float *__restrict__ L, float *__restrict__ acc) {
  constexpr int NC = ncoef(P);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const uint32_t k = leaves[t];
  const float inv_h = 1.f / hs[k];
  const float s = G * inv_h * inv_h;
  float l[NC];
  load_row<NC>(L + (size_t)k * ldm, l);
  for (uint32_t i = first[k]; i < first[k] + count[k]; ++i) {
    const float4 q = pm4[i];
    float ax = 0.f, ay = 0.f, az = 0.f;
    L2PBody<P>::run(q.x * inv_h, q.y * inv_h, q.z * inv_h, l, ax, ay, az);
    const uint32_t o = perm[i];
    acc[o] = s * ax;
    acc[n + o] = s * ay;
    acc[2 * n + o] = s * az;
  }
}

template <int P>
cudaError_t kd_upward_p(Ctx &c, cudaStream_t st) {
  const int T = 128;
  KdTree &kd = c.kd;
  k_kd_p2m<P><<<blocks_for(c.nleaves, T), T, 0, st>>>(hfmm::P<uint32_t>(c.leaves), c.nleaves,
                                                      hfmm::P<uint32_t>(kd.first), hfmm::P<uint32_t>(kd.count),
                                                      hfmm::P<float>(kd.hs), hfmm::P<float4>(c.pm4), c.ldm,
                                                      hfmm::P<float>(c.M));
  note_launch();
  for (int l = c.nlevels - 2; l >= 0; --l) {
    const int64_t lo = kd.level_start[l], cnt = kd.level_start[l + 1] - lo;
    k_kd_m2m<P><<<blocks_for(cnt, T), T, 0, st>>>(lo, cnt, hfmm::P<int>(kd.child), hfmm::P<double>(kd.geo), kd.cap,
                                                 hfmm::P<float>(kd.hs), c.ldm, hfmm::P<float>(c.M));
    note_launch();
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t kd_downward_p(Ctx &c, float *acc, cudaStream_t st) {
  const int T = 128;
  KdTree &kd = c.kd;
  for (int l = 1; l < c.nlevels; ++l) {
    const int64_t lo = kd.level_start[l], cnt = kd.level_start[l + 1] - lo;
    k_kd_l2l<P><<<blocks_for(cnt, T), T, 0, st>>>(lo, cnt, hfmm::P<int>(kd.parent), hfmm::P<double>(kd.geo), kd.cap,
                                                 hfmm::P<float>(kd.hs), c.ldm, hfmm::P<float>(c.L));
    note_launch();
  }
  k_kd_l2p<P><<<blocks_for(c.nleaves, T), T, 0, st>>>(hfmm::P<uint32_t>(c.leaves), c.nleaves,
                                                      hfmm::P<uint32_t>(kd.first), hfmm::P<uint32_t>(kd.count),
                                                      hfmm::P<float>(kd.hs), hfmm::P<float4>(c.pm4),
                                                      hfmm::P<uint32_t>(c.idx), c.n, (float)c.prm.G, c.ldm,
                                                      hfmm::P<float>(c.L), acc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t kd_upward(Ctx &c, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  switch (c.p) {
    case 1: return kd_upward_p<1>(c, st);
    case 2: return kd_upward_p<2>(c, st);
    case 3: return kd_upward_p<3>(c, st);
    case 4: return kd_upward_p<4>(c, st);
    case 5: return kd_upward_p<5>(c, st);
    case 6: return kd_upward_p<6>(c, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t kd_downward(Ctx &c, float *acc, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  switch (c.p) {
    case 1: return kd_downward_p<1>(c, acc, st);
    case 2: return kd_downward_p<2>(c, acc, st);
    case 3: return kd_downward_p<3>(c, acc, st);
    case 4: return kd_downward_p<4>(c, acc, st);
    case 5: return kd_downward_p<5>(c, acc, st);
    case 6: return kd_downward_p<6>(c, acc, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t upward(Ctx &c, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  switch (c.p) {
    case 1: return upward_p<1>(c, st);
    case 2: return upward_p<2>(c, st);
    case 3: return upward_p<3>(c, st);
    case 4: return upward_p<4>(c, st);
    case 5: return upward_p<5>(c, st);
    case 6: return upward_p<6>(c, st);
    case 7: return upward_p<7>(c, st);
    case 8: return upward_p<8>(c, st);
  }
  return cudaErrorInvalidValue;
}

// L2L top-down, then L2P (overwrites acc in input order; P2P adds to it).
cudaError_t downward(Ctx &c, float *acc, cudaStream_t st, const float *add) {
  if (c.nleaves == 0) return cudaSuccess;
  switch (c.p) {
    case 1: return downward_p<1>(c, acc, st, add);
    case 2: return downward_p<2>(c, acc, st, add);
    case 3: return downward_p<3>(c, acc, st, add);
    case 4: return downward_p<4>(c, acc, st, add);
    case 5: return downward_p<5>(c, acc, st, add);
    case 6: return downward_p<6>(c, acc, st, add);
    case 7: return downward_p<7>(c, acc, st, add);
    case 8: return downward_p<8>(c, acc, st, add);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hfmm
