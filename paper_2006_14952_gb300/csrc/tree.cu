// Octree build (Sec. 2.1, a tree with a leaf limiter; here a Morton octree):
// periodic wrap, 63-bit Morton keys, stable key sort, level-synchronous split
// of cells holding more than leaf_max particles, and per-particle FP32
// offsets from the geometric centre of the leaf.
#include "common.cuh"

namespace hfmm {
namespace {

// x - L floor(x / L), each operation rounded separately (no FMA contraction).
__device__ __forceinline__ double wrap_box(double x, double box) {
  double q = floor(__ddiv_rn(x, box));
  return __dsub_rn(x, __dmul_rn(box, q));
}

__device__ __forceinline__ uint32_t grid_coord(double w, double box) {
  double t = floor(__dmul_rn(__ddiv_rn(w, box), 2097152.0));
  t = fmax(0.0, fmin(t, 2097151.0));
  return (uint32_t)t;
}

// spread the low 21 bits of v to every third bit
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__global__ void k_keys(const double *__restrict__ pos, int64_t n, double box, uint64_t *__restrict__ key,
                       uint32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k0 = grid_coord(wrap_box(pos[i], box), box);
  uint32_t k1 = grid_coord(wrap_box(pos[n + i], box), box);
  uint32_t k2 = grid_coord(wrap_box(pos[2 * n + i], box), box);
  key[i] = (spread3(k0) << 2) | (spread3(k1) << 1) | spread3(k2);
  idx[i] = (uint32_t)i;
}

__global__ void k_gather(const double *__restrict__ pos, const uint32_t *__restrict__ idx, int64_t n, double box,
                         double *__restrict__ xs) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  uint32_t i = idx[s];
  xs[s] = wrap_box(pos[i], box);
  xs[n + s] = wrap_box(pos[n + i], box);
  xs[2 * n + s] = wrap_box(pos[2 * n + i], box);
}

__global__ void k_root(uint4 *cell, uint2 *range, int64_t n) {
  cell[0] = make_uint4(0, 0, 0, 0);
  range[0] = make_uint2(0, (uint32_t)n);
}

// For each node of one level: child boundaries by binary search on the sorted
// keys (the octant digit is monotone inside the parent's range).
__global__ void k_split_count(const uint2 *__restrict__ range, int64_t lo, int64_t cnt, int level, int leaf_max,
                              const uint64_t *__restrict__ key, uint32_t *__restrict__ bounds,
                              uint32_t *__restrict__ nk) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  uint2 r = range[lo + t];
  if ((int)r.y <= leaf_max || level >= kDepth) {
    nk[t] = 0;
    return;
  }
  const int shift = 3 * (kDepth - level - 1);
  uint32_t b[9];
  b[0] = r.x;
  b[8] = r.x + r.y;
  for (uint32_t o = 1; o < 8; ++o) {
    uint32_t a = b[o - 1], e = r.x + r.y;  // first index with digit >= o
    while (a < e) {
      uint32_t m = a + (e - a) / 2;
      if (((uint32_t)(key[m] >> shift) & 7u) < o)
        a = m + 1;
      else
        e = m;
    }
    b[o] = a;
  }
  uint32_t c = 0;
  for (int o = 0; o < 8; ++o) {
    bounds[t * 9 + o] = b[o];
    c += b[o + 1] > b[o];
  }
  bounds[t * 9 + 8] = b[8];
  nk[t] = c;
}

__global__ void k_emit_children(int64_t lo, int64_t cnt, int64_t next_lo, const uint32_t *__restrict__ bounds,
                                const uint32_t *__restrict__ nk, const uint32_t *__restrict__ koff,
                                uint4 *__restrict__ cell, uint2 *__restrict__ range, int2 *__restrict__ kids) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  int64_t k = lo + t;
  uint32_t c = nk[t];
  if (c == 0) {
    kids[k] = make_int2(-1, 0);
    return;
  }
  int64_t base = next_lo + koff[t];
  kids[k] = make_int2((int)base, (int)c);
  uint4 pc = cell[k];
  uint32_t q = 0;
  for (uint32_t o = 0; o < 8; ++o) {
    uint32_t b0 = bounds[t * 9 + o], b1 = bounds[t * 9 + o + 1];
    if (b1 > b0) {
      cell[base + q] = make_uint4(2 * pc.x + ((o >> 2) & 1u), 2 * pc.y + ((o >> 1) & 1u), 2 * pc.z + (o & 1u), pc.w + 1);
      range[base + q] = make_uint2(b0, b1 - b0);
      ++q;
    }
  }
}

__global__ void k_leaf_flags(const int2 *__restrict__ kids, int64_t nn, uint32_t *__restrict__ flag) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn) flag[k] = kids[k].y == 0;
}

__global__ void k_leaf_list(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ off, int64_t nn,
                            uint32_t *__restrict__ leaves) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn && flag[k]) leaves[off[k]] = (uint32_t)k;
}

// FP64 offset from the geometric leaf centre, rounded once to FP32.
__global__ void k_leaf_offsets(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
                               const uint2 *__restrict__ range, const double *__restrict__ xs,
                               const float *__restrict__ mass, const uint32_t *__restrict__ perm, int64_t n,
                               double box, float4 *__restrict__ pm4) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  uint32_t k = leaves[t];
  uint4 c = cell[k];
  uint2 r = range[k];
  double h = box / (double)(1u << c.w);
  double zx = ((double)c.x + 0.5) * h, zy = ((double)c.y + 0.5) * h, zz = ((double)c.z + 0.5) * h;
  for (uint32_t i = r.x; i < r.x + r.y; ++i) {
    pm4[i] = make_float4((float)(xs[i] - zx), (float)(xs[n + i] - zy), (float)(xs[2 * n + i] - zz), mass[perm[i]]);
  }
}

}  // namespace

cudaError_t build_tree(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  c.n = n;
  c.nnodes = c.nleaves = 0;
  c.nlevels = 0;
  c.have_tree = false;
  if (n == 0) {
    c.have_tree = true;
    return cudaSuccess;
  }
  const int T = 256;
  TRY(ensure(c.key, n * 8));
  TRY(ensure(c.key_alt, n * 8));
  TRY(ensure(c.idx, n * 4));
  TRY(ensure(c.idx_alt, n * 4));
  TRY(ensure(c.xs, n * 24));
  TRY(ensure(c.pm4, n * 16));
  TRY(ensure(c.d_small, 256));
  if (c.prm.profile & 1) cudaEventRecord(c.ev[0], st);
  k_keys<<<blocks_for(n, T), T, 0, st>>>(pos, n, c.prm.box, P<uint64_t>(c.key), P<uint32_t>(c.idx));
  note_launch();
  bool alt = false;
  TRY(radix_sort_u64(P<uint64_t>(c.key), P<uint32_t>(c.idx), P<uint64_t>(c.key_alt), P<uint32_t>(c.idx_alt), n, 0,
                     63, &alt, c.tmp, st));
  if (alt) {
    std::swap(c.key, c.key_alt);
    std::swap(c.idx, c.idx_alt);
  }
  uint64_t *key = P<uint64_t>(c.key);
  uint32_t *perm = P<uint32_t>(c.idx);
  if (c.prm.profile & 1) cudaEventRecord(c.ev[1], st);
  k_gather<<<blocks_for(n, T), T, 0, st>>>(pos, perm, n, c.prm.box, P<double>(c.xs));
  note_launch();

  // level-synchronous node build
  size_t cap_nodes = (size_t)(2 * n / (c.prm.leaf_max > 1 ? c.prm.leaf_max : 1) + 64);
  TRY(ensure(c.cell, cap_nodes * sizeof(uint4)));
  TRY(ensure(c.range, cap_nodes * sizeof(uint2)));
  TRY(ensure(c.kids, cap_nodes * sizeof(int2)));
  k_root<<<1, 1, 0, st>>>(P<uint4>(c.cell), P<uint2>(c.range), n);
  note_launch();
  int64_t lo = 0, cnt = 1, total = 1;
  int level = 0;
  c.level_start[0] = 0;
  uint64_t *d_tot = P<uint64_t>(c.d_small);
  for (;;) {
    TRY(ensure(c.bounds, cnt * 9 * sizeof(uint32_t)));
    TRY(ensure(c.nkids, cnt * sizeof(uint32_t)));
    TRY(ensure(c.koff, cnt * sizeof(uint32_t)));
    k_split_count<<<blocks_for(cnt, T), T, 0, st>>>(P<uint2>(c.range), lo, cnt, level, c.prm.leaf_max, key,
                                                    P<uint32_t>(c.bounds), P<uint32_t>(c.nkids));
    note_launch();
    TRY(scan_u32(P<uint32_t>(c.nkids), P<uint32_t>(c.koff), d_tot, cnt, c.tmp2, st));
    TRY(cudaMemcpyAsync(c.h_pinned, d_tot, 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    int64_t nxt = (int64_t)c.h_pinned[0];
    if (total + nxt > (int64_t)cap_nodes) {
      size_t nc = (size_t)(total + nxt) * 2;
      TRY(ensure_keep(c.cell, nc * sizeof(uint4), total * sizeof(uint4), st));
      TRY(ensure_keep(c.range, nc * sizeof(uint2), total * sizeof(uint2), st));
      TRY(ensure_keep(c.kids, nc * sizeof(int2), total * sizeof(int2), st));
      cap_nodes = nc;
    }
    k_emit_children<<<blocks_for(cnt, T), T, 0, st>>>(lo, cnt, total, P<uint32_t>(c.bounds), P<uint32_t>(c.nkids),
                                                      P<uint32_t>(c.koff), P<uint4>(c.cell), P<uint2>(c.range),
                                                      P<int2>(c.kids));
    note_launch();
    TRY(cudaGetLastError());
    ++level;
    if (nxt == 0) break;
    lo = total;
    cnt = nxt;
    total += nxt;
    c.level_start[level] = lo;
  }
  c.nlevels = level;
  c.level_start[level] = total;
  c.nnodes = total;
  if (total >= ((int64_t)1 << kSinkBits)) return cudaErrorInvalidValue;  // mapped to HFMM_ERR_CAPACITY

  // leaves
  TRY(ensure(c.nkids, total * sizeof(uint32_t)));
  TRY(ensure(c.koff, total * sizeof(uint32_t)));
  k_leaf_flags<<<blocks_for(total, T), T, 0, st>>>(P<int2>(c.kids), total, P<uint32_t>(c.nkids));
  note_launch();
  TRY(scan_u32(P<uint32_t>(c.nkids), P<uint32_t>(c.koff), d_tot, total, c.tmp2, st));
  TRY(cudaMemcpyAsync(c.h_pinned, d_tot, 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  c.nleaves = (int64_t)c.h_pinned[0];
  TRY(ensure(c.leaves, c.nleaves * sizeof(uint32_t)));
  k_leaf_list<<<blocks_for(total, T), T, 0, st>>>(P<uint32_t>(c.nkids), P<uint32_t>(c.koff), total,
                                                  P<uint32_t>(c.leaves));
  note_launch();
  k_leaf_offsets<<<blocks_for(c.nleaves, T), T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint4>(c.cell),
                                                         P<uint2>(c.range), P<double>(c.xs), mass, perm, n,
                                                         c.prm.box, P<float4>(c.pm4));
  note_launch();
  TRY(cudaGetLastError());
  if (c.prm.profile & 1) cudaEventRecord(c.ev[2], st);
  c.have_tree = true;
  return cudaSuccess;
#undef TRY
}

}  // namespace hfmm
