// Octree build (Sec. 2.1, a tree with a leaf limiter; here a Morton octree):
// periodic wrap, 63-bit Morton keys, stable key sort, level-synchronous split
// of cells holding more than leaf_max particles, and per-particle FP32
// offsets from the geometric centre of the leaf.
#include <cooperative_groups.h>

#include <cstring>

#include "common.cuh"

namespace hfmm {
namespace {

namespace cg = cooperative_groups;

__global__ void k_keys(const double *__restrict__ pos, int64_t n, double box, double inv_pow2, uint64_t *__restrict__ key,
                       uint32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = morton_key(pos[i], pos[n + i], pos[2 * n + i], box, inv_pow2);
  idx[i] = (uint32_t)i;
}

__global__ void k_gather(const double *__restrict__ pos, const uint32_t *__restrict__ idx, int64_t n, double box,
                         double inv_pow2,
                         double *__restrict__ xs) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  uint32_t i = idx[s];
  xs[s] = wrap_box_fast(pos[i], box, inv_pow2);
  xs[n + s] = wrap_box_fast(pos[n + i], box, inv_pow2);
  xs[2 * n + s] = wrap_box_fast(pos[2 * n + i], box, inv_pow2);
}


// FP64 offset from the geometric leaf centre, rounded once to FP32 (a thread
// per leaf; the cell side L 2^-level built from its bits: no FP64 division).
__global__ void k_leaf_offsets(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
                               const uint2 *__restrict__ range, const double *__restrict__ xs,
                               const float *__restrict__ mass, const uint32_t *__restrict__ perm, int64_t n,
                               double box, float4 *__restrict__ pm4, const TreeState *tz) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tree_leaves(tz, nl)) return;
  uint32_t k = leaves[t];
  uint4 c = cell[k];
  uint2 r = range[k];
  const double h = box * __longlong_as_double((long long)(1023 - (int)c.w) << 52);
  double zx = ((double)c.x + 0.5) * h, zy = ((double)c.y + 0.5) * h, zz = ((double)c.z + 0.5) * h;
  for (uint32_t i = r.x; i < r.x + r.y; ++i) {
    pm4[i] = make_float4((float)(xs[i] - zx), (float)(xs[n + i] - zy), (float)(xs[2 * n + i] - zz), mass[perm[i]]);
  }
}

constexpr int kBT = 256;


// Level-synchronous octree build in one cooperative launch (Sec. 2.1 tree, as a
// Morton octree): per level every node with more than leaf_max particles (and
// above the depth cap) is split at the octant boundaries of the sorted keys;
// a grid-wide scan of the child counts places the children breadth-first (key
// order within a level) and a scan of the leaf flags lists the leaves.  The
// sizes stay on the device; the host reads them once at the end.
__global__ void __launch_bounds__(kBT) k_tree_levels(const uint64_t *__restrict__ key, int64_t n, int leaf_max,
                                                     uint4 *__restrict__ cell, uint2 *__restrict__ range,
                                                     int2 *__restrict__ kids, uint32_t *__restrict__ leaves,
                                                     unsigned long long capN, uint32_t *__restrict__ nk,
                                                     uint32_t *__restrict__ bnd, unsigned long long *__restrict__ btot,
                                                     TreeState *__restrict__ st, int max_levels) {
  cg::grid_group grid = cg::this_grid();
  __shared__ unsigned long long lo, cnt, total, nleaves;
  __shared__ unsigned long long wsum[kBT / 32][2], pre[2], all[2], run[2];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const unsigned nb = gridDim.x, bid = blockIdx.x;
  if (bid == 0 && tid == 0) {
    cell[0] = make_uint4(0, 0, 0, 0);
    range[0] = make_uint2(0, (uint32_t)n);
    st->level_start[0] = 0;
  }
  if (tid == 0) {
    lo = 0;
    cnt = 1;
    total = 1;
    nleaves = 0;
  }
  __syncthreads();
  grid.sync();
  int level = 0;
  for (; level <= kDepth; ++level) {
    const unsigned long long L0 = lo, C = cnt, T0 = total, N0 = nleaves;
    const unsigned long long ch = (C + nb - 1) / nb;
    const unsigned long long blo = ch * bid < C ? ch * bid : C, bhi = blo + ch < C ? blo + ch : C;
    // phase A: eight lanes per node, lane o finds the first key with octant digit >= o
    // (independent searches over the node's range); child counts and block sums
    unsigned long long sc = 0, sl = 0;
    for (unsigned long long tb = 8 * blo; tb < 8 * bhi; tb += kBT) {  // uniform trip count (shuffles)
      const unsigned long long tt = tb + tid, t = tt / 8;
      const uint32_t o = (uint32_t)(tt % 8);
      const bool valid = tt < 8 * bhi;
      uint2 r = make_uint2(0, 0);
      bool split = false;
      if (valid) {
        r = range[L0 + t];
        split = (int)r.y > leaf_max && level < kDepth;
      }
      uint32_t bo = r.x;
      if (split && o > 0) {
        const int shift = 3 * (kDepth - level - 1);
        uint32_t a = r.x, e = r.x + r.y;
        while (a < e) {
          const uint32_t mid = a + (e - a) / 2;
          if (((uint32_t)(key[mid] >> shift) & 7u) < o)
            a = mid + 1;
          else
            e = mid;
        }
        bo = a;
      }
      // boundary o + 1 from the next lane of the group (the last lane: the range end)
      uint32_t bn = __shfl_down_sync(0xffffffffu, bo, 1, 8);
      if (o == 7) bn = r.x + r.y;
      const uint32_t nonempty = split && bn > bo ? 1u : 0u;
      uint32_t c = nonempty;
      c += __shfl_xor_sync(0xffffffffu, c, 1, 8);
      c += __shfl_xor_sync(0xffffffffu, c, 2, 8);
      c += __shfl_xor_sync(0xffffffffu, c, 4, 8);
      if (valid) {
        bnd[9 * t + o] = bo;
        if (o == 7) bnd[9 * t + 8] = r.x + r.y;
        if (o == 0) {
          nk[t] = c;
          sc += c;
          sl += c == 0;
        }
      }
    }
    for (int o = 16; o; o >>= 1) {
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
      sl += __shfl_xor_sync(0xffffffffu, sl, o);
    }
    if (lane == 0) {
      wsum[wp][0] = sc;
      wsum[wp][1] = sl;
    }
    __syncthreads();
    if (tid < 2) {
      unsigned long long v = 0;
      for (int q = 0; q < kBT / 32; ++q) v += wsum[q][tid];
      btot[2 * bid + tid] = v;
    }
    __threadfence();
    grid.sync();
    // phase B: block prefixes, then each node's children and leaf slot
    if (tid < 2) {
      unsigned long long b = 0, a = 0;
      for (unsigned q = 0; q < nb; ++q) {
        const unsigned long long v = btot[2 * q + tid];
        if (q < bid) b += v;
        a += v;
      }
      pre[tid] = b;
      all[tid] = a;
      run[tid] = b;
    }
    __syncthreads();
    const unsigned long long Cn = all[0], Ln = all[1];
    // node capacity, or (graph mode) more levels than the host sized its level loops for
    if (T0 + Cn > capN || (Cn > 0 && level + 2 > max_levels)) {
      if (bid == 0 && tid == 0) st->overflow = 1;
      break;  // every block takes the same decision
    }
    for (unsigned long long tb = blo; tb < bhi; tb += kBT) {
      const unsigned long long t = tb + tid;
      const bool valid = t < bhi;
      const uint32_t c = valid ? nk[t] : 0u;
      const unsigned long long lf = valid && c == 0 ? 1ull : 0ull;
      unsigned long long xc = c, xl = lf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long yc = __shfl_up_sync(0xffffffffu, xc, o), yl = __shfl_up_sync(0xffffffffu, xl, o);
        if (lane >= o) {
          xc += yc;
          xl += yl;
        }
      }
      if (lane == 31) {
        wsum[wp][0] = xc;
        wsum[wp][1] = xl;
      }
      __syncthreads();
      unsigned long long wc = 0, wl = 0, tc = 0, tl = 0;
      for (int q = 0; q < kBT / 32; ++q) {
        if (q < wp) {
          wc += wsum[q][0];
          wl += wsum[q][1];
        }
        tc += wsum[q][0];
        tl += wsum[q][1];
      }
      if (valid) {
        const unsigned long long k = L0 + t;
        if (c == 0) {
          kids[k] = make_int2(-1, 0);
          leaves[N0 + run[1] + wl + xl - lf] = (uint32_t)k;
        } else {
          const unsigned long long base = T0 + run[0] + wc + xc - c;
          kids[k] = make_int2((int)base, (int)c);
          const uint4 pc = cell[k];
          uint32_t b[9];
#pragma unroll
          for (int o = 0; o < 9; ++o) b[o] = bnd[9 * t + o];
          uint32_t q = 0;
          for (uint32_t o = 0; o < 8; ++o) {
            if (b[o + 1] > b[o]) {
              cell[base + q] = make_uint4(2 * pc.x + ((o >> 2) & 1u), 2 * pc.y + ((o >> 1) & 1u), 2 * pc.z + (o & 1u),
                                          pc.w + 1);
              range[base + q] = make_uint2(b[o], b[o + 1] - b[o]);
              ++q;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        run[0] += tc;
        run[1] += tl;
      }
      __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      lo = T0;
      cnt = Cn;
      total = T0 + Cn;
      nleaves = N0 + Ln;
    }
    if (bid == 0 && tid == 0) st->level_start[level + 1] = T0;  // start of level + 1 (or the end)
    grid.sync();
    if (Cn == 0) {
      ++level;
      break;
    }
  }
  if (bid == 0 && tid == 0) {
    st->total = total;
    st->nleaves = nleaves;
    st->nlevels = level;
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
  const double inv_pow2 = box_inverse_if_pow2(c.prm.box);
  k_keys<<<blocks_for(n, T), T, 0, st>>>(pos, n, c.prm.box, inv_pow2, P<uint64_t>(c.key), P<uint32_t>(c.idx));
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
  k_gather<<<blocks_for(n, T), T, 0, st>>>(pos, perm, n, c.prm.box, inv_pow2, P<double>(c.xs));
  note_launch();

  // octree levels: one cooperative launch; node capacity from the last build, grown on overflow
  if (c.cap_nodes < (uint64_t)(2 * n / (c.prm.leaf_max > 1 ? c.prm.leaf_max : 1) + 64))
    c.cap_nodes = (uint64_t)(2 * n / (c.prm.leaf_max > 1 ? c.prm.leaf_max : 1) + 64);
  int dev = 0, nsm = 0, per_sm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_levels, kBT, 0));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned nb = (unsigned)(nsm * (per_sm < 2 ? per_sm : 2));
  TreeState hs{};
  TreeState *dst = reinterpret_cast<TreeState *>(c.tstate.p);
  TRY(ensure(c.tstate, sizeof(TreeState)));
  dst = reinterpret_cast<TreeState *>(c.tstate.p);
  TRY(ensure(c.bounds, (size_t)nb * 2 * sizeof(unsigned long long)));
  for (int attempt = 0;; ++attempt) {
    if (attempt == 8) return cudaErrorInvalidValue;
    const unsigned long long capN = c.cap_nodes;
    TRY(ensure(c.cell, capN * sizeof(uint4)));
    TRY(ensure(c.range, capN * sizeof(uint2)));
    TRY(ensure(c.kids, capN * sizeof(int2)));
    TRY(ensure(c.leaves, capN * sizeof(uint32_t)));
    TRY(ensure(c.nkids, capN * sizeof(uint32_t)));
    TRY(ensure(c.koff, capN * 9 * sizeof(uint32_t)));  // octant boundaries of a level's nodes
    TRY(cudaMemsetAsync(dst, 0, sizeof(TreeState), st));
    uint4 *cl = P<uint4>(c.cell);
    uint2 *rg = P<uint2>(c.range);
    int2 *kd = P<int2>(c.kids);
    uint32_t *lv = P<uint32_t>(c.leaves), *nkp = P<uint32_t>(c.nkids), *bd = P<uint32_t>(c.koff);
    unsigned long long *bt = P<unsigned long long>(c.bounds);
    int lm = c.prm.leaf_max, ml = kDepth + 1;
    int64_t nn = n;
    void *args[] = {(void *)&key, (void *)&nn, (void *)&lm, (void *)&cl, (void *)&rg, (void *)&kd, (void *)&lv,
                    (void *)&capN, (void *)&nkp, (void *)&bd, (void *)&bt, (void *)&dst, (void *)&ml};
    TRY(cudaLaunchCooperativeKernel((const void *)k_tree_levels, dim3(nb), dim3(kBT), args, 0, st));
    note_launch();
    TRY(cudaMemcpyAsync(c.h_pinned, dst, sizeof(TreeState), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    std::memcpy(&hs, c.h_pinned, sizeof(TreeState));
    if (!hs.overflow) break;
    c.cap_nodes *= 2;
  }
  const int64_t total = (int64_t)hs.total;
  c.nlevels = hs.nlevels;
  for (int l = 0; l <= hs.nlevels && l < kDepth + 3; ++l) c.level_start[l] = (int64_t)hs.level_start[l];
  c.nnodes = total;
  c.nleaves = (int64_t)hs.nleaves;
  if (total >= ((int64_t)1 << kSinkBits)) return cudaErrorInvalidValue;  // mapped to HFMM_ERR_CAPACITY
  k_leaf_offsets<<<blocks_for(c.nleaves, T), T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint4>(c.cell),
                                                         P<uint2>(c.range), P<double>(c.xs), mass, perm, n,
                                                         c.prm.box, P<float4>(c.pm4), nullptr);
  note_launch();
  TRY(cudaGetLastError());
  if (c.prm.profile & 1) cudaEventRecord(c.ev[2], st);
  c.have_tree = true;
  return cudaSuccess;
#undef TRY
}

// Graph mode (a step captured as one graph): every buffer of the build sized
// for n particles and the node capacity (outside the capture) ...
cudaError_t build_tree_prepare(Ctx &c, int64_t n) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  TRY(ensure(c.key, n * 8));
  TRY(ensure(c.key_alt, n * 8));
  TRY(ensure(c.idx, n * 4));
  TRY(ensure(c.idx_alt, n * 4));
  TRY(ensure(c.xs, n * 24));
  TRY(ensure(c.pm4, n * 16));
  TRY(ensure(c.tmp, radix_sort_scratch_bytes((size_t)n)));
  if (c.cap_nodes < (uint64_t)(2 * n / (c.prm.leaf_max > 1 ? c.prm.leaf_max : 1) + 64))
    c.cap_nodes = (uint64_t)(2 * n / (c.prm.leaf_max > 1 ? c.prm.leaf_max : 1) + 64);
  const unsigned long long capN = c.cap_nodes;
  TRY(ensure(c.cell, capN * sizeof(uint4)));
  TRY(ensure(c.range, capN * sizeof(uint2)));
  TRY(ensure(c.kids, capN * sizeof(int2)));
  TRY(ensure(c.leaves, capN * sizeof(uint32_t)));
  TRY(ensure(c.nkids, capN * sizeof(uint32_t)));
  TRY(ensure(c.koff, capN * 9 * sizeof(uint32_t)));
  TRY(ensure(c.tstate, sizeof(TreeState)));
  // levels the graph's level loops cover: the last tree's and two more
  if (c.cap_levels < c.nlevels + 2) c.cap_levels = c.nlevels + 2;
  if (c.cap_levels > kDepth + 1) c.cap_levels = kDepth + 1;
  int dev = 0, nsm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TRY(ensure(c.bounds, (size_t)nsm * 2 * 2 * sizeof(unsigned long long)));
  return cudaSuccess;
#undef TRY
}

// ... and the build enqueued with no read-back: the sizes stay in the device
// state (c.tstate), which the later kernels of the graph read; a node capacity
// overflow shows there too and makes them treat the tree as empty.
cudaError_t build_tree_launch(Ctx &c, const double *pos, const float *mass, int64_t n, cudaStream_t st) {
  cudaError_t e;
  const int T = 256;
  const double inv_pow2 = box_inverse_if_pow2(c.prm.box);
  k_keys<<<blocks_for(n, T), T, 0, st>>>(pos, n, c.prm.box, inv_pow2, P<uint64_t>(c.key), P<uint32_t>(c.idx));
  note_launch();
  bool alt = false;
  if ((e = radix_sort_u64(P<uint64_t>(c.key), P<uint32_t>(c.idx), P<uint64_t>(c.key_alt), P<uint32_t>(c.idx_alt), n,
                          0, 63, &alt, c.tmp, st)) != cudaSuccess)
    return e;
  if (alt) {
    std::swap(c.key, c.key_alt);
    std::swap(c.idx, c.idx_alt);
  }
  uint64_t *key = P<uint64_t>(c.key);
  uint32_t *perm = P<uint32_t>(c.idx);
  k_gather<<<blocks_for(n, T), T, 0, st>>>(pos, perm, n, c.prm.box, inv_pow2, P<double>(c.xs));
  note_launch();
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_levels, kBT, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned nb = (unsigned)(nsm * (per_sm < 2 ? per_sm : 2));
  TreeState *dst = P<TreeState>(c.tstate);
  if ((e = cudaMemsetAsync(dst, 0, sizeof(TreeState), st)) != cudaSuccess) return e;
  unsigned long long capN = c.cap_nodes;
  uint4 *cl = P<uint4>(c.cell);
  uint2 *rg = P<uint2>(c.range);
  int2 *kd = P<int2>(c.kids);
  uint32_t *lv = P<uint32_t>(c.leaves), *nkp = P<uint32_t>(c.nkids), *bd = P<uint32_t>(c.koff);
  unsigned long long *bt = P<unsigned long long>(c.bounds);
  int lm = c.prm.leaf_max, ml = c.cap_levels;
  int64_t nn = n;
  void *args[] = {(void *)&key, (void *)&nn, (void *)&lm, (void *)&cl, (void *)&rg, (void *)&kd, (void *)&lv,
                  (void *)&capN, (void *)&nkp, (void *)&bd, (void *)&bt, (void *)&dst, (void *)&ml};
  if ((e = cudaLaunchCooperativeKernel((const void *)k_tree_levels, dim3(nb), dim3(kBT), args, 0, st)) != cudaSuccess)
    return e;
  note_launch();
  k_leaf_offsets<<<blocks_for(c.cap_nodes, T), T, 0, st>>>(P<uint32_t>(c.leaves), (int64_t)c.cap_nodes,
                                                           P<uint4>(c.cell), P<uint2>(c.range), P<double>(c.xs),
                                                           mass, perm, n, c.prm.box, P<float4>(c.pm4), dst);
  note_launch();
  return cudaGetLastError();
}

// After the graph: the device state's sizes on the host.  False on an overflow
// of the node or level capacity (both are then grown for the next capture).
bool build_tree_finish(Ctx &c, const TreeState &hs) {
  if (hs.overflow) {
    // which limit it was is not recorded: grow both (the direct rebuild sizes them exactly)
    c.cap_nodes *= 2;
    c.cap_levels = c.cap_levels + 2 > kDepth + 1 ? kDepth + 1 : c.cap_levels + 2;
    return false;
  }
  c.nlevels = hs.nlevels;
  for (int l = 0; l <= hs.nlevels && l < kDepth + 3; ++l) c.level_start[l] = (int64_t)hs.level_start[l];
  c.nnodes = (int64_t)hs.total;
  c.nleaves = (int64_t)hs.nleaves;
  c.have_tree = c.nnodes < ((int64_t)1 << kSinkBits);
  return c.have_tree;
}

}  // namespace hfmm
