// Dual-tree traversal with the hybrid multipole acceptance criterion (Sec. 2.3):
//  1. skip a cell pair whose minimum separation S_m exceeds the cut-off R_c;
//  2. accept M2L when theta = L / S_c <= theta_MAC, otherwise open the larger
//     cell (both on a tie; the other one when the larger is a leaf);
//  3. always open pairs in the transition region (S_c > R_c >= S_m as printed,
//     or S_max > R_c >= S_m with transition_rule 1).
// Two leaves that are not accepted become a P2P pair.  Distances are exact
// integers in half units (L / 2^22); the comparisons use one FP64 product each,
// so the decisions are reproducible bit for bit.
//
// The traversal is level-synchronous: a frontier of packed (sink, source,
// shift) pairs is classified, the outputs are counted and prefix-summed, and
// the M2L pairs, P2P pairs and child pairs are written in frontier order.
//
// Learned acceptance (mac_mode 1) keeps rules 1 and 3 and the self-pair rule;
// in place of rule 2 a pair whose larger side satisfies L / S_c <= theta (the
// safety bound) is a candidate: its 12 features go through the network
// (mlp.cuh, tensor-core inference, batches of 16 candidates per warp) and the
// class chooses between opening the pair and M2L at an order q = 2..p.
// Collection mode records a hash-sampled subset of candidates while opening
// every pair (training data for the network).
#include <cooperative_groups.h>

#include <cstring>

#include "mlp.cuh"

namespace cg = cooperative_groups;

namespace hfmm {
namespace {

enum : uint8_t { kSkip = 0, kM2L = 1, kP2P = 2, kOpenA = 3, kOpenB = 4, kOpenAB = 5 };
constexpr uint8_t kCandidate = 6;  // internal: needs the network's decision

struct Mac {
  int64_t rc2i;                 // floor of (R_c in half units)^2
  int64_t acc_thr[kDepth + 1];  // accept iff S_c^2 >= acc_thr[level of the larger cell]
  int rule, size_rule;
  int mode;   // 0 geometric, 1 learned, 2 collect
  int order;  // p (geometric M2L order, and the largest learned order)
  int tab_k;  // operator-table half extent (0: no table)
  // learned / collect
  const __nv_bfloat16 *w;
  const float *M;
  const uint2 *range;
  int ldm;
  float inv_rs_h, inv_rc_h;
  uint64_t *cand;
  unsigned long long *ncand;
  uint64_t cand_cap;
  uint32_t sample_mod;
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ uint8_t open_rule(uint4 ca, uint4 cb, int2 ka, int2 kb) {
  bool la = ka.y == 0, lb = kb.y == 0;
  if (la && lb) return kP2P;
  if (la) return kOpenB;
  if (lb) return kOpenA;
  if (ca.w < cb.w) return kOpenA;
  if (cb.w < ca.w) return kOpenB;
  return kOpenAB;
}

__device__ __forceinline__ uint8_t classify(uint4 ca, uint4 cb, uint32_t s, int2 ka, int2 kb, const Mac &m) {
  int dd[3];
  half_delta32(ca, cb, s, dd);
  const int ext = (1 << (kDepth - ca.w)) + (1 << (kDepth - cb.w));
  int64_t sc2 = 0, sm2 = 0, sx2 = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int a = dd[d] < 0 ? -dd[d] : dd[d];
    const int g = a - ext > 0 ? a - ext : 0;
    const int f = a + ext;
    sc2 += (int64_t)a * a;
    sm2 += (int64_t)g * g;
    sx2 += (int64_t)f * f;
  }
  if (sm2 > m.rc2i) return kSkip;
  const bool trans = m.rule == 0 ? sc2 > m.rc2i : sx2 > m.rc2i;
  const uint32_t lv = m.size_rule == 0 ? cb.w : (ca.w < cb.w ? ca.w : cb.w);  // level of the cell setting L
  if (!trans && sc2 >= m.acc_thr[lv]) return m.mode == 0 ? kM2L : kCandidate;  // acc_thr >= 1: self pairs open
  return open_rule(ca, cb, ka, kb);
}

// One frontier pair: its class (bits 0..2) and M2L order (bits 3..6), and the
// number of M2L entries, P2P entries and child pairs it produces.  Called by
// all 32 lanes of a warp (the network runs on warp batches of candidates).
struct Item {
  uint8_t cls;
  uint32_t nm, np, nch;
};

// An M2L pair outside the operator table: cells of different levels, or a
// cell offset beyond the table's extent in some axis.
__device__ __forceinline__ bool table_miss(uint4 ca, uint4 cb, uint32_t s, int k) {
  if (k == 0 || ca.w != cb.w) return true;
  int dd[3];
  half_delta32(ca, cb, s, dd);
  const int lim = (2 << (kDepth - ca.w)) * k;  // k cell sides
  return dd[0] > lim || dd[0] < -lim || dd[1] > lim || dd[1] < -lim || dd[2] > lim || dd[2] < -lim;
}

template <bool kNet>
__device__ __forceinline__ Item mac_item(const uint64_t *__restrict__ f, int64_t t, bool valid,
                                         const uint4 *__restrict__ cell, const int2 *__restrict__ kids, const Mac &m,
                                         const uint32_t *sw, __nv_bfloat16 *xs, uint8_t *dec) {
  const int lane = threadIdx.x & 31;
  uint64_t e = 0;
  uint32_t a = 0, b = 0, s = 0;
  int2 ka = make_int2(-1, 0), kb = make_int2(-1, 0);
  uint4 ca = make_uint4(0, 0, 0, 0), cb = ca;
  uint8_t c = kSkip;
  uint32_t order = (uint32_t)m.order;
  if (valid) {
    e = f[t];
    a = pair_sink(e);
    b = pair_src(e);
    s = pair_shift(e);
    ka = kids[a];
    kb = kids[b];
    ca = cell[a];
    cb = cell[b];
    c = classify(ca, cb, s, ka, kb, m);
  }
  if (m.mode == 2 && c == kCandidate) {
    if (mix64(e) % m.sample_mod == 0) {
      const unsigned long long q = atomicAdd(m.ncand, 1ull);
      if (q < m.cand_cap) m.cand[q] = e;
    }
    c = open_rule(ca, cb, ka, kb);
  }
  if (kNet && m.mode == 1) {  // warp-batched network decisions for the candidates
    const unsigned want = __ballot_sync(0xffffffffu, c == kCandidate);
    if (want) {
      const int slot = __popc(want & ((1u << lane) - 1u)), nc = __popc(want);
      __nv_bfloat16 *row = xs + slot * 16;
      if (c == kCandidate) {
        float ft[kMlpIn];
        pair_features(ca, cb, s, m.range[a].y, m.range[b].y, m.M + (size_t)b * m.ldm, m.inv_rs_h, m.inv_rc_h, ft);
#pragma unroll
        for (int k = 0; k < 16; ++k) row[k] = __float2bfloat16_rn(k < kMlpIn ? ft[k] : 0.f);
      }
      for (int r = nc + lane; r < ((nc + 15) & ~15); r += 32)
#pragma unroll
        for (int k = 0; k < 16; ++k) xs[r * 16 + k] = __float2bfloat16_rn(0.f);
      __syncwarp();
      for (int bt = 0; bt < nc; bt += 16) {
        float l[4];
        mlp_logits16(sw, xs + bt * 16, l);
        int c0, c8;
        mlp_argmax16(l, c0, c8);
        if ((lane & 3) == 0) {
          dec[bt + (lane >> 2)] = (uint8_t)c0;
          dec[bt + (lane >> 2) + 8] = (uint8_t)c8;
        }
      }
      __syncwarp();
      if (c == kCandidate) {
        const int k = dec[slot];
        if (k == 0) {
          c = open_rule(ca, cb, ka, kb);
        } else {
          c = kM2L;
          order = (uint32_t)(k + 1) < order ? (uint32_t)(k + 1) : order;
        }
      }
      __syncwarp();
    }
  }
  Item it;
  const uint32_t miss = (c == kM2L && table_miss(ca, cb, s, m.tab_k)) ? 1u : 0u;
  it.cls = (uint8_t)(c | (order << 3) | (miss << 7));
  it.nm = c == kM2L;
  it.np = c == kP2P;
  it.nch = c == kOpenA ? (uint32_t)ka.y : c == kOpenB ? (uint32_t)kb.y : c == kOpenAB ? (uint32_t)(ka.y * kb.y) : 0u;
  return it;
}

struct TravState {
  unsigned long long nm2l, np2p, nf;
  int iters, overflow;
};

constexpr int kTT = 256;  // threads of the traversal kernel

// Persistent level-synchronous traversal: one cooperative launch processes
// every level.  Per level each block classifies a contiguous chunk of the
// frontier and publishes its counts; after a grid barrier every block forms
// its output offsets from the counts of the blocks before it and writes its
// M2L entries, P2P entries and child pairs in frontier order (the same order
// as a serial pass, so the lists are deterministic).  Outputs beyond the
// given capacities set st->overflow and stop the walk; the host grows the
// buffers and runs it again.
template <bool kNet>
__global__ void __launch_bounds__(kTT, kNet ? 2 : 4) k_traverse(const uint4 *__restrict__ cell,
                                                  const int2 *__restrict__ kids, Mac m,
                                                  uint64_t *fa, uint64_t *fb, unsigned long long capF,
                                                  uint8_t *__restrict__ cls, uint64_t *__restrict__ m2l,
                                                  unsigned long long capM, uint64_t *__restrict__ p2p,
                                                  unsigned long long capP, uint32_t *__restrict__ btot,
                                                  TravState *__restrict__ st, int max_iters) {
  cg::grid_group grid = cg::this_grid();
  constexpr int kSw = kNet ? kMlpSmemWords : 1, kXs = kNet ? 32 * 16 : 1, kDec = kNet ? 32 : 1;
  __shared__ uint32_t sw[kSw];
  __shared__ __align__(16) __nv_bfloat16 xs[kTT / 32][kXs];
  __shared__ uint8_t dec[kTT / 32][kDec];
  __shared__ uint32_t ws[kTT / 32][3];
  __shared__ unsigned long long pre[3], sums[3];
  if (kNet) mlp_stage(m.w, sw);
  const int tid = threadIdx.x, wp = tid >> 5;
  const unsigned nb = gridDim.x, bid = blockIdx.x;
  if (bid == 0 && tid < 27) fa[tid] = pack_pair(0, 0, (uint32_t)tid);
  __syncthreads();
  grid.sync();
  uint64_t *cur = fa, *nxt = fb;
  unsigned long long nf = 27, nm = 0, np = 0;
  const int lane = tid & 31;
  constexpr int kW = kTT / 32;
  int iter = 0;
  for (; iter < max_iters && nf > 0; ++iter) {
    // block range, then one contiguous sub-range per warp
    const unsigned long long chunk = (nf + nb - 1) / nb;
    const unsigned long long lo = chunk * bid < nf ? chunk * bid : nf;
    const unsigned long long hi = lo + chunk < nf ? lo + chunk : nf;
    const unsigned long long wch = (hi - lo + kW - 1) / kW;
    const unsigned long long wlo = lo + wch * wp < hi ? lo + wch * wp : hi;
    const unsigned long long whi = wlo + wch < hi ? wlo + wch : hi;
    uint32_t cnt[3] = {0, 0, 0};
    for (unsigned long long base = wlo; base < whi; base += 32) {
      const unsigned long long t = base + lane;
      const bool valid = t < whi;
      const Item it = mac_item<kNet>(cur, (int64_t)t, valid, cell, kids, m, sw, xs[wp], dec[wp]);
      if (valid) {
        cls[t] = it.cls;
        cnt[0] += it.nm;
        cnt[1] += it.np;
        cnt[2] += it.nch;
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int o = 16; o; o >>= 1) cnt[k] += __shfl_xor_sync(0xffffffffu, cnt[k], o);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 3; ++k) ws[wp][k] = cnt[k];
    __syncthreads();
    if (tid < 3) {
      uint32_t t = 0;
      for (int q = 0; q < kW; ++q) t += ws[q][tid];
      btot[3 * bid + tid] = t;
    }
    __threadfence();
    grid.sync();
    if (tid < 3) {
      unsigned long long before = 0, all = 0;
      for (unsigned q = 0; q < nb; ++q) {
        const unsigned long long v = btot[3 * q + tid];
        if (q < bid) before += v;
        all += v;
      }
      pre[tid] = before;
      sums[tid] = all;
    }
    __syncthreads();
    const unsigned long long Tm = sums[0], Tp = sums[1], Tc = sums[2];
    if (nm + Tm > capM || np + Tp > capP || Tc > capF) {
      if (bid == 0 && tid == 0) st->overflow = 1;
      break;  // every block takes the same decision
    }
    // this warp's offsets: the block's offsets plus the counts of the warps before it
    unsigned long long om = nm + pre[0], op = np + pre[1], oc = pre[2];
    for (int q = 0; q < wp; ++q) {
      om += ws[q][0];
      op += ws[q][1];
      oc += ws[q][2];
    }
    for (unsigned long long base = wlo; base < whi; base += 32) {
      const unsigned long long t = base + lane;
      const bool valid = t < whi;
      uint8_t cc = 0;
      uint64_t e = 0;
      int2 ka = make_int2(-1, 0), kb = make_int2(-1, 0);
      uint32_t v[3] = {0, 0, 0};
      if (valid) {
        cc = cls[t];
        e = cur[t];
        const uint8_t c = cc & 7;
        if (c == kM2L) v[0] = 1;
        if (c == kP2P) v[1] = 1;
        if (c == kOpenA || c == kOpenB || c == kOpenAB) {
          ka = kids[pair_sink(e)];
          kb = kids[pair_src(e)];
          v[2] = c == kOpenA ? ka.y : c == kOpenB ? kb.y : ka.y * kb.y;
        }
      }
      uint32_t x[3] = {v[0], v[1], v[2]};
#pragma unroll
      for (int o = 1; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x[k], o);
          if (lane >= o) x[k] += y;
        }
      if (valid) {
        const uint8_t c = cc & 7;
        if (c == kM2L) m2l[om + x[0] - v[0]] = with_order(e, (cc >> 3) & 15) | ((uint64_t)(cc >> 7) << kGenericBit);
        if (c == kP2P) p2p[op + x[1] - v[1]] = e;
        if (c == kOpenA || c == kOpenB || c == kOpenAB) {
          const uint32_t a = pair_sink(e), b = pair_src(e), s = pair_shift(e);
          uint32_t a0 = a, na = 1, b0 = b, nbb = 1;
          if (c == kOpenA || c == kOpenAB) {
            a0 = (uint32_t)ka.x;
            na = (uint32_t)ka.y;
          }
          if (c == kOpenB || c == kOpenAB) {
            b0 = (uint32_t)kb.x;
            nbb = (uint32_t)kb.y;
          }
          uint64_t *o = nxt + oc + x[2] - v[2];
          for (uint32_t xx = 0; xx < na; ++xx)
            for (uint32_t y = 0; y < nbb; ++y) *o++ = pack_pair(a0 + xx, b0 + y, s);
        }
      }
      om += __shfl_sync(0xffffffffu, x[0], 31);
      op += __shfl_sync(0xffffffffu, x[1], 31);
      oc += __shfl_sync(0xffffffffu, x[2], 31);
    }
    nm += Tm;
    np += Tp;
    nf = Tc;
    uint64_t *tmp = cur;
    cur = nxt;
    nxt = tmp;
    __threadfence();
    __syncthreads();  // ws is rewritten by the next level
    grid.sync();
  }
  if (bid == 0 && tid == 0) {
    st->nm2l = nm;
    st->np2p = np;
    st->nf = nf;
    st->iters = iter;
  }
}

// CSR bounds of the entries [lo, hi) of a list sorted by (sink, generic bit):
// beg[k] .. end[k]; with mid != null also mid[k], the first entry of sink k
// whose operator is evaluated per pair (end[k] when there is none).
__global__ void k_list_bounds(const uint64_t *__restrict__ lst, int64_t lo, int64_t hi, uint32_t *__restrict__ beg,
                              uint32_t *__restrict__ end, uint32_t *__restrict__ mid) {
  int64_t t = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= hi) return;
  const uint64_t e = lst[t];
  const uint32_t s = pair_sink(e);
  const bool first = t == lo || pair_sink(lst[t - 1]) != s;
  const bool last = t == hi - 1 || pair_sink(lst[t + 1]) != s;
  if (first) beg[s] = (uint32_t)t;
  if (last) end[s] = (uint32_t)(t + 1);
  if (mid) {
    const bool g = pair_generic(e);
    if (g && (first || !pair_generic(lst[t - 1]))) mid[s] = (uint32_t)t;
    if (!g && last) mid[s] = (uint32_t)(t + 1);
  }
}

// first[q] = index of the first entry with order >= q (q = 0..9) in a list sorted by (order, sink)
__global__ void k_order_bounds(const uint64_t *__restrict__ lst, int64_t n, uint64_t *__restrict__ first) {
  const int q = threadIdx.x;
  if (q > 9) return;
  int64_t a = 0, b = n;
  while (a < b) {
    const int64_t mid = a + (b - a) / 2;
    if ((int)pair_order(lst[mid]) < q) a = mid + 1; else b = mid;
  }
  first[q] = (uint64_t)a;
}

__global__ void k_pairs_in_list(const uint64_t *__restrict__ lst, int64_t n, const uint2 *__restrict__ range,
                                unsigned long long *__restrict__ acc) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (t < n) {
    uint64_t e = lst[t];
    v = (unsigned long long)range[pair_sink(e)].y * range[pair_src(e)].y;
  }
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

__global__ void k_count_table(const uint64_t *__restrict__ lst, int64_t n, unsigned long long *__restrict__ acc) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = (t < n && !pair_generic(lst[t])) ? 1ull : 0ull;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

}  // namespace

cudaError_t traverse(Ctx &c, cudaStream_t st) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  c.nm2l = c.np2p = 0;
  c.traverse_iters = 0;
  if (c.n == 0) return cudaSuccess;
  Mac m{};
  m.rc2i = c.rc2i;
  for (int l = 0; l <= kDepth; ++l) m.acc_thr[l] = c.acc_thr[l];
  m.rule = c.prm.transition_rule;
  m.size_rule = c.prm.size_rule;
  m.mode = c.collect ? 2 : c.prm.mac_mode;
  m.order = c.p;
  m.tab_k = (c.prm.m2l_precision == 0 && c.prm.m2l_tables) ? c.tab_k : 0;
  m.w = static_cast<const __nv_bfloat16 *>(c.mlp_w.p);
  m.M = P<float>(c.M);
  m.range = P<uint2>(c.range);
  m.ldm = c.ldm;
  m.inv_rs_h = (float)(c.prm.box / (double)kHalfBox / c.rs);
  m.inv_rc_h = (float)(c.prm.box / (double)kHalfBox / c.rc);
  m.cand = P<uint64_t>(c.cand);
  m.ncand = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 7);
  m.cand_cap = c.cand_cap;
  m.sample_mod = c.sample_mod ? c.sample_mod : 1u;

  int dev = 0, nsm = 0, per_sm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const bool net = m.mode == 1;
  const void *kern = net ? (const void *)k_traverse<true> : (const void *)k_traverse<false>;
  TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, net ? k_traverse<true> : k_traverse<false>, kTT, 0));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned nb = (unsigned)(nsm * (per_sm < 4 ? per_sm : 4));
  TRY(ensure(c.counts, (size_t)nb * 3 * sizeof(uint32_t)));
  // capacities: the last call's sizes with head-room, at least a few per node
  auto grow = [](uint64_t want) { return want + want / 4 + 1024; };
  if (c.cap_front < (uint64_t)(4 * c.nnodes + 1024)) c.cap_front = 4 * c.nnodes + 1024;
  if (c.cap_m2l < (uint64_t)(8 * c.nnodes + 1024)) c.cap_m2l = 8 * c.nnodes + 1024;
  if (c.cap_p2p < (uint64_t)(16 * c.nleaves + 1024)) c.cap_p2p = 16 * c.nleaves + 1024;
  TravState *dst = reinterpret_cast<TravState *>(P<uint64_t>(c.d_small) + 8);
  for (int attempt = 0; attempt < 8; ++attempt) {
    TRY(ensure(c.front, c.cap_front * 8));
    TRY(ensure(c.front_next, c.cap_front * 8));
    TRY(ensure(c.cls, c.cap_front));
    TRY(ensure(c.m2l, c.cap_m2l * 8));
    TRY(ensure(c.p2p, c.cap_p2p * 8));
    TRY(cudaMemsetAsync(dst, 0, sizeof(TravState), st));
    uint64_t *fa = P<uint64_t>(c.front), *fb = P<uint64_t>(c.front_next);
    uint8_t *cl = P<uint8_t>(c.cls);
    uint64_t *ml = P<uint64_t>(c.m2l), *pl = P<uint64_t>(c.p2p);
    unsigned long long capF = c.cap_front, capM = c.cap_m2l, capP = c.cap_p2p;
    uint32_t *bt = P<uint32_t>(c.counts);
    int max_iters = 2 * kDepth + 6;
    void *args[] = {(void *)&c.cell.p, (void *)&c.kids.p, (void *)&m, (void *)&fa, (void *)&fb, (void *)&capF,
                    (void *)&cl, (void *)&ml, (void *)&capM, (void *)&pl, (void *)&capP, (void *)&bt,
                    (void *)&dst, (void *)&max_iters};
    TRY(cudaLaunchCooperativeKernel(kern, dim3(nb), dim3(kTT), args, 0, st));
    note_launch();
    TravState hs;
    TRY(cudaMemcpyAsync(c.h_pinned, dst, sizeof(TravState), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    std::memcpy(&hs, c.h_pinned, sizeof(TravState));
    if (!hs.overflow) {
      if (hs.nf != 0) return cudaErrorInvalidValue;  // more levels than any octree can have
      c.nm2l = (int64_t)hs.nm2l;
      c.np2p = (int64_t)hs.np2p;
      c.traverse_iters = hs.iters;
      return cudaSuccess;
    }
    // grow every list (the walk stopped at the first overflow, so the sizes seen are lower bounds)
    c.cap_front = grow(c.cap_front * 2);
    c.cap_m2l = grow(c.cap_m2l * 2);
    c.cap_p2p = grow(c.cap_p2p * 2);
  }
  return cudaErrorInvalidValue;
#undef TRY
}

// Group both lists by sink (stable, so the traversal order is kept within a
// sink) and build CSR bounds; count the particle pairs P2P evaluates.
cudaError_t sort_lists(Ctx &c, cudaStream_t st) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  const int T = 256;
  int64_t nn = c.nnodes > 0 ? c.nnodes : 1;
  TRY(ensure(c.m2l_beg, nn * 4));
  TRY(ensure(c.m2l_end, nn * 4));
  TRY(ensure(c.p2p_beg, nn * 4));
  TRY(ensure(c.p2p_end, nn * 4));
  TRY(ensure(c.m2l_mid, nn * 4));
  TRY(cudaMemsetAsync(c.m2l_mid.p, 0, nn * 4, st));
  TRY(cudaMemsetAsync(c.m2l_beg.p, 0, nn * 4, st));
  TRY(cudaMemsetAsync(c.m2l_end.p, 0, nn * 4, st));
  TRY(cudaMemsetAsync(c.p2p_beg.p, 0, nn * 4, st));
  TRY(cudaMemsetAsync(c.p2p_end.p, 0, nn * 4, st));
  int sink_bits = 1;
  while (((int64_t)1 << sink_bits) < nn) ++sink_bits;
  for (int which = 0; which < 2; ++which) {
    DBuf &L = which ? c.p2p : c.m2l;
    DBuf &A = which ? c.p2p_alt : c.m2l_alt;
    int64_t n = which ? c.np2p : c.nm2l;
    if (n == 0) continue;
    TRY(ensure(A, n * 8));
    bool alt = false;
    // learned M2L entries carry their order in the top bits: group by (order, sink);
    // M2L entries are also ordered by the generic bit (table pairs first in each sink)
    const int hi_bit = (!which && c.prm.mac_mode == 1) ? 64 : kSinkShift + sink_bits;
    const int lo_bit = which ? kSinkShift : kGenericBit;
    TRY(radix_sort_u64(P<uint64_t>(L), nullptr, P<uint64_t>(A), nullptr, n, lo_bit, hi_bit, &alt, c.tmp, st));
    if (alt) std::swap(L, A);
    if (which || c.prm.mac_mode != 1) {
      k_list_bounds<<<blocks_for(n, T), T, 0, st>>>(P<uint64_t>(L), 0, n, P<uint32_t>(which ? c.p2p_beg : c.m2l_beg),
                                                    P<uint32_t>(which ? c.p2p_end : c.m2l_end),
                                                    which ? nullptr : P<uint32_t>(c.m2l_mid));
      note_launch();
      TRY(cudaGetLastError());
    }
  }
  c.p2p_particle_pairs = -1;
  c.nm2l_table = -1;
  if (c.prm.profile & 2) {
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c.d_small.p);
    TRY(cudaMemsetAsync(cnt, 0, 16, st));
    if (c.np2p > 0) {
      k_pairs_in_list<<<blocks_for(c.np2p, T), T, 0, st>>>(P<uint64_t>(c.p2p), c.np2p, P<uint2>(c.range), cnt);
      note_launch();
    }
    if (c.nm2l > 0) {
      k_count_table<<<blocks_for(c.nm2l, T), T, 0, st>>>(P<uint64_t>(c.m2l), c.nm2l, cnt + 1);
      note_launch();
    }
    TRY(cudaGetLastError());
    TRY(cudaMemcpyAsync(c.h_pinned, c.d_small.p, 16, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    c.p2p_particle_pairs = (int64_t)c.h_pinned[0];
    c.nm2l_table = (int64_t)c.h_pinned[1];
  }
  return cudaSuccess;
#undef TRY
}

cudaError_t m2l_all(Ctx &c, cudaStream_t st) {
  if (c.nm2l == 0) return cudaSuccess;
  const bool tab = c.prm.m2l_precision == 0 && c.prm.m2l_tables && c.tab_k > 0;
  if (tab && !c.tab_ready) {
    cudaError_t e = m2l_table_build(c, st);
    if (e != cudaSuccess) return e;
  }
  auto run = [&](int q) -> cudaError_t {
    if (c.prm.m2l_precision == 1 && m2l_tc_supported(q)) return m2l_pass_tc(c, q, st);
    if (tab) {
      cudaError_t e = m2l_pass_table(c, q, st);
      if (e != cudaSuccess) return e;
    }
    return m2l_pass(c, q, st);
  };
  if (c.prm.mac_mode != 1) return run(c.p);
  cudaError_t e;
  const int T = 256;
  const int64_t nn = c.nnodes;
  uint64_t *first = P<uint64_t>(c.d_small) + 16;
  k_order_bounds<<<1, 32, 0, st>>>(P<uint64_t>(c.m2l), c.nm2l, first);
  note_launch();
  if ((e = cudaMemcpyAsync(c.h_pinned, first, 10 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  uint64_t fb[10];
  for (int q = 0; q < 10; ++q) fb[q] = c.h_pinned[q];
  for (int q = 1; q <= c.p && q <= 8; ++q) {
    const int64_t lo = (int64_t)fb[q], hi = (int64_t)fb[q + 1];
    if (hi <= lo) continue;
    if ((e = cudaMemsetAsync(c.m2l_beg.p, 0, nn * 4, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c.m2l_end.p, 0, nn * 4, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c.m2l_mid.p, 0, nn * 4, st)) != cudaSuccess) return e;
    k_list_bounds<<<blocks_for(hi - lo, T), T, 0, st>>>(P<uint64_t>(c.m2l), lo, hi, P<uint32_t>(c.m2l_beg),
                                                        P<uint32_t>(c.m2l_end), P<uint32_t>(c.m2l_mid));
    note_launch();
    if ((e = run(q)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace hfmm
