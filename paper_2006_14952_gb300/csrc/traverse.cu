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
// The conventional walk (interaction counts of Sec. 3) applies rule 2 alone,
// with no cut-off skip and no transition region, from the single root pair of
// the primary box (shift index 13) instead of the 27 nearest periodic images.
//
// Learned acceptance (mac_mode 1) keeps rules 1 and 3 and the self-pair rule;
// in place of rule 2 a pair whose larger side satisfies L / S_c <= theta (the
// safety bound) is a candidate: its 12 features go through the network
// (mlp.cuh, tensor-core inference, batches of 16 candidates per warp) and the
// class chooses between opening the pair and M2L at an order q = 2..p.
// Collection mode records a hash-sampled subset of candidates while opening
// every pair (training data for the network).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
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
  int conv;   // 1: conventional acceptance (rule 2 alone, primary box only)
  int order;  // p (geometric M2L order, and the largest learned order)
  int tab_k;  // operator-table half extent (0: no table)
  int mutual; // 1: keep a P2P pair only as (A, B, s) with A < B, or A = B and s <= 13
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
  if (!m.conv && sm2 > m.rc2i) return kSkip;
  const bool trans = !m.conv && (m.rule == 0 ? sc2 > m.rc2i : sx2 > m.rc2i);
  const uint32_t lv = m.size_rule == 0 ? cb.w : (ca.w < cb.w ? ca.w : cb.w);  // level of the cell setting L
  if (!trans && sc2 >= m.acc_thr[lv]) return m.mode == 0 ? kM2L : kCandidate;  // acc_thr >= 1: self pairs open
  return open_rule(ca, cb, ka, kb);
}

// One frontier pair: its class (bits 0..2) and M2L order (bits 3..6), and the
// number of M2L entries, P2P entries and child pairs it produces.  Called by
// all 32 lanes of a warp (the network runs on warp batches of candidates).
struct Item {
  uint8_t cls;
  uint32_t nm, np, nchB;  // M2L entry, P2P entry, children of the source cell
  uint32_t sink;
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
__device__ __forceinline__ Item mac_item(uint64_t e, bool valid, const uint4 *__restrict__ cell,
                                         const int2 *__restrict__ kids, const Mac &m, const uint32_t *sw,
                                         __nv_bfloat16 *xs, uint8_t *dec) {
  const int lane = threadIdx.x & 31;
  uint32_t a = 0, b = 0, s = 0;
  int2 ka = make_int2(-1, 0), kb = make_int2(-1, 0);
  uint4 ca = make_uint4(0, 0, 0, 0), cb = ca;
  uint8_t c = kSkip;
  uint32_t order = (uint32_t)m.order;
  if (valid) {
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
  // mutual P2P: of the mirror pairs (a, b, s) and (b, a, 26 - s) the walk meets
  // both (it is symmetric under size_rule 1); keep one
  if (m.mutual && c == kP2P && !p2p_owner(a, b, s, ca.w, cb.w)) c = kSkip;
  Item it;
  const uint32_t miss = (c == kM2L && table_miss(ca, cb, s, m.tab_k)) ? 1u : 0u;
  it.cls = (uint8_t)(c | (order << 3) | (miss << 7));
  it.nm = c == kM2L;
  it.np = c == kP2P;
  it.nchB = kb.y > 0 ? (uint32_t)kb.y : 0u;
  it.sink = a;
  return it;
}

struct TravState {
  unsigned long long nm2l, np2p, nf, nseg;  // nf, nseg: the frontier left when the walk stopped
  int iters, overflow;
  int ovf_lists;                      // capacity overflow: bit 0 M2L, 1 P2P, 2 frontier, 3 segments, 4 runs
  unsigned long long need[5];         // entries those lists needed up to the level that overflowed
  unsigned long long items;           // frontier pairs classified over all levels
  unsigned long long nrun_m, nrun_p;  // M2L / P2P runs recorded
};

// Per-segment bases of one level: first output item (next frontier), the
// item prefix of the children-per-sink-child counts at the segment start, the
// first next-level segment, and the segment's children-per-sink-child total.
struct SegBase {
  unsigned long long o, c;
  uint32_t s, C;
};

// Frontier and output buffers of the walk (device pointers and capacities).
struct TravBufs {
  uint64_t *fa, *fb;                    // frontier pairs (ping-pong)
  uint32_t *map_a, *map_b;              // segment of each sink cell at this level (a sink has one)
  uint8_t *cls;                         // class of each frontier pair
  uint32_t *seg_a, *seg_b;              // sink of each segment (ping-pong)
  unsigned long long *st_a, *st_b;      // first frontier pair of each segment (ping-pong)
  unsigned long long *spre;             // per segment: pair prefixes (C, M, P) at its start
  SegBase *base;                        // bases of the current level's segments
  uint8_t *cc;                          // child pairs per child of the sink, per frontier pair
  unsigned long long *ctot;             // per 32-pair chunk: totals (C, M, P), then exclusive prefixes
  uint64_t *m2l, *p2p;                  // outputs
  uint64_t *rm_key, *rp_key;            // runs: (sink << 8 | level)
  uint64_t *rm_beg, *rp_beg;            // runs: first output entry
  uint32_t *rm_cnt, *rp_cnt;            // runs: entries
  uint32_t *rm_rank, *rp_rank;          // runs: rank among the runs of its sink (its level order)
  uint32_t *rcnt_m, *rcnt_p;            // per sink: runs recorded so far (one per level at most)
  unsigned long long *btot;             // per-block partial sums (4 per block)
  unsigned long long capF, capS, capM, capP, capR;
  const TreeState *tz;                  // graph mode: the device tree state (else null)
  // resume (sink batches): the walk starts from the frontier already in fa, seg_a,
  // st_a and map_a (init_nf pairs in init_nseg segments) instead of the root,
  // with level index iter0 for its first iteration
  int resume, iter0;
  unsigned long long init_nf, init_nseg;
};

constexpr int kTT = 256;  // threads of the traversal kernel
// a chunk with at most this many open pairs writes their child pairs warp-flattened
#ifndef HFMM_FLATTEN
#define HFMM_FLATTEN 16
#endif
constexpr int kFlatten = HFMM_FLATTEN;
constexpr int kTW = kTT / 32;

// Block-wide exclusive scans of N values per thread in one round (two block
// barriers for all N); tot receives the N block totals.
template <int N>
__device__ __forceinline__ void block_exscan_n(const unsigned long long (&v)[N], unsigned long long (&ex)[N],
                                               unsigned long long (&tot)[N], unsigned long long (*wsum)[kTW]) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  unsigned long long x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = v[i];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x[i], o);
      if (lane >= o) x[i] += y;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int i = 0; i < N; ++i) wsum[i][wp] = x[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) {
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int q = 0; q < kTW; ++q) {
      const unsigned long long w = wsum[i][q];
      if (q < wp) before += w;
      all += w;
    }
    ex[i] = before + x[i] - v[i];
    tot[i] = all;
  }
  __syncthreads();
}

// Prefix over the blocks before this one of column k of the per-block partials
// (ncol <= 4 columns), and the column totals.  The rows are read by all threads
// (strided), then reduced over the warps and the block.
__device__ __forceinline__ void block_prefixes(const unsigned long long *btot, int ncol, unsigned long long *pre,
                                               unsigned long long *all) {
  __shared__ unsigned long long red[kTW][8];
  const unsigned nb = gridDim.x, bid = blockIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  unsigned long long b[4] = {0, 0, 0, 0}, a[4] = {0, 0, 0, 0};
  for (unsigned q = threadIdx.x; q < nb; q += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < ncol) {
        const unsigned long long v = btot[4 * q + c];
        a[c] += v;
        if (q < bid) b[c] += v;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      b[c] += __shfl_xor_sync(0xffffffffu, b[c], o);
      a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      red[wp][c] = b[c];
      red[wp][4 + c] = a[c];
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < 2 * ncol) {
    const int j = threadIdx.x < (unsigned)ncol ? (int)threadIdx.x : 4 + (int)threadIdx.x - ncol;
    unsigned long long v = 0;
#pragma unroll
    for (int w = 0; w < kTW; ++w) v += red[w][j];
    if ((int)threadIdx.x < ncol) pre[threadIdx.x] = v;
    else all[threadIdx.x - ncol] = v;
  }
  __syncthreads();
}

// Persistent level-synchronous traversal, sink-major: one cooperative launch
// processes every level.  The frontier is kept in segments, one per sink cell,
// each holding that sink's pairs contiguously.  Per level:
//   1. every warp classifies interleaved 32-pair chunks (the acceptance rules
//      of Sec. 2.3; interleaving spreads dense regions over all warps) and
//      records per chunk the number of child pairs given to each child of the
//      sink (C), of M2L entries (M) and of P2P entries (P);
//   2. a scan over the chunks gives every chunk its exclusive prefixes; the
//      prefixes at the segment starts give each segment its totals; a scan
//      over the segments gives each its next-frontier base, writes the next
//      level's segments (one per child of an opened sink, or the sink itself
//      when it is a leaf whose partners open) and records the runs of M2L and
//      P2P entries each sink received at this level;
//   3. every warp emits its chunks again: M2L / P2P entries in pair order (so
//      grouped by sink within the level), child pairs at
//      base + child * C + (prefix within the segment), so that every child's
//      pairs are contiguous in the next frontier.
// A non-leaf sink only ever opens itself (open A or both): the larger cell is
// opened, and a pair with a larger source arises only when the sink is a leaf.
// Outputs beyond the given capacities set st->overflow and stop the walk; the
// host grows the buffers and runs it again.
template <bool kNet>
__global__ void __launch_bounds__(kTT, 4) k_traverse(const uint4 *__restrict__ cell,
                                                                const int2 *__restrict__ kids, Mac m, TravBufs B,
                                                                TravState *__restrict__ st, int max_iters) {
  cg::grid_group grid = cg::this_grid();
  constexpr int kSw = kNet ? kMlpSmemWords : 1, kXs = kNet ? 32 * 16 : 1, kDec = kNet ? 32 : 1;
  __shared__ uint32_t sw[kSw];
  __shared__ __align__(16) __nv_bfloat16 xs[kTW][kXs];
  __shared__ uint8_t dec[kTW][kDec];
  __shared__ unsigned long long pre[4], all[4], run[4];
  __shared__ unsigned long long wsum4[4][kTW];
  // level state, uniform over the grid (kept in shared memory, out of the registers)
  __shared__ uint64_t *cur, *nxt;
  __shared__ uint32_t *cmap, *nmap, *segs, *nsegs;
  __shared__ unsigned long long *sst, *nsst;
  __shared__ unsigned long long nf, nseg, nm, np, nrm, nrp, items;
  if (B.tz && B.tz->overflow) {  // graph mode, the tree did not fit: no walk (every block leaves here)
    if (blockIdx.x == 0 && threadIdx.x == 0) st->overflow = 3;
    return;
  }
  if (kNet) mlp_stage(m.w, sw);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  const unsigned nb = gridDim.x, bid = blockIdx.x;
  const unsigned long long gw = (unsigned long long)bid * kTW + wp, nw = (unsigned long long)nb * kTW;
  // the root against its 27 nearest periodic images, or (conventional) itself
  const unsigned nroot = m.conv ? 1u : 27u;
  if (!B.resume) {
    if (bid == 0 && tid < nroot) B.fa[tid] = pack_pair(0, 0, m.conv ? 13u : (uint32_t)tid);
    if (bid == 0 && tid == 0) {
      B.map_a[0] = 0;
      B.seg_a[0] = 0;
      B.st_a[0] = 0;
    }
  }
  if (tid == 0) {
    cur = B.fa;
    nxt = B.fb;
    cmap = B.map_a;
    nmap = B.map_b;
    segs = B.seg_a;
    nsegs = B.seg_b;
    sst = B.st_a;
    nsst = B.st_b;
    nf = B.resume ? B.init_nf : nroot;
    nseg = B.resume ? B.init_nseg : 1;
    nm = np = nrm = nrp = items = 0;
  }
  __syncthreads();
  grid.sync();
  int iter = 0;
  for (; iter < max_iters && nf > 0; ++iter) {
    const unsigned long long NF = nf, K = (NF + 31) / 32;  // 32-pair chunks
    // ---- 1. classify interleaved chunks; chunk totals (C, M, P).  The frontier
    //         pair of the warp's next chunk is fetched while this one is classified.
    uint64_t e_pf = 0;
    if (gw < K && 32 * gw + lane < NF) e_pf = cur[32 * gw + lane];
    for (unsigned long long k = gw; k < K; k += nw) {
      const unsigned long long t = 32 * k + lane;
      const bool valid = t < NF;
      const uint64_t e_now = e_pf;
      if (k + nw < K && t + 32 * nw < NF) e_pf = cur[t + 32 * nw];
      const Item it = mac_item<kNet>(e_now, valid, cell, kids, m, sw, xs[wp], dec[wp]);
      uint32_t v[3] = {0, 0, 0};
      if (valid) {
        const uint8_t c = it.cls & 7;
        v[0] = c == kOpenA ? 1u : (c == kOpenAB || c == kOpenB) ? it.nchB : 0u;
        v[1] = it.nm;
        v[2] = it.np;
        B.cls[t] = it.cls;
        B.cc[t] = (uint8_t)v[0];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) v[q] = __reduce_add_sync(0xffffffffu, v[q]);
      if (lane < 3) B.ctot[3 * k + lane] = v[lane];
    }
    __threadfence();
    grid.sync();
    // ---- 2a. chunk scan: block partials over contiguous chunk ranges
    const unsigned long long kch = (K + nb - 1) / nb;
    const unsigned long long klo = kch * bid < K ? kch * bid : K, khi = klo + kch < K ? klo + kch : K;
    // each thread takes a contiguous run of the block's chunks (also in 2b)
    const unsigned long long kper = (khi - klo + kTT - 1) / kTT;
    const unsigned long long tlo = klo + kper * tid < khi ? klo + kper * tid : khi;
    const unsigned long long thi = tlo + kper < khi ? tlo + kper : khi;
    {
      unsigned long long loc[3] = {0, 0, 0}, ex[3], tot[3];
      for (unsigned long long k = tlo; k < thi; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) loc[q] += B.ctot[3 * k + q];
      block_exscan_n<3>(loc, ex, tot, wsum4);
      if (tid < 3) B.btot[4 * bid + tid] = tot[tid];
    }
    __threadfence();
    grid.sync();
    // ---- 2b. chunk scan: exclusive prefixes in place
    block_prefixes(B.btot, 3, pre, all);
    const unsigned long long Tc = all[0], Tm = all[1], Tp = all[2];
    {
      unsigned long long loc[3] = {0, 0, 0}, ex[3], tot[3];
      for (unsigned long long k = tlo; k < thi; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) loc[q] += B.ctot[3 * k + q];
      block_exscan_n<3>(loc, ex, tot, wsum4);
      unsigned long long rq[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) rq[q] = pre[q] + ex[q];
      for (unsigned long long k = tlo; k < thi; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const unsigned long long v = B.ctot[3 * k + q];
          B.ctot[3 * k + q] = rq[q];
          rq[q] += v;
        }
    }
    __threadfence();
    grid.sync();
    // ---- 2c. segment prefixes at their starts, totals by differences; block partials of
    //          (next items, next segments, M2L runs, P2P runs)
    const unsigned long long NS = nseg;
    const unsigned long long sch = (NS + nb - 1) / nb;
    const unsigned long long slo = sch * bid < NS ? sch * bid : NS, shi = slo + sch < NS ? slo + sch : NS;
    // prefix (C, M, P) of the pairs before frontier position t
    auto prefix_at = [&](unsigned long long t, unsigned long long (&pv)[3]) {
      if (t >= NF) {
        pv[0] = Tc;
        pv[1] = Tm;
        pv[2] = Tp;
        return;
      }
      const unsigned long long k = t / 32;
#pragma unroll
      for (int q = 0; q < 3; ++q) pv[q] = B.ctot[3 * k + q];
      for (unsigned long long j = 32 * k; j < t; ++j) {
        const uint8_t c = B.cls[j] & 7;
        pv[0] += B.cc[j];
        pv[1] += c == kM2L;
        pv[2] += c == kP2P;
      }
    };
    auto seg_prefix = [&](unsigned long long s, unsigned long long (&pv)[3]) { prefix_at(s < NS ? sst[s] : NF, pv); };
    {
      unsigned long long loc[4] = {0, 0, 0, 0};
      for (unsigned long long s = slo + tid; s < shi; s += kTT) {
        unsigned long long pv[3], pn[3];
        seg_prefix(s, pv);
        seg_prefix(s + 1, pn);
        const int2 kk = kids[segs[s]];
        const unsigned long long mult = kk.y > 0 ? (unsigned long long)kk.y : 1ull, C = pn[0] - pv[0];
        loc[0] += mult * C;
        loc[1] += C > 0 ? mult : 0;
        loc[2] += pn[1] > pv[1];
        loc[3] += pn[2] > pv[2];
#pragma unroll
        for (int q = 0; q < 3; ++q) B.spre[3 * s + q] = pv[q];
      }
      unsigned long long ex[4], tot[4];
      block_exscan_n<4>(loc, ex, tot, wsum4);
      if (tid < 4) B.btot[4 * bid + tid] = tot[tid];
    }
    __threadfence();
    grid.sync();
    // ---- 2d. segment scan: bases, next-level segments, runs
    block_prefixes(B.btot, 4, pre, all);
    const unsigned long long To = all[0], Ts = all[1], Trm = all[2], Trp = all[3];
    if (nm + Tm > B.capM || np + Tp > B.capP || To > B.capF || Ts > B.capS || nrm + Trm > B.capR ||
        nrp + Trp > B.capR) {
      if (bid == 0 && tid == 0) {
        st->overflow = 1;
        st->ovf_lists = (nm + Tm > B.capM ? 1 : 0) | (np + Tp > B.capP ? 2 : 0) | (To > B.capF ? 4 : 0) |
                        (Ts > B.capS ? 8 : 0) | (nrm + Trm > B.capR || nrp + Trp > B.capR ? 16 : 0);
        st->need[0] = nm + Tm;
        st->need[1] = np + Tp;
        st->need[2] = To;
        st->need[3] = Ts;
        st->need[4] = nrm + Trm > nrp + Trp ? nrm + Trm : nrp + Trp;
      }
      break;  // every block takes the same decision
    }
    if (tid < 4) run[tid] = pre[tid];
    __syncthreads();
    for (unsigned long long sb0 = slo; sb0 < shi; sb0 += kTT) {
      const unsigned long long s = sb0 + tid;
      const bool valid = s < shi;
      unsigned long long tv[3] = {0, 0, 0}, pv[3] = {0, 0, 0};
      uint32_t sink = 0;
      int2 kk = make_int2(-1, 0);
      if (valid) {
#pragma unroll
        for (int q = 0; q < 3; ++q) pv[q] = B.spre[3 * s + q];
        if (s + 1 < NS) {
#pragma unroll
          for (int q = 0; q < 3; ++q) tv[q] = B.spre[3 * (s + 1) + q] - pv[q];
        } else {
          tv[0] = Tc - pv[0];
          tv[1] = Tm - pv[1];
          tv[2] = Tp - pv[2];
        }
        sink = segs[s];
        kk = kids[sink];
      }
      const unsigned long long mult = kk.y > 0 ? (unsigned long long)kk.y : 1ull;
      unsigned long long ex[4], tot[4];
      const unsigned long long sv[4] = {valid ? mult * tv[0] : 0ull, valid && tv[0] > 0 ? mult : 0ull,
                                        valid && tv[1] > 0 ? 1ull : 0ull, valid && tv[2] > 0 ? 1ull : 0ull};
      block_exscan_n<4>(sv, ex, tot, wsum4);
      if (valid) {
        const unsigned long long o = run[0] + ex[0], sn = run[1] + ex[1];
        SegBase sbv;
        sbv.o = o;
        sbv.s = (uint32_t)sn;
        sbv.c = pv[0];
        sbv.C = (uint32_t)tv[0];
        B.base[s] = sbv;
        if (tv[0] > 0) {  // next-level segments: the sink itself (leaf) or each of its children
          if (kk.y > 0) {
            for (int i = 0; i < kk.y; ++i) {
              nsegs[sn + i] = (uint32_t)kk.x + (uint32_t)i;
              nmap[(uint32_t)kk.x + (uint32_t)i] = (uint32_t)(sn + i);
              nsst[sn + i] = o + (unsigned long long)i * tv[0];
            }
          } else {
            nsegs[sn] = sink;
            nmap[sink] = (uint32_t)sn;
            nsst[sn] = o;
          }
        }
        if (tv[1] > 0) {
          const unsigned long long r = nrm + run[2] + ex[2];
          B.rm_key[r] = ((unsigned long long)sink << 8) | (unsigned)(B.iter0 + iter);
          B.rm_beg[r] = nm + pv[1];
          B.rm_cnt[r] = (uint32_t)tv[1];
          B.rm_rank[r] = B.rcnt_m[sink]++;  // a sink has one segment per level: no other writer
        }
        if (tv[2] > 0) {
          const unsigned long long r = nrp + run[3] + ex[3];
          B.rp_key[r] = ((unsigned long long)sink << 8) | (unsigned)(B.iter0 + iter);
          B.rp_beg[r] = np + pv[2];
          B.rp_cnt[r] = (uint32_t)tv[2];
          B.rp_rank[r] = B.rcnt_p[sink]++;
        }
      }
      __syncthreads();
      if (tid < 4) run[tid] += tot[tid];
      __syncthreads();
    }
    __threadfence();
    grid.sync();
    // ---- 3. emit interleaved chunks (the next chunk's pair and class fetched ahead)
    uint64_t e_nx = 0;
    uint8_t c_nx = 0;
    if (gw < K && 32 * gw + lane < NF) {
      e_nx = cur[32 * gw + lane];
      c_nx = B.cls[32 * gw + lane];
    }
    for (unsigned long long k = gw; k < K; k += nw) {
      const unsigned long long t = 32 * k + lane;
      const bool valid = t < NF;
      uint8_t cc = 0;
      uint64_t e = 0;
      int2 ka = make_int2(-1, 0), kb = make_int2(-1, 0);
      uint32_t v[3] = {0, 0, 0};
      const uint64_t e_in = e_nx;
      const uint8_t c_in = c_nx;
      if (k + nw < K && t + 32 * nw < NF) {
        e_nx = cur[t + 32 * nw];
        c_nx = B.cls[t + 32 * nw];
      }
      if (valid) {
        cc = c_in;
        e = e_in;
        const uint8_t c = cc & 7;
        if (c == kM2L) v[1] = 1;
        if (c == kP2P) v[2] = 1;
        if (c == kOpenA || c == kOpenB || c == kOpenAB) {
          ka = kids[pair_sink(e)];
          kb = kids[pair_src(e)];
          v[0] = c == kOpenA ? 1u : (uint32_t)kb.y;
        }
      }
      uint32_t x[3] = {v[0], v[1], v[2]};
#pragma unroll
      for (int o = 1; o < 32; o <<= 1)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x[q], o);
          if (lane >= o) x[q] += y;
        }
      if (valid) {
        const uint8_t c = cc & 7;
        if (c == kM2L)
          B.m2l[nm + B.ctot[3 * k + 1] + x[1] - v[1]] = with_order(e, (cc >> 3) & 15) | ((uint64_t)(cc >> 7) << kGenericBit);
        if (c == kP2P) B.p2p[np + B.ctot[3 * k + 2] + x[2] - v[2]] = e;
      }
      // child pairs: each open pair's outputs, flattened over the warp so that every
      // lane writes (the open pairs are a few percent of the frontier)
      uint32_t nout = 0, nbk = 1, a0 = 0, b0 = 0, shv = 0, Cs = 0;
      unsigned long long p0 = 0;
      if (valid) {
        const uint8_t c = cc & 7;
        if (c == kOpenA || c == kOpenB || c == kOpenAB) {
          const uint32_t a = pair_sink(e), b = pair_src(e);
          shv = pair_shift(e);
          const SegBase sb = B.base[cmap[a]];
          p0 = sb.o + (B.ctot[3 * k] + x[0] - v[0] - sb.c);
          Cs = sb.C;
          // the last slot this item writes; beyond the next frontier means inconsistent bases
          const unsigned long long last =
              c == kOpenB ? p0 + kb.y : p0 + (unsigned long long)(ka.y - 1) * sb.C + (c == kOpenA ? 1 : kb.y);
          const bool bad = (c == kOpenB && ka.y > 0) || last > To;  // cannot happen (see above)
          if (bad) {
            st->overflow = 2;  // refuse rather than write out of place
          } else if (c == kOpenB) {  // the sink is a leaf: one next-level segment
            nout = (uint32_t)kb.y;
            nbk = (uint32_t)kb.y;
            a0 = a;
            b0 = (uint32_t)kb.x;
          } else {
            nbk = c == kOpenA ? 1u : (uint32_t)kb.y;
            nout = (uint32_t)ka.y * nbk;
            a0 = (uint32_t)ka.x;
            b0 = c == kOpenA ? b : (uint32_t)kb.x;
          }
        }
      }
      // 2^16 / nbk rounded up: r / nbk = (r * inv) >> 16 exactly for r < 64, nbk <= 8
      const uint32_t inv = (65536u + nbk - 1) / nbk;
      // many open pairs in the chunk: every lane has work, each writes its own outputs
      if (__popc(__ballot_sync(0xffffffffu, nout > 0)) > kFlatten) {
        for (uint32_t r = 0; r < nout; ++r) {
          const uint32_t i = (r * inv) >> 16, q = r - i * nbk;
          nxt[p0 + (unsigned long long)i * Cs + q] = pack_pair(a0 + i, b0 + q, shv);
        }
        continue;
      }
      // a few open pairs: flatten their outputs over the warp
      uint32_t oin = nout;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, oin, o);
        if (lane >= o) oin += y;
      }
      const uint32_t oex = oin - nout, ototal = __shfl_sync(0xffffffffu, oin, 31);
      for (uint32_t jb = 0; jb < ototal; jb += 32) {  // uniform trip count: every lane shuffles
        const uint32_t j = jb + lane;
        int src = 0;  // the last lane whose outputs start at or before j
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const uint32_t ex = __shfl_sync(0xffffffffu, oex, src + step);
          if (ex <= j) src += step;
        }
        const uint32_t r = j - __shfl_sync(0xffffffffu, oex, src);
        const uint32_t snbk = __shfl_sync(0xffffffffu, nbk, src), sinv = __shfl_sync(0xffffffffu, inv, src);
        const uint32_t sa0 = __shfl_sync(0xffffffffu, a0, src), sb0 = __shfl_sync(0xffffffffu, b0, src);
        const uint32_t ssh = __shfl_sync(0xffffffffu, shv, src), sC = __shfl_sync(0xffffffffu, Cs, src);
        const unsigned long long sp0 = __shfl_sync(0xffffffffu, p0, src);
        const uint32_t i = (r * sinv) >> 16, q = r - i * snbk;
        // open A: b0 fixed, q = 0; open B: i = 0 (one child block); open both: child i, source q
        if (j < ototal) nxt[sp0 + (unsigned long long)i * sC + q] = pack_pair(sa0 + i, sb0 + q, ssh);
      }
    }
    __syncthreads();  // every thread is done with this level's state
    if (tid == 0) {
      items += nf;
      nm += Tm;
      np += Tp;
      nrm += Trm;
      nrp += Trp;
      nf = To;
      nseg = Ts;
      uint64_t *t1 = cur;
      cur = nxt;
      nxt = t1;
      uint32_t *t2 = cmap;
      cmap = nmap;
      nmap = t2;
      uint32_t *t3 = segs;
      segs = nsegs;
      nsegs = t3;
      unsigned long long *t4 = sst;
      sst = nsst;
      nsst = t4;
    }
    __threadfence();
    grid.sync();
  }
  if (bid == 0 && tid == 0) {
    st->nm2l = nm;
    st->np2p = np;
    st->nf = nf;
    st->nseg = nseg;
    st->iters = iter;
    st->items = items;
    st->nrun_m = nrm;
    st->nrun_p = nrp;
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

namespace {

// The walk's parameters and grid, and the first guesses of its list capacities.
struct WalkPlan {
  Mac m;
  unsigned nb;
};

// First guess of the P2P list's entries per particle (the scale of the walk_plan guesses).
double p2p_guess_per_particle(const Ctx &c) {
  const double lf = c.prm.leaf_max > 16 ? std::pow(16.0 / c.prm.leaf_max, 1.5) * 1.5 : 1.0;
  return 128.0 * (lf < 1.0 ? lf : 1.0);
}

cudaError_t walk_plan(Ctx &c, WalkPlan &w) {
  cudaError_t e;
  Mac &m = w.m;
  m = Mac{};
  m.rc2i = c.rc2i;
  for (int l = 0; l <= kDepth; ++l) m.acc_thr[l] = c.acc_thr[l];
  m.rule = c.prm.transition_rule;
  m.size_rule = c.prm.size_rule;
  m.mode = c.collect ? 2 : c.count_walk ? 0 : c.prm.mac_mode;
  m.conv = c.count_walk == 2 ? 1 : 0;
  m.order = c.p;
  m.tab_k = ((c.prm.m2l_precision == 0 && c.prm.m2l_tables) || c.prm.m2l_precision >= 3) ? c.tab_k : 0;
  m.mutual = (c.prm.p2p_mutual && !c.collect && !c.count_walk) ? 1 : 0;
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
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const bool net = m.mode == 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, net ? k_traverse<true> : k_traverse<false>, kTT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int want = c.prm.tile_trav_blocks > 0 ? c.prm.tile_trav_blocks : 4;
  w.nb = (unsigned)(nsm * (per_sm < want ? per_sm : want));
  // capacities: the last call's sizes with head-room, at least a few per node.
  // First guesses from the 2M clustered set: at leaves of 16, about 60 frontier
  // pairs per particle at the largest level, 50 M2L and 115 P2P entries per
  // particle in total; these fall about as (16 / leaf_max)^1.5 (8 M2L and 21 P2P
  // per particle at 48), so the guesses are scaled so, with a margin of 1.5.
  // A list that overflows is grown alone (to what the walk needed so far, at least
  // twice its size) and the walk is repeated.  A positive list_init replaces every
  // first guess (a test knob for the retry path).
  const double lf = c.prm.leaf_max > 16 ? std::pow(16.0 / c.prm.leaf_max, 1.5) * 1.5 : 1.0;
  const double sc = (lf < 1.0 ? lf : 1.0) * c.walk_share;  // sink batches: one batch's share
  const uint64_t init = (uint64_t)c.prm.list_init;
  auto first_guess = [&](uint64_t guess) { return init > 0 ? init : guess; };
  const uint64_t g_front = first_guess((uint64_t)(sc * 64 * c.n + 1024));
  const uint64_t g_m2l = first_guess((uint64_t)(sc * 64 * c.n + 1024));
  const uint64_t g_p2p = first_guess((uint64_t)(sc * 128 * c.n + 1024));
  const uint64_t g_seg = first_guess((uint64_t)(2 * c.nnodes + 1024));
  const uint64_t g_run = first_guess((uint64_t)(4 * c.nnodes + 1024));
  if (c.cap_front < g_front) c.cap_front = g_front;
  if (c.cap_m2l < g_m2l) c.cap_m2l = g_m2l;
  if (c.cap_p2p < g_p2p) c.cap_p2p = g_p2p;
  if (c.cap_seg < g_seg) c.cap_seg = g_seg;
  if (c.cap_run < g_run) c.cap_run = g_run;
  return cudaSuccess;
}

cudaError_t walk_buffers(Ctx &c, unsigned nb) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  TRY(ensure(c.btot2, (size_t)nb * 4 * sizeof(unsigned long long)));
  TRY(ensure(c.front, c.cap_front * 8));
  TRY(ensure(c.front_next, c.cap_front * 8));
  TRY(ensure(c.fseg, c.nnodes * 4 + 64));
  TRY(ensure(c.fseg_next, c.nnodes * 4 + 64));
  TRY(ensure(c.cls, c.cap_front * 2));  // class and child count per frontier pair
  TRY(ensure(c.seg_a, c.cap_seg * 4));
  TRY(ensure(c.seg_b, c.cap_seg * 4));
  TRY(ensure(c.acc_a, c.cap_seg * 8));  // segment starts (ping-pong)
  TRY(ensure(c.acc_b, c.cap_seg * 8));
  TRY(ensure(c.segpre, c.cap_seg * 24));
  TRY(ensure(c.segbase, c.cap_seg * sizeof(SegBase)));
  TRY(ensure(c.ctot, ((c.cap_front + 31) / 32) * 24 + 64));
  TRY(ensure(c.m2l, c.cap_m2l * 8));
  TRY(ensure(c.p2p, c.cap_p2p * 8));
  TRY(ensure(c.rm_key, c.cap_run * 8));
  TRY(ensure(c.rm_beg, c.cap_run * 8));
  TRY(ensure(c.rm_cnt, c.cap_run * 4));
  TRY(ensure(c.rp_key, c.cap_run * 8));
  TRY(ensure(c.rp_beg, c.cap_run * 8));
  TRY(ensure(c.rp_cnt, c.cap_run * 4));
  TRY(ensure(c.rm_rank, c.cap_run * 4));
  TRY(ensure(c.rp_rank, c.cap_run * 4));
  TRY(ensure(c.rcnt_m, (size_t)c.nnodes * 4 + 64));
  TRY(ensure(c.rcnt_p, (size_t)c.nnodes * 4 + 64));
  return cudaSuccess;
#undef TRY
}

// the walk's state sits after the eight counters of the 256-byte d_small and is read back into h_pinned
TravState *walk_state(Ctx &c) {
  static_assert(8 * sizeof(uint64_t) + sizeof(TravState) <= 256, "TravState must fit in d_small");
  return reinterpret_cast<TravState *>(P<uint64_t>(c.d_small) + 8);
}

// Where a walk starts: the root (resume 0) or a frontier already in the
// walk's first buffers (sink batches), and how many levels it may take.
struct WalkStart {
  int resume = 0, iter0 = 0, max_iters = 2 * kDepth + 6;
  unsigned long long nf = 0, nseg = 0;
};

// Zero the counters and launch the cooperative walk (no allocation, no read-back).
cudaError_t walk_launch(Ctx &c, const WalkPlan &w, cudaStream_t st, const WalkStart &ws = WalkStart()) {
  cudaError_t e;
  TravState *dst = walk_state(c);
  if ((e = cudaMemsetAsync(c.rcnt_m.p, 0, (size_t)c.nnodes * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.rcnt_p.p, 0, (size_t)c.nnodes * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(dst, 0, sizeof(TravState), st)) != cudaSuccess) return e;
  TravBufs B;
  B.fa = P<uint64_t>(c.front);
  B.fb = P<uint64_t>(c.front_next);
  B.map_a = P<uint32_t>(c.fseg);
  B.map_b = P<uint32_t>(c.fseg_next);
  B.cls = P<uint8_t>(c.cls);
  B.cc = P<uint8_t>(c.cls) + c.cap_front;
  B.seg_a = P<uint32_t>(c.seg_a);
  B.seg_b = P<uint32_t>(c.seg_b);
  B.st_a = P<unsigned long long>(c.acc_a);
  B.st_b = P<unsigned long long>(c.acc_b);
  B.spre = P<unsigned long long>(c.segpre);
  B.base = P<SegBase>(c.segbase);
  B.ctot = P<unsigned long long>(c.ctot);
  B.m2l = P<uint64_t>(c.m2l);
  B.p2p = P<uint64_t>(c.p2p);
  B.rm_key = P<uint64_t>(c.rm_key);
  B.rp_key = P<uint64_t>(c.rp_key);
  B.rm_beg = P<uint64_t>(c.rm_beg);
  B.rp_beg = P<uint64_t>(c.rp_beg);
  B.rm_cnt = P<uint32_t>(c.rm_cnt);
  B.rp_cnt = P<uint32_t>(c.rp_cnt);
  B.rm_rank = P<uint32_t>(c.rm_rank);
  B.rp_rank = P<uint32_t>(c.rp_rank);
  B.rcnt_m = P<uint32_t>(c.rcnt_m);
  B.rcnt_p = P<uint32_t>(c.rcnt_p);
  B.btot = P<unsigned long long>(c.btot2);
  B.capF = c.cap_front;
  B.capS = c.cap_seg;
  B.capM = c.cap_m2l;
  B.capP = c.cap_p2p;
  B.capR = c.cap_run;
  B.tz = c.graph_tree ? P<TreeState>(c.tstate) : nullptr;
  B.resume = ws.resume;
  B.iter0 = ws.iter0;
  B.init_nf = ws.nf;
  B.init_nseg = ws.nseg;
  int max_iters = ws.max_iters;
  Mac m = w.m;
  const bool net = m.mode == 1;
  const void *kern = net ? (const void *)k_traverse<true> : (const void *)k_traverse<false>;
  void *args[] = {(void *)&c.cell.p, (void *)&c.kids.p, (void *)&m, (void *)&B, (void *)&dst, (void *)&max_iters};
  e = cudaLaunchCooperativeKernel(kern, dim3(w.nb), dim3(kTT), args, 0, st);
  note_launch();
  return e;
}

// Interpret the read-back state: 0 done, 1 a list overflowed (grow and repeat),
// -1 the walk cannot complete (more levels than any octree, or a bad opening).
int walk_result(Ctx &c, const TravState &hs) {
  if (hs.overflow == 2) return -1;  // a non-leaf sink was asked to open its partner
  if (hs.overflow) return 1;
  if (hs.nf != 0) return -1;  // more levels than any octree can have
  c.nm2l = (int64_t)hs.nm2l;
  c.np2p = (int64_t)hs.np2p;
  c.traverse_iters = hs.iters;
  c.frontier_items = (int64_t)hs.items;
  c.nrun_m = (int64_t)hs.nrun_m;
  c.nrun_p = (int64_t)hs.nrun_p;
  return 0;
}

}  // namespace

cudaError_t traverse(Ctx &c, cudaStream_t st) {
  cudaError_t e;
  c.nm2l = c.np2p = 0;
  c.traverse_iters = 0;
  if (c.n == 0) return cudaSuccess;
  WalkPlan w;
  if ((e = walk_plan(c, w)) != cudaSuccess) return e;
  c.traverse_walks = 0;
  for (int attempt = 0; attempt < 32; ++attempt) {
    ++c.traverse_walks;
    if ((e = walk_buffers(c, w.nb)) != cudaSuccess) return e;
    if ((e = walk_launch(c, w, st)) != cudaSuccess) return e;
    TravState hs;
    if ((e = cudaMemcpyAsync(c.h_pinned, walk_state(c), sizeof(TravState), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    std::memcpy(&hs, c.h_pinned, sizeof(TravState));
    const int r = walk_result(c, hs);
    if (r < 0) return cudaErrorInvalidValue;
    if (r == 0) return cudaSuccess;
    // grow the lists that overflowed (the walk stopped at the first overflow, so the
    // sizes seen are lower bounds)
    auto grow = [](uint64_t want) { return want + want / 4 + 1024; };
    auto up = [&](uint64_t &cap, int bit, int k) {
      if (hs.ovf_lists & bit) cap = grow(std::max<uint64_t>(cap * 2, hs.need[k]));
    };
    up(c.cap_m2l, 1, 0);
    up(c.cap_p2p, 2, 1);
    up(c.cap_front, 4, 2);
    up(c.cap_seg, 8, 3);
    up(c.cap_run, 16, 4);
  }
  return cudaErrorInvalidValue;
}

// Graph mode: the walk without its read-back.  _prepare sizes every buffer
// (outside the capture), _launch enqueues the walk (inside it), _finish reads
// the state back after the graph ran and reports whether the lists fit.
cudaError_t traverse_graph_prepare(Ctx &c) {
  WalkPlan w;
  cudaError_t e = walk_plan(c, w);
  if (e == cudaSuccess) e = walk_buffers(c, w.nb);
  return e;
}

cudaError_t traverse_graph_launch(Ctx &c, cudaStream_t st) {
  WalkPlan w;
  cudaError_t e = walk_plan(c, w);
  if (e == cudaSuccess) e = walk_launch(c, w, st);
  return e;
}

cudaError_t traverse_graph_finish(Ctx &c, cudaStream_t st, bool *ok) {
  cudaError_t e;
  TravState hs;
  if ((e = cudaMemcpyAsync(c.h_pinned, walk_state(c), sizeof(TravState), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  std::memcpy(&hs, c.h_pinned, sizeof(TravState));
  *ok = walk_result(c, hs) == 0;
  c.traverse_walks = 1;
  return cudaSuccess;
}

// Graph mode: every buffer the list grouping of sort_lists can touch, sized for
// the capacities, so that nothing is allocated during the capture.
cudaError_t sort_lists_prepare(Ctx &c) {
  cudaError_t e;
  const size_t nn = (size_t)(c.nnodes > 0 ? c.nnodes : 1);
  const size_t nr = (size_t)c.cap_run;
  if ((e = ensure(c.m2l_beg, nn * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.m2l_end, nn * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.m2l_mid, nn * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.p2p_beg, nn * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.p2p_end, nn * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.m2l_alt, c.cap_m2l * 8)) != cudaSuccess) return e;
  if ((e = ensure(c.p2p_alt, c.cap_p2p * 8)) != cudaSuccess) return e;
  if ((e = ensure(c.tmp2, nr * 20 + nn * 4 + 64)) != cudaSuccess) return e;
  const size_t most = nr > nn ? nr : nn;
  return ensure(c.offs, ((most + 4095) / 1024 + 1) * sizeof(uint64_t));  // scan block sums, with room
}

StepGuard step_guard(Ctx &c) {
  StepGuard g;
  g.tree_overflow = &P<TreeState>(c.tstate)->overflow;
  g.walk_overflow = &walk_state(c)->overflow;
  g.walk_left = &walk_state(c)->nf;
  return g;
}

// Device address of the run counts the walk recorded (M2L, P2P), for the list
// grouping of graph mode.
const unsigned long long *walk_run_counts(Ctx &c, int which) {
  TravState *st = walk_state(c);
  return which == 0 ? &st->nrun_m : &st->nrun_p;
}

namespace {

// Counting sort of the runs by sink: run r of sink s goes to roff[s] + rank[r]
// (rank = its level order among the sink's runs), the order a stable sort by
// (sink, level) gives.
// nr_dev (graph mode): the run count on the device; the grid then covers the capacity nr.
__global__ void k_run_place(const uint64_t *__restrict__ key, const uint32_t *__restrict__ rank,
                            const uint32_t *__restrict__ roff, int64_t nr, const unsigned long long *nr_dev,
                            uint64_t *__restrict__ key_s, uint32_t *__restrict__ idx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (nr_dev ? (int64_t)*nr_dev : nr)) return;
  const uint64_t k = key[r];
  const uint32_t pos = roff[(uint32_t)(k >> 8)] + rank[r];
  key_s[pos] = k;
  idx[pos] = (uint32_t)r;
}

__global__ void k_run_gather(const uint32_t *__restrict__ idx, const uint32_t *__restrict__ cnt,
                             uint32_t *__restrict__ cnt_s, int64_t nr, const unsigned long long *nr_dev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  cnt_s[i] = i < (nr_dev ? (int64_t)*nr_dev : nr) ? cnt[idx[i]] : 0u;  // zeros beyond the runs (graph mode)
}

// One warp per run (runs sorted by (sink, level)): CSR bounds of its sink and a
// coalesced copy of its entries to their place in the sink-grouped list.
__global__ void k_run_copy(const uint64_t *__restrict__ key_s, const uint32_t *__restrict__ idx,
                           const uint64_t *__restrict__ beg, const uint32_t *__restrict__ cnt_s,
                           const uint32_t *__restrict__ dst, int64_t nr_host, const unsigned long long *nr_dev,
                           const uint64_t *__restrict__ src, uint64_t *__restrict__ out,
                           uint32_t *__restrict__ csr_beg, uint32_t *__restrict__ csr_end,
                           uint32_t *__restrict__ csr_mid) {
  const int64_t nr = nr_dev ? (int64_t)*nr_dev : nr_host;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nr; i += nw) {
    const uint32_t sink = (uint32_t)(key_s[i] >> 8);
    const uint32_t d = dst[i], n = cnt_s[i];
    if (lane == 0) {
      if (i == 0 || (uint32_t)(key_s[i - 1] >> 8) != sink) {
        csr_beg[sink] = d;
        if (csr_mid) csr_mid[sink] = d;  // no operator-table pairs on this path
      }
      if (i == nr - 1 || (uint32_t)(key_s[i + 1] >> 8) != sink) csr_end[sink] = d + n;
    }
    const uint64_t b = beg[idx[i]];
    for (uint32_t j = lane; j < n; j += 32) out[d + j] = src[b + j];
  }
}

}  // namespace

// The walk leaves each level's entries grouped by sink; a sink that stays a
// leaf over several levels has one run per level.  Order the runs by (sink,
// level) with a counting sort (the walk counted each sink's runs and ranked
// them by level), place them with a prefix sum of their lengths and copy: the
// list ends up grouped by sink (levels in order, walk order within a level)
// with CSR bounds.  Cost: a scan over the cells, a pass over the runs and one
// pass over the entries.
// nr_dev (graph mode): the run count on the device, nr its capacity; n is then the
// list's capacity.
static cudaError_t merge_runs(Ctx &c, DBuf &L, DBuf &A, int64_t n, DBuf &rkey, DBuf &rbeg, DBuf &rcnt, int64_t nr,
                              DBuf &rrank, DBuf &rsink, uint32_t *csr_beg, uint32_t *csr_end, uint32_t *csr_mid,
                              cudaStream_t st, const unsigned long long *nr_dev = nullptr) {
  cudaError_t e;
  if (n == 0 || nr == 0) return cudaSuccess;
  if ((e = ensure(A, n * 8)) != cudaSuccess) return e;
  // scratch: key_s u64 | idx u32 | roff u32 [nnodes] | cnt_s u32 | dst u32
  const int64_t nn = c.nnodes > 0 ? c.nnodes : 1;
  if ((e = ensure(c.tmp2, (size_t)nr * 20 + (size_t)nn * 4 + 64)) != cudaSuccess) return e;
  uint64_t *keys = P<uint64_t>(c.tmp2);
  uint32_t *idx = reinterpret_cast<uint32_t *>(keys + nr);
  uint32_t *roff = idx + nr, *cnt_s = roff + nn, *dst = cnt_s + nr;
  const int T = 256;
  uint64_t *rtotal = P<uint64_t>(c.d_small) + 1;  // (reused for the entry total below)
  if ((e = scan_u32(P<uint32_t>(rsink), roff, rtotal, (size_t)nn, c.offs, st)) != cudaSuccess) return e;
  k_run_place<<<blocks_for(nr, T), T, 0, st>>>(P<uint64_t>(rkey), P<uint32_t>(rrank), roff, nr, nr_dev, keys, idx);
  note_launch();
  k_run_gather<<<blocks_for(nr, T), T, 0, st>>>(idx, P<uint32_t>(rcnt), cnt_s, nr, nr_dev);
  note_launch();
  uint64_t *total = P<uint64_t>(c.d_small) + 1;
  if ((e = scan_u32(cnt_s, dst, total, (size_t)nr, c.offs, st)) != cudaSuccess) return e;
  unsigned g = blocks_for((size_t)nr, 8);
  if (g > 152 * 32) g = 152 * 32;
  k_run_copy<<<g, T, 0, st>>>(keys, idx, P<uint64_t>(rbeg), cnt_s, dst, nr, nr_dev, P<uint64_t>(L), P<uint64_t>(A),
                              csr_beg, csr_end, csr_mid);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::swap(L, A);
  return cudaSuccess;
}

cudaError_t p2p_list_particle_pairs(Ctx &c, cudaStream_t st, int64_t *out) {
  *out = 0;
  if (c.np2p == 0) return cudaSuccess;
  const unsigned T = 256;
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c.d_small.p);
  cudaError_t e;
  if ((e = cudaMemsetAsync(cnt, 0, 8, st)) != cudaSuccess) return e;
  k_pairs_in_list<<<blocks_for(c.np2p, T), T, 0, st>>>(P<uint64_t>(c.p2p), c.np2p, P<uint2>(c.range), cnt);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.h_pinned, cnt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  *out = (int64_t)c.h_pinned[0];
  return cudaSuccess;
}

// Group both lists by sink (the walk's order kept within a sink) and build CSR
// bounds; count the particle pairs P2P evaluates.
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
  // graph mode: capacities for the sizes, the run counts read on the device
  const bool gw = c.graph_walk;
  TRY(merge_runs(c, c.p2p, c.p2p_alt, gw ? (int64_t)c.cap_p2p : c.np2p, c.rp_key, c.rp_beg, c.rp_cnt,
                 gw ? (int64_t)c.cap_run : c.nrun_p, c.rp_rank, c.rcnt_p, P<uint32_t>(c.p2p_beg),
                 P<uint32_t>(c.p2p_end), nullptr, st, gw ? walk_run_counts(c, 1) : nullptr));
  const bool tables = ((c.prm.m2l_precision == 0 && c.prm.m2l_tables) || c.prm.m2l_precision >= 3) && c.tab_k > 0;
  if (c.nm2l > 0 && !tables) {
    TRY(merge_runs(c, c.m2l, c.m2l_alt, gw ? (int64_t)c.cap_m2l : c.nm2l, c.rm_key, c.rm_beg, c.rm_cnt,
                   gw ? (int64_t)c.cap_run : c.nrun_m, c.rm_rank, c.rcnt_m, P<uint32_t>(c.m2l_beg),
                   P<uint32_t>(c.m2l_end), P<uint32_t>(c.m2l_mid), st, gw ? walk_run_counts(c, 0) : nullptr));
    if (c.prm.mac_mode == 1) {  // learned orders: stable pass on the order bits -> (order, sink)
      bool alt = false;
      TRY(ensure(c.m2l_alt, c.nm2l * 8));
      TRY(radix_sort_u64(P<uint64_t>(c.m2l), nullptr, P<uint64_t>(c.m2l_alt), nullptr, c.nm2l, kOrderShift, 64,
                         &alt, c.tmp, st));
      if (alt) std::swap(c.m2l, c.m2l_alt);
    }
  } else if (c.nm2l > 0) {
    // operator tables: group by (sink, table bit) (learned: (order, sink, table bit))
    TRY(ensure(c.m2l_alt, c.nm2l * 8));
    bool alt = false;
    const int hi_bit = c.prm.mac_mode == 1 ? 64 : kSinkShift + sink_bits;
    TRY(radix_sort_u64(P<uint64_t>(c.m2l), nullptr, P<uint64_t>(c.m2l_alt), nullptr, c.nm2l, kGenericBit, hi_bit,
                       &alt, c.tmp, st));
    if (alt) std::swap(c.m2l, c.m2l_alt);
    if (c.prm.mac_mode != 1) {
      k_list_bounds<<<blocks_for(c.nm2l, T), T, 0, st>>>(P<uint64_t>(c.m2l), 0, c.nm2l, P<uint32_t>(c.m2l_beg),
                                                         P<uint32_t>(c.m2l_end), P<uint32_t>(c.m2l_mid));
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
  const bool lo = c.prm.m2l_precision >= 3 && c.tab_k > 0;
  const bool tab = (c.prm.m2l_precision == 0 && c.prm.m2l_tables && c.tab_k > 0) || lo;
  if (tab && !c.tab_ready) {
    cudaError_t e = m2l_table_build(c, st);
    if (e != cudaSuccess) return e;
  }
  auto run = [&](int q) -> cudaError_t {
    if (lo && m2l_lo_supported(q)) return m2l_pass_lo(c, q, st);
    if (c.prm.m2l_precision >= 3) return m2l_pass(c, q, st);  // no table: every pair on the FP32 kernel
    if (c.prm.m2l_precision != 0 && m2l_tc_supported(q)) return m2l_pass_tc(c, q, st);
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


namespace {

}  // namespace

int sink_batches_for(const Ctx &c) {
  if (c.prm.sink_batches > 0) return c.prm.sink_batches;
  const double guess = p2p_guess_per_particle(c) * (double)c.n;
  // one batch while the guess stays below 2^28 entries; beyond, batches of about 2^27
  if (guess <= (double)(1u << 28)) return 1;
  return (int)std::min(4096.0, std::ceil(guess / (double)(1u << 27)));
}

namespace {

// One batch's frontier: the pairs [f_lo, f_lo + nfb) and segments
// [s_lo, s_lo + nsb) of the saved top-level frontier, rebased to the start of
// the walk's first buffers (segment starts, and the segment of each sink).
__global__ void k_batch_frontier(const uint64_t *__restrict__ tp, const uint32_t *__restrict__ tsegs,
                                 const unsigned long long *__restrict__ tsst, unsigned long long f_lo,
                                 unsigned long long nfb, unsigned long long s_lo, unsigned long long nsb,
                                 uint64_t *__restrict__ fa, uint32_t *__restrict__ seg_a,
                                 unsigned long long *__restrict__ st_a, uint32_t *__restrict__ map_a) {
  const unsigned long long n = nfb > nsb ? nfb : nsb;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (i < nfb) fa[i] = tp[f_lo + i];
    if (i < nsb) {
      const uint32_t sk = tsegs[s_lo + i];
      seg_a[i] = sk;
      st_a[i] = tsst[s_lo + i] - f_lo;
      map_a[sk] = (uint32_t)i;
    }
  }
}

// Particles in each segment's sink cell (the batches are balanced on them).
__global__ void k_seg_counts(const uint32_t *__restrict__ segs, unsigned long long ns, const uint2 *__restrict__ range,
                             uint32_t *__restrict__ cnt) {
  const unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) cnt[s] = range[segs[s]].y;
}

// the levels the walk takes before its frontier is split into batches: up to
// 8^4 sink cells (and shallower leaves) for a few batches, 8^5 or 8^6 for more,
// so that one cell holds a small share of a batch
inline int batch_level(int nbatch) { return 4 + (nbatch > 8 ? 1 : 0) + (nbatch > 64 ? 1 : 0); }

}  // namespace

// Sink batches.  The walk is sink-major: at each level its frontier is grouped
// into segments, one per sink cell, in Morton order of the sinks, and a
// segment's pairs are contiguous.  A batch of sinks is therefore a contiguous
// run of segments of the frontier, and the walk below it touches no other
// sink.  The walk first takes the top levels alone; what it emitted there (M2L
// to cells above the batch level, P2P of leaves above it) is grouped and
// evaluated at once.  Its frontier is saved and cut into nbatch runs whose sink
// cells hold about equal particle counts; each run is copied into the walk's buffers, the walk
// resumes from it to the leaves, and its lists are grouped and evaluated (M2L
// into L, P2P into c.pacc); the next batch reuses the buffers, whose first
// guesses are a batch's share.  The same pairs are classified as in one walk,
// so the lists are the same entries, split by sink; a leaf above the batch
// level gets its entries in two groups (top levels, then its batch), summed in
// two steps.  Finally L2L, and L2P adds the P2P accelerations.
cudaError_t short_range_batched(Ctx &c, float *acc, int nbatch, cudaStream_t st) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  const int64_t n = c.n;
  TRY(ensure(c.pacc, (size_t)3 * n * sizeof(float)));
  TRY(cudaMemsetAsync(c.pacc.p, 0, (size_t)3 * n * sizeof(float), st));
  float *pacc = P<float>(c.pacc);
  c.walk_share = 1.0 / nbatch;
  WalkPlan w;
  e = walk_plan(c, w);
  c.walk_share = 1.0;
  if (e != cudaSuccess) return e;
  int64_t tot_m2l = 0, tot_p2p = 0, walks = 0, items = 0;
  int iters = 0;
  auto grow_lists = [&](const TravState &hs) {
    auto grow = [](uint64_t want) { return want + want / 4 + 1024; };
    auto up = [&](uint64_t &cap, int bit, int k) {
      if (hs.ovf_lists & bit) cap = grow(std::max<uint64_t>(cap * 2, hs.need[k]));
    };
    up(c.cap_m2l, 1, 0);
    up(c.cap_p2p, 2, 1);
    up(c.cap_front, 4, 2);
    up(c.cap_seg, 8, 3);
    up(c.cap_run, 16, 4);
  };
  auto read_state = [&](TravState &hs) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(c.h_pinned, walk_state(c), sizeof(TravState), cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    if (r == cudaSuccess) std::memcpy(&hs, c.h_pinned, sizeof(TravState));
    return r;
  };
  // group and evaluate what one walk emitted (its sizes from the state)
  auto evaluate = [&](const TravState &hs) -> cudaError_t {
    c.nm2l = (int64_t)hs.nm2l;
    c.np2p = (int64_t)hs.np2p;
    c.nrun_m = (int64_t)hs.nrun_m;
    c.nrun_p = (int64_t)hs.nrun_p;
    tot_m2l += c.nm2l;
    tot_p2p += c.np2p;
    items += (int64_t)hs.items;
    iters += hs.iters;
    if (c.nm2l > (int64_t)UINT32_MAX || c.np2p > (int64_t)UINT32_MAX) return cudaErrorInvalidValue;
    cudaError_t r = sort_lists(c, st);
    if (r == cudaSuccess) r = m2l_all(c, st);
    if (r == cudaSuccess) r = c.prm.p2p_mutual ? p2p_pass_mutual(c, pacc, st) : p2p_pass(c, pacc, st);
    return r;
  };
  // ---- the top levels
  TravState hs;
  WalkStart top;
  const int split_level = batch_level(nbatch);
  top.max_iters = split_level;
  for (int attempt = 0;; ++attempt) {
    if (attempt == 32) return cudaErrorInvalidValue;
    ++walks;
    TRY(walk_buffers(c, w.nb));
    TRY(walk_launch(c, w, st, top));
    TRY(read_state(hs));
    if (hs.overflow == 2) return cudaErrorInvalidValue;
    if (!hs.overflow) break;
    grow_lists(hs);
  }
  const unsigned long long nf_top = hs.nf, ns_top = hs.nseg;
  const bool odd = (hs.iters & 1) != 0;  // the frontier left is in the second buffers
  // save the frontier before the evaluation reuses anything
  if (nf_top > 0) {
    TRY(ensure(c.tf_pairs, nf_top * 8));
    TRY(ensure(c.tf_segs, ns_top * 4));
    TRY(ensure(c.tf_sst, ns_top * 8));
    TRY(cudaMemcpyAsync(c.tf_pairs.p, odd ? c.front_next.p : c.front.p, nf_top * 8, cudaMemcpyDeviceToDevice, st));
    TRY(cudaMemcpyAsync(c.tf_segs.p, odd ? c.seg_b.p : c.seg_a.p, ns_top * 4, cudaMemcpyDeviceToDevice, st));
    TRY(cudaMemcpyAsync(c.tf_sst.p, odd ? c.acc_b.p : c.acc_a.p, ns_top * 8, cudaMemcpyDeviceToDevice, st));
  }
  TRY(evaluate(hs));
  // ---- the batches: runs of segments with about equal particle counts in their sinks
  std::vector<unsigned long long> sst(ns_top), cum(ns_top + 1, 0);
  if (ns_top > 0) {
    std::vector<uint32_t> cnt(ns_top);
    TRY(ensure(c.tmp2, ns_top * 4));
    k_seg_counts<<<blocks_for(ns_top, 256), 256, 0, st>>>(P<uint32_t>(c.tf_segs), ns_top, P<uint2>(c.range),
                                                           P<uint32_t>(c.tmp2));
    note_launch();
    TRY(cudaGetLastError());
    TRY(cudaMemcpyAsync(cnt.data(), c.tmp2.p, ns_top * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(sst.data(), c.tf_sst.p, ns_top * 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    for (unsigned long long q = 0; q < ns_top; ++q) cum[q + 1] = cum[q] + cnt[q];
  }
  unsigned long long s_lo = 0;
  int ran = 0;
  for (int b = 0; b < nbatch && s_lo < ns_top; ++b, ++ran) {
    const unsigned long long target = (unsigned long long)((double)cum[ns_top] * (b + 1) / nbatch);
    unsigned long long s_hi = s_lo + 1;
    while (s_hi < ns_top && (b == nbatch - 1 || cum[s_hi] < target)) ++s_hi;
    const unsigned long long f_lo = sst[s_lo], f_hi = s_hi < ns_top ? sst[s_hi] : nf_top;
    WalkStart ws;
    ws.resume = 1;
    ws.iter0 = split_level;
    ws.max_iters = 2 * kDepth + 6 - split_level;
    ws.nf = f_hi - f_lo;
    ws.nseg = s_hi - s_lo;
    for (int attempt = 0;; ++attempt) {
      if (attempt == 32) return cudaErrorInvalidValue;
      ++walks;
      if (c.cap_front < ws.nf) c.cap_front = ws.nf + ws.nf / 4 + 1024;
      if (c.cap_seg < ws.nseg) c.cap_seg = ws.nseg + ws.nseg / 4 + 1024;
      TRY(walk_buffers(c, w.nb));
      const int T = 256;
      unsigned g = blocks_for(std::max(ws.nf, ws.nseg), T);
      if (g > 152u * 8u) g = 152u * 8u;
      k_batch_frontier<<<g, T, 0, st>>>(P<uint64_t>(c.tf_pairs), P<uint32_t>(c.tf_segs),
                                        P<unsigned long long>(c.tf_sst), f_lo, ws.nf, s_lo, ws.nseg,
                                        P<uint64_t>(c.front), P<uint32_t>(c.seg_a), P<unsigned long long>(c.acc_a),
                                        P<uint32_t>(c.fseg));
      note_launch();
      TRY(cudaGetLastError());
      TRY(walk_launch(c, w, st, ws));
      TRY(read_state(hs));
      if (hs.overflow == 2) return cudaErrorInvalidValue;
      if (!hs.overflow) break;
      grow_lists(hs);
    }
    if (hs.nf != 0) return cudaErrorInvalidValue;  // more levels than any octree
    TRY(evaluate(hs));
    s_lo = s_hi;
  }
  c.nm2l = tot_m2l;
  c.np2p = tot_p2p;
  c.traverse_walks = walks;
  c.frontier_items = items;
  c.traverse_iters = iters;
  c.last_batches = ran > 1 ? ran : 1;
  c.lists_split = true;  // the top levels' lists and each batch's were evaluated in turn
  return downward(c, acc, st, pacc);
#undef TRY
}

}  // namespace hfmm
