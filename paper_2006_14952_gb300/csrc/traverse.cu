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
#include "mlp.cuh"

namespace hfmm {
namespace {

enum : uint8_t { kSkip = 0, kM2L = 1, kP2P = 2, kOpenA = 3, kOpenB = 4, kOpenAB = 5 };
constexpr uint8_t kCandidate = 6;  // internal: needs the network's decision

struct Mac {
  double rc2h, theta2;
  int rule, size_rule;
  int mode;   // 0 geometric, 1 learned, 2 collect
  int order;  // p (geometric M2L order, and the largest learned order)
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
  int64_t dd[3];
  half_delta(ca, cb, s, dd);
  const int64_t wa = half_width(ca.w), wb = half_width(cb.w), ext = wa + wb;
  int64_t sc2 = 0, sm2 = 0, sx2 = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int64_t a = dd[d] < 0 ? -dd[d] : dd[d];
    int64_t g = a - ext > 0 ? a - ext : 0;
    int64_t f = a + ext;
    sc2 += a * a;
    sm2 += g * g;
    sx2 += f * f;
  }
  if ((double)sm2 > m.rc2h) return kSkip;
  bool trans = m.rule == 0 ? ((double)sc2 > m.rc2h) : ((double)sx2 > m.rc2h);
  int64_t wl = m.size_rule == 0 ? wb : (wa > wb ? wa : wb);
  if (!trans && (double)(4 * wl * wl) <= __dmul_rn(m.theta2, (double)sc2))
    return m.mode == 0 ? kM2L : kCandidate;  // sc2 = 0 (a self pair) never passes
  return open_rule(ca, cb, ka, kb);
}

__global__ void k_init_frontier(uint64_t *f) {
  int s = threadIdx.x;
  if (s < 27) f[s] = pack_pair(0, 0, (uint32_t)s);
}

// counts layout [3][nf]: M2L flags, P2P flags, child-pair counts.
// cls: bits 0..2 the class, bits 3..6 the M2L order.
__global__ void __launch_bounds__(256) k_mac_count(const uint64_t *__restrict__ f, int64_t nf,
                                                   const uint4 *__restrict__ cell, const int2 *__restrict__ kids,
                                                   Mac m, uint8_t *__restrict__ cls, uint32_t *__restrict__ counts) {
  __shared__ uint32_t sw[kMlpSmemWords];
  __shared__ __align__(16) __nv_bfloat16 xs[8][32 * 16];
  __shared__ uint8_t dec[8][32];
  if (m.mode == 1) {
    mlp_stage(m.w, sw);
    __syncthreads();
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < nf;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
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
  if (m.mode == 1) {  // warp-batched network decisions for the candidates
    const unsigned want = __ballot_sync(0xffffffffu, c == kCandidate);
    if (want) {
      const int slot = __popc(want & ((1u << lane) - 1u)), nc = __popc(want);
      __nv_bfloat16 *row = xs[wp] + slot * 16;
      if (c == kCandidate) {
        float ft[kMlpIn];
        pair_features(ca, cb, s, m.range[a].y, m.range[b].y, m.M + (size_t)b * m.ldm, m.inv_rs_h, m.inv_rc_h, ft);
#pragma unroll
        for (int k = 0; k < 16; ++k) row[k] = __float2bfloat16_rn(k < kMlpIn ? ft[k] : 0.f);
      }
      for (int r = nc + lane; r < ((nc + 15) & ~15); r += 32)
#pragma unroll
        for (int k = 0; k < 16; ++k) xs[wp][r * 16 + k] = __float2bfloat16_rn(0.f);
      __syncwarp();
      for (int bt = 0; bt < nc; bt += 16) {
        float l[4];
        mlp_logits16(sw, xs[wp] + bt * 16, l);
        int c0, c8;
        mlp_argmax16(l, c0, c8);
        if ((lane & 3) == 0) {
          dec[wp][bt + (lane >> 2)] = (uint8_t)c0;
          dec[wp][bt + (lane >> 2) + 8] = (uint8_t)c8;
        }
      }
      __syncwarp();
      if (c == kCandidate) {
        const int k = dec[wp][slot];
        if (k == 0) {
          c = open_rule(ca, cb, ka, kb);
        } else {
          c = kM2L;
          order = (uint32_t)(k + 1) < order ? (uint32_t)(k + 1) : order;
        }
      }
    }
  }
  if (!valid) return;
  cls[t] = (uint8_t)(c | (order << 3));
  uint32_t nm = c == kM2L, np = c == kP2P, nch = 0;
  if (c == kOpenA) nch = ka.y;
  if (c == kOpenB) nch = kb.y;
  if (c == kOpenAB) nch = ka.y * kb.y;
  counts[t] = nm;
  counts[nf + t] = np;
  counts[2 * nf + t] = nch;
}

__global__ void k_mac_emit(const uint64_t *__restrict__ f, int64_t nf, const uint8_t *__restrict__ cls,
                           const uint32_t *__restrict__ offs, const int2 *__restrict__ kids,
                           uint64_t *__restrict__ m2l, uint64_t *__restrict__ p2p, uint64_t *__restrict__ next) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  const uint8_t cc = cls[t];
  const uint8_t c = cc & 7;
  if (c == kSkip) return;
  uint64_t e = f[t];
  if (c == kM2L) {
    m2l[offs[t]] = with_order(e, cc >> 3);
    return;
  }
  uint32_t base1 = offs[nf], base2 = offs[2 * nf];
  if (c == kP2P) {
    p2p[offs[nf + t] - base1] = e;
    return;
  }
  uint32_t a = pair_sink(e), b = pair_src(e), s = pair_shift(e);
  int2 ka = kids[a], kb = kids[b];
  uint32_t a0 = a, na = 1, b0 = b, nb = 1;
  if (c == kOpenA || c == kOpenAB) {
    a0 = (uint32_t)ka.x;
    na = (uint32_t)ka.y;
  }
  if (c == kOpenB || c == kOpenAB) {
    b0 = (uint32_t)kb.x;
    nb = (uint32_t)kb.y;
  }
  uint64_t *o = next + (offs[2 * nf + t] - base2);
  for (uint32_t x = 0; x < na; ++x)
    for (uint32_t y = 0; y < nb; ++y) *o++ = pack_pair(a0 + x, b0 + y, s);
}

// CSR bounds of the entries [lo, hi) of a list sorted by sink: beg[k] .. end[k].
__global__ void k_list_bounds(const uint64_t *__restrict__ lst, int64_t lo, int64_t hi, uint32_t *__restrict__ beg,
                              uint32_t *__restrict__ end) {
  int64_t t = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= hi) return;
  uint32_t s = pair_sink(lst[t]);
  if (t == lo || pair_sink(lst[t - 1]) != s) beg[s] = (uint32_t)t;
  if (t == hi - 1 || pair_sink(lst[t + 1]) != s) end[s] = (uint32_t)(t + 1);
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

}  // namespace

cudaError_t traverse(Ctx &c, cudaStream_t st) {
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  const int T = 256;
  c.nm2l = c.np2p = 0;
  c.traverse_iters = 0;
  if (c.n == 0) return cudaSuccess;
  Mac m{};
  m.rc2h = c.rc2h;
  m.theta2 = c.theta2;
  m.rule = c.prm.transition_rule;
  m.size_rule = c.prm.size_rule;
  m.mode = c.collect ? 2 : c.prm.mac_mode;
  m.order = c.p;
  m.w = static_cast<const __nv_bfloat16 *>(c.mlp_w.p);
  m.M = P<float>(c.M);
  m.range = P<uint2>(c.range);
  m.ldm = c.nc;
  m.inv_rs_h = (float)(c.prm.box / (double)kHalfBox / c.rs);
  m.inv_rc_h = (float)(c.prm.box / (double)kHalfBox / c.rc);
  m.cand = P<uint64_t>(c.cand);
  m.ncand = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 7);
  m.cand_cap = c.cand_cap;
  m.sample_mod = c.sample_mod ? c.sample_mod : 1u;
  int64_t nf = 27;
  TRY(ensure(c.front, 1024 * 8));
  k_init_frontier<<<1, 32, 0, st>>>(P<uint64_t>(c.front));
  note_launch();
  size_t cap_m2l = c.m2l.cap / 8, cap_p2p = c.p2p.cap / 8;
  uint64_t *d_tot = P<uint64_t>(c.d_small);
  while (nf > 0) {
    TRY(ensure(c.cls, nf));
    TRY(ensure(c.counts, 3 * nf * sizeof(uint32_t)));
    TRY(ensure(c.offs, 3 * nf * sizeof(uint32_t)));
    k_mac_count<<<blocks_for(nf, T), T, 0, st>>>(P<uint64_t>(c.front), nf, P<uint4>(c.cell), P<int2>(c.kids), m,
                                                 P<uint8_t>(c.cls), P<uint32_t>(c.counts));
    note_launch();
    TRY(scan_u32(P<uint32_t>(c.counts), P<uint32_t>(c.offs), d_tot, 3 * nf, c.tmp, st));
    TRY(cudaMemcpyAsync(c.h_pinned, P<uint32_t>(c.offs) + nf, 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(reinterpret_cast<uint32_t *>(c.h_pinned) + 1, P<uint32_t>(c.offs) + 2 * nf, 4,
                        cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(c.h_pinned + 1, d_tot, 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    uint64_t s0 = reinterpret_cast<uint32_t *>(c.h_pinned)[0];
    uint64_t s01 = reinterpret_cast<uint32_t *>(c.h_pinned)[1];
    uint64_t tot = c.h_pinned[1];
    if (tot >= 0xffffffffull) return cudaErrorInvalidValue;
    int64_t add_m2l = (int64_t)s0, add_p2p = (int64_t)(s01 - s0), nch = (int64_t)(tot - s01);
    if ((size_t)(c.nm2l + add_m2l) > cap_m2l) {
      TRY(ensure_keep(c.m2l, (c.nm2l + add_m2l) * 8 * 2, c.nm2l * 8, st));
      cap_m2l = c.m2l.cap / 8;
    }
    if ((size_t)(c.np2p + add_p2p) > cap_p2p) {
      TRY(ensure_keep(c.p2p, (c.np2p + add_p2p) * 8 * 2, c.np2p * 8, st));
      cap_p2p = c.p2p.cap / 8;
    }
    TRY(ensure(c.front_next, (nch > 0 ? nch : 1) * 8));
    k_mac_emit<<<blocks_for(nf, T), T, 0, st>>>(P<uint64_t>(c.front), nf, P<uint8_t>(c.cls), P<uint32_t>(c.offs),
                                                P<int2>(c.kids), P<uint64_t>(c.m2l) + c.nm2l,
                                                P<uint64_t>(c.p2p) + c.np2p, P<uint64_t>(c.front_next));
    note_launch();
    TRY(cudaGetLastError());
    c.nm2l += add_m2l;
    c.np2p += add_p2p;
    std::swap(c.front, c.front_next);
    nf = nch;
    ++c.traverse_iters;
  }
  return cudaSuccess;
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
    // learned M2L entries carry their order in the top bits: group by (order, sink)
    const int hi_bit = (!which && c.prm.mac_mode == 1) ? 64 : kSinkShift + sink_bits;
    TRY(radix_sort_u64(P<uint64_t>(L), nullptr, P<uint64_t>(A), nullptr, n, kSinkShift, hi_bit, &alt, c.tmp, st));
    if (alt) std::swap(L, A);
    if (which || c.prm.mac_mode != 1) {
      k_list_bounds<<<blocks_for(n, T), T, 0, st>>>(P<uint64_t>(L), 0, n, P<uint32_t>(which ? c.p2p_beg : c.m2l_beg),
                                                    P<uint32_t>(which ? c.p2p_end : c.m2l_end));
      note_launch();
      TRY(cudaGetLastError());
    }
  }
  c.p2p_particle_pairs = -1;
  if ((c.prm.profile & 2) && c.np2p > 0) {
    TRY(cudaMemsetAsync(c.d_small.p, 0, 8, st));
    k_pairs_in_list<<<blocks_for(c.np2p, T), T, 0, st>>>(P<uint64_t>(c.p2p), c.np2p, P<uint2>(c.range),
                                                         reinterpret_cast<unsigned long long *>(c.d_small.p));
    note_launch();
    TRY(cudaMemcpyAsync(c.h_pinned, c.d_small.p, 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    c.p2p_particle_pairs = (int64_t)c.h_pinned[0];
  }
  return cudaSuccess;
#undef TRY
}

cudaError_t m2l_all(Ctx &c, cudaStream_t st) {
  if (c.nm2l == 0) return cudaSuccess;
  auto run = [&](int q) -> cudaError_t {
    if (c.prm.m2l_precision == 1 && m2l_tc_supported(q)) return m2l_pass_tc(c, q, st);
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
    k_list_bounds<<<blocks_for(hi - lo, T), T, 0, st>>>(P<uint64_t>(c.m2l), lo, hi, P<uint32_t>(c.m2l_beg),
                                                        P<uint32_t>(c.m2l_end));
    note_launch();
    if ((e = run(q)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace hfmm
