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
#include "common.cuh"

namespace hfmm {
namespace {

enum : uint8_t { kSkip = 0, kM2L = 1, kP2P = 2, kOpenA = 3, kOpenB = 4, kOpenAB = 5 };

struct Mac {
  double rc2h, theta2;
  int rule, size_rule;
};

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
  if (!trans && (double)(4 * wl * wl) <= __dmul_rn(m.theta2, (double)sc2)) return kM2L;
  bool la = ka.y == 0, lb = kb.y == 0;
  if (la && lb) return kP2P;
  if (la) return kOpenB;
  if (lb) return kOpenA;
  if (ca.w < cb.w) return kOpenA;
  if (cb.w < ca.w) return kOpenB;
  return kOpenAB;
}

__global__ void k_init_frontier(uint64_t *f) {
  int s = threadIdx.x;
  if (s < 27) f[s] = pack_pair(0, 0, (uint32_t)s);
}

// counts layout [3][nf]: M2L flags, P2P flags, child-pair counts.
__global__ void k_mac_count(const uint64_t *__restrict__ f, int64_t nf, const uint4 *__restrict__ cell,
                            const int2 *__restrict__ kids, Mac m, uint8_t *__restrict__ cls,
                            uint32_t *__restrict__ counts) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  uint64_t e = f[t];
  uint32_t a = pair_sink(e), b = pair_src(e), s = pair_shift(e);
  int2 ka = kids[a], kb = kids[b];
  uint8_t c = classify(cell[a], cell[b], s, ka, kb, m);
  cls[t] = c;
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
  uint8_t c = cls[t];
  if (c == kSkip) return;
  uint64_t e = f[t];
  if (c == kM2L) {
    m2l[offs[t]] = e;
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

// CSR bounds of a list sorted by sink: beg[k] .. end[k].
__global__ void k_list_bounds(const uint64_t *__restrict__ lst, int64_t n, uint32_t *__restrict__ beg,
                              uint32_t *__restrict__ end) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint32_t s = pair_sink(lst[t]);
  if (t == 0 || pair_sink(lst[t - 1]) != s) beg[s] = (uint32_t)t;
  if (t == n - 1 || pair_sink(lst[t + 1]) != s) end[s] = (uint32_t)(t + 1);
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
  Mac m{c.rc2h, c.theta2, c.prm.transition_rule, c.prm.size_rule};
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
    TRY(radix_sort_u64(P<uint64_t>(L), nullptr, P<uint64_t>(A), nullptr, n, kSinkShift, kSinkShift + sink_bits, &alt,
                       c.tmp, st));
    if (alt) std::swap(L, A);
    k_list_bounds<<<blocks_for(n, T), T, 0, st>>>(P<uint64_t>(L), n, P<uint32_t>(which ? c.p2p_beg : c.m2l_beg),
                                                  P<uint32_t>(which ? c.p2p_end : c.m2l_end));
    note_launch();
    TRY(cudaGetLastError());
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

}  // namespace hfmm
