// Mutual cut-off P2P (Newton's third law; p2p_mutual = 1): every particle pair
// of a leaf pair is evaluated once and acts on both particles.
//
// The walk keeps one ordered pair (A, B, s) of each mirror couple (p2p_owner:
// the deeper leaf, by parity within a level; a leaf against its own periodic
// images keeps s <= 13), so each sink leaf A's list holds the partners it owns.  Pass 1 (k_p2p_mut) runs one warp
// per sink leaf like the one-sided kernel: the sources of the leaf's list are
// staged through shared memory in fills (asynchronous copies one fill ahead,
// moved into A's frame, culled against the bounding box of the sink chunk,
// paired up), and each lane keeps kPL pairs of staged sources in registers for a
// round while the chunk's sinks rotate through the lanes: in a group of G lanes
// (G the power of two at or above the chunk size) the sink and the force it has
// gathered move one lane per step, so after G steps every sink has met every
// source pair of the group and is back home, and each lane's two sources have
// gathered the reaction of every sink in registers.  A source's reaction is
// stored in a partial sum of its list entry (the first sink chunk of the leaf
// stores, later chunks add; a culled source gets a zero from the first chunk).
// Pass 2 (k_p2p_reactions) adds, for every source leaf B, the partials of the
// entries it appears in, in the order of a stable sort of those entries by B,
// to B's accelerations.  No atomics: the sums do not depend on scheduling.
// The leaf against itself (shift 13) stays one-sided: both orders of each pair
// are evaluated by the sink warp and there is no reaction.
#include <utility>

#include "p2p_common.cuh"

namespace hfmm {
namespace {

constexpr uint32_t kNoSlot = 0xffffffffu;  // a staged source without a reaction (the leaf itself)
constexpr int kCapM = 256;                 // source particles per fill
constexpr int kPL = 4;                     // source pairs a lane holds in one rotation round

__device__ __forceinline__ int pow2_at_least(int c) {
  return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : 32;
}

template <bool kCount, int kSplit>
__global__ void __launch_bounds__(256, 2)
    k_p2p_mut(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
              const uint2 *__restrict__ range, const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
              const uint64_t *__restrict__ lst, const uint32_t *__restrict__ poff, const float4 *__restrict__ pm4,
              const uint32_t *__restrict__ perm, int64_t n, float box, PairFit2 fit, float G,
              float *__restrict__ acc_out, float *__restrict__ part, uint64_t npart,
              unsigned long long *__restrict__ ctr) {
  extern __shared__ float4 p2p_smem[];
  // per warp: the 32 list entries of the pending fill (first staged particle,
  // exclusive candidate offset, leaf-centre offset in the sink's frame, partial
  // base and whether the entry has a reaction), each candidate's entry, the
  // partial slot of each kept source and the chunk's sink bounding box
  __shared__ uint32_t e_src[8][32], e_excl[8][32], e_pb[8][32];
  __shared__ float e_off[8][3][32];
  __shared__ uint8_t e_re[8][32];
  __shared__ uint8_t e_own[8][kCapM];
  __shared__ uint32_t ks[8][kCapM];
  __shared__ float e_box[8][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float4 *raw = p2p_smem + wid * kCapM;
  float4 *buf = p2p_smem + (8 + wid) * kCapM;
  float *bf = reinterpret_cast<float *>(buf);
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);
  const float rc2_cull = fit.rc2 * (1.f + 1.f / 4096.f);
  const float half_unit = box / (float)kHalfBox;
  float *px_part = part, *py_part = part + npart, *pz_part = part + 2 * npart;
  uint32_t n_in = 0;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= nl) break;
    const uint32_t k = leaves[t];
    const uint4 ca = cell[k];
    const uint2 r = range[k];
    const uint32_t tb = beg[k], te = end[k];

    uint64_t pf_e = 0;
    uint32_t pf_po = 0;
    uint2 pf_rb = make_uint2(0u, 0u);
    uint4 pf_cb = make_uint4(0u, 0u, 0u, 0u);
    auto fetch_lst = [&](uint32_t q) {
      if (q + lane < te) {
        pf_e = lst[q + lane];
        pf_po = poff[q + lane];
      }
    };
    auto fetch_src = [&](uint32_t q) {
      if (q + lane < te) {
        const uint32_t b = pair_src(pf_e);
        pf_rb = range[b];
        pf_cb = cell[b];
      }
    };
    // issue the fill starting at list entry q (first jq particles of it taken)
    auto issue = [&](uint32_t &q, uint32_t &jq) -> uint32_t {
      const uint32_t qi = q + lane;
      const bool valid = qi < te;
      uint32_t cnt = 0, first = 0, pb = 0;
      uint8_t re = 0;
      float dx = 0.f, dy = 0.f, dz = 0.f;
      if (valid) {
        const uint64_t e = pf_e;
        const uint2 rb = pf_rb;
        int dd[3];
        half_delta32(ca, pf_cb, pair_shift(e), dd);
        dx = (float)dd[0] * half_unit;
        dy = (float)dd[1] * half_unit;
        dz = (float)dd[2] * half_unit;
        first = rb.x;
        cnt = rb.y;
        re = (pair_src(e) == k && pair_shift(e) == 13u) ? 0 : 1;
        pb = pf_po - rb.x;  // slot of particle g of B: pb + g (modulo 2^32)
      }
      const uint32_t start = lane == 0 ? jq : 0u;
      const uint32_t avail = valid ? cnt - start : 0u;
      uint32_t incl = avail;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t excl = incl - avail;
      e_src[wid][lane] = first + start;
      e_excl[wid][lane] = excl;
      e_pb[wid][lane] = pb;
      e_re[wid][lane] = re;
      e_off[wid][0][lane] = dx;
      e_off[wid][1][lane] = dy;
      e_off[wid][2][lane] = dz;
      __syncwarp();
      const uint32_t all = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t tot = all < (uint32_t)kCapM ? all : (uint32_t)kCapM;
      for (uint32_t pb0 = 0; pb0 < tot; pb0 += 128) {
        int own[4];
        uint32_t idx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t p = pb0 + lane + 32 * u;
          int o = 0;
#pragma unroll
          for (int step = 16; step; step >>= 1)
            if (e_excl[wid][o + step] <= p) o += step;
          own[u] = o;
          idx[u] = e_src[wid][o] + (p - e_excl[wid][o]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t p = pb0 + lane + 32 * u;
          if (p < tot) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(raw_s + 16u * p), "l"(pm4 + idx[u])
                         : "memory");
            e_own[wid][p] = (uint8_t)own[u];
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      const unsigned full = __ballot_sync(0xffffffffu, valid && incl <= (uint32_t)kCapM);
      const int nfull = __popc(full);
      const uint32_t pex = __shfl_sync(0xffffffffu, excl, nfull & 31);
      const uint32_t pstart = nfull == 0 ? jq : 0u;
      const bool partial = nfull < 32 && q + nfull < te;
      jq = partial ? pstart + (pex < (uint32_t)kCapM ? (uint32_t)kCapM - pex : 0u) : 0u;
      q += nfull;
      fetch_lst(q);
      return tot;
    };

    for (uint32_t cbase = r.x; cbase < r.x + r.y; cbase += 32) {
      const uint32_t rem = r.x + r.y - cbase;
      const int cs = rem < 32 ? (int)rem : 32;
      const bool first_chunk = cbase == r.x;
      const int Gs = pow2_at_least(cs);  // lanes per rotation group
      const int grp0 = lane & ~(Gs - 1), lg = lane & (Gs - 1);
      const int src_lane = grp0 + ((lg + 1) & (Gs - 1));
      // the rotating sink (position in the leaf frame, mass) and the force it has gathered
      float4 si = lg < cs ? pm4[cbase + lg] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
      float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);  // packed halves, added at the end
      {
        const float4 xi = pm4[cbase + (lane < cs ? lane : 0)];
        float lo0 = xi.x, lo1 = xi.y, lo2 = xi.z, hi0 = xi.x, hi1 = xi.y, hi2 = xi.z;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
          lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
          lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
          hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
          hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
          hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
        }
        if (lane == 0) {
          e_box[wid][0] = lo0;
          e_box[wid][1] = lo1;
          e_box[wid][2] = lo2;
          e_box[wid][3] = hi0;
          e_box[wid][4] = hi1;
          e_box[wid][5] = hi2;
        }
      }
      uint32_t q = tb, jq = 0;
      bool pending = q < te;
      fetch_lst(q);
      fetch_src(q);
      uint32_t tot = pending ? issue(q, jq) : 0u;
      while (pending) {
        fetch_src(q);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        uint32_t kept = 0;
        {
          const float bx0 = e_box[wid][0], by0 = e_box[wid][1], bz0 = e_box[wid][2];
          const float bx1 = e_box[wid][3], by1 = e_box[wid][4], bz1 = e_box[wid][5];
          for (uint32_t pb0 = 0; pb0 < tot; pb0 += 128) {
            float4 v[4];
            int o[4];
            uint32_t slot[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t p = pb0 + lane + 32 * u;
              const uint32_t pc = p < tot ? p : 0u;
              v[u] = raw[pc];
              o[u] = e_own[wid][pc];
              const uint32_t gi = e_src[wid][o[u]] + (pc - e_excl[wid][o[u]]);
              slot[u] = e_re[wid][o[u]] ? e_pb[wid][o[u]] + gi : kNoSlot;
            }
            bool keep[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              v[u].x += e_off[wid][0][o[u]];
              v[u].y += e_off[wid][1][o[u]];
              v[u].z += e_off[wid][2][o[u]];
              const float gx = fmaxf(fmaxf(bx0 - v[u].x, v[u].x - bx1), 0.f);
              const float gy = fmaxf(fmaxf(by0 - v[u].y, v[u].y - by1), 0.f);
              const float gz = fmaxf(fmaxf(bz0 - v[u].z, v[u].z - bz1), 0.f);
              const bool in = pb0 + lane + 32 * u < tot;
              keep[u] = in && gx * gx + gy * gy + gz * gz <= rc2_cull;
              // a culled source gets no reaction from this chunk; the first chunk
              // still writes its partial (zero), later chunks add to it
              if (in && !keep[u] && first_chunk && slot[u] != kNoSlot) {
                px_part[slot[u]] = 0.f;
                py_part[slot[u]] = 0.f;
                pz_part[slot[u]] = 0.f;
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned kb = __ballot_sync(0xffffffffu, keep[u]);
              if (keep[u]) {
                const uint32_t s = kept + (uint32_t)__popc(kb & ((1u << lane) - 1u));
                float *a = bf + (s >> 1) * 8 + (s & 1);  // pair s/2: {x0 x1 y0 y1} {z0 z1 w0 w1}
                a[0] = -v[u].x;
                a[2] = -v[u].y;
                a[4] = -v[u].z;
                a[6] = -v[u].w;
                ks[wid][s] = slot[u];
              }
              kept += (uint32_t)__popc(kb);
            }
          }
        }
        if ((kept & 1) && lane == 0) {  // pad: massless, far beyond the cut-off, no reaction
          float *a = bf + (kept >> 1) * 8 + 1;
          a[0] = -1e18f;
          a[2] = -1e18f;
          a[4] = -1e18f;
          a[6] = 0.f;
          ks[wid][kept] = kNoSlot;
        }
        __syncwarp();
        pending = q < te;
        if (pending) tot = issue(q, jq);
        // rounds of 32 kPL source pairs: lane holds pairs base + 32 u + lane (u < kPL,
        // independent chains between two rotations), the sinks rotate
        const int np = (int)((kept + 1) >> 1);
        for (int base = 0; base < np; base += 32 * kPL) {
          float2 jx[kPL], jy[kPL], jz[kPL], nmj[kPL], Rx[kPL], Ry[kPL], Rz[kPL];
          uint32_t s0[kPL], s1[kPL];
#pragma unroll
          for (int u = 0; u < kPL; ++u) {
            const int qq = base + 32 * u + lane;
            float4 A = make_float4(-1e18f, -1e18f, -1e18f, -1e18f), B = make_float4(-1e18f, -1e18f, 0.f, 0.f);
            s0[u] = kNoSlot;
            s1[u] = kNoSlot;
            if (qq < np) {
              A = buf[2 * qq];
              B = buf[2 * qq + 1];
              s0[u] = ks[wid][2 * qq];
              s1[u] = ks[wid][2 * qq + 1];
            }
            jx[u] = make_float2(A.x, A.y);
            jy[u] = make_float2(A.z, A.w);
            jz[u] = make_float2(B.x, B.y);
            nmj[u] = make_float2(B.z, B.w);  // -m_j
            Rx[u] = f2(0.f);
            Ry[u] = f2(0.f);
            Rz[u] = f2(0.f);
          }
          // slices that hold no source pair in any lane are skipped (warp-uniform)
          const int nu = (np - base + 31) / 32 < kPL ? (np - base + 31) / 32 : kPL;
          for (int st = 0; st < Gs; ++st) {
            const float2 sx = f2(si.x), sy = f2(si.y), sz = f2(si.z), smi = f2(si.w);
#pragma unroll
            for (int u = 0; u < kPL; ++u) {
              if (u < nu) {
                const float2 dx = __fadd2_rn(sx, jx[u]);
                const float2 dy = __fadd2_rn(sy, jy[u]);
                const float2 dz = __fadd2_rn(sz, jz[u]);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const bool in0 = (r2.x < fit.rc2) && (r2.x > 0.f);
                const bool in1 = (r2.y < fit.rc2) && (r2.y > 0.f);
                if (kCount)
                  n_in += (uint32_t)in0 * (s0[u] != kNoSlot ? 2u : 1u) + (uint32_t)in1 * (s1[u] != kNoSlot ? 2u : 1u);
                const float2 rinv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                const float2 r3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
                float2 g;  // -f_(1)(r): S / r^3 (Gaussian) or 1/r^3 - 5 / (2 R_c^3) + 3 r^2 / (2 R_c^5)
                if constexpr (kSplit == 1) {
                  g = __fadd2_rn(r3, __ffma2_rn(r2, fit.pc1, fit.pc0));
                } else {
                  const float2 tt = __ffma2_rn(r2, rinv, fit.nrmid);
                  float2 qv = fit.c[9];
#pragma unroll
                  for (int j = 8; j >= 0; --j) qv = __ffma2_rn(qv, tt, fit.c[j]);
                  const float2 ea = __fmul2_rn(r2, fit.kexp);
                  g = __fmul2_rn(__fmul2_rn(make_float2(exp2_mufu(ea.x), exp2_mufu(ea.y)), qv), r3);
                }
                g.x = in0 ? g.x : 0.f;
                g.y = in1 ? g.y : 0.f;
                // on the sink: m_j f_(1) d = (-m_j) g d; on the sources: m_i g d
                const float2 fa = __fmul2_rn(g, nmj[u]);
                ax = __ffma2_rn(fa, dx, ax);
                ay = __ffma2_rn(fa, dy, ay);
                az = __ffma2_rn(fa, dz, az);
                const float2 fr = __fmul2_rn(g, smi);
                Rx[u] = __ffma2_rn(fr, dx, Rx[u]);
                Ry[u] = __ffma2_rn(fr, dy, Ry[u]);
                Rz[u] = __ffma2_rn(fr, dz, Rz[u]);
              }
            }
            // the sink and its force move one lane down the group
            si.x = __shfl_sync(0xffffffffu, si.x, src_lane);
            si.y = __shfl_sync(0xffffffffu, si.y, src_lane);
            si.z = __shfl_sync(0xffffffffu, si.z, src_lane);
            si.w = __shfl_sync(0xffffffffu, si.w, src_lane);
            ax.x = __shfl_sync(0xffffffffu, ax.x, src_lane);
            ax.y = __shfl_sync(0xffffffffu, ax.y, src_lane);
            ay.x = __shfl_sync(0xffffffffu, ay.x, src_lane);
            ay.y = __shfl_sync(0xffffffffu, ay.y, src_lane);
            az.x = __shfl_sync(0xffffffffu, az.x, src_lane);
            az.y = __shfl_sync(0xffffffffu, az.y, src_lane);
          }
#pragma unroll
          for (int u = 0; u < kPL; ++u) {
            if (s0[u] != kNoSlot) {
              if (first_chunk) {
                px_part[s0[u]] = Rx[u].x;
                py_part[s0[u]] = Ry[u].x;
                pz_part[s0[u]] = Rz[u].x;
              } else {
                px_part[s0[u]] += Rx[u].x;
                py_part[s0[u]] += Ry[u].x;
                pz_part[s0[u]] += Rz[u].x;
              }
            }
            if (s1[u] != kNoSlot) {
              if (first_chunk) {
                px_part[s1[u]] = Rx[u].y;
                py_part[s1[u]] = Ry[u].y;
                pz_part[s1[u]] = Rz[u].y;
              } else {
                px_part[s1[u]] += Rx[u].y;
                py_part[s1[u]] += Ry[u].y;
                pz_part[s1[u]] += Rz[u].y;
              }
            }
          }
        }
        __syncwarp();  // the evaluation buffer and slots are rewritten by the next fill
      }
      // each group holds every sink's force from its source pairs: add the groups in order
      buf[lane] = make_float4(ax.x + ax.y, ay.x + ay.y, az.x + az.y, 0.f);
      __syncwarp();
      if (lane < cs) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int gq = 0; gq < 32; gq += Gs) {
          const float4 v = buf[gq + lane];
          sx += v.x;
          sy += v.y;
          sz += v.z;
        }
        const uint32_t o = perm[cbase + lane];
        acc_out[o] += G * sx;
        acc_out[n + o] += G * sy;
        acc_out[2 * n + o] += G * sz;
      }
      __syncwarp();  // also orders this chunk's partial writes before the next chunk's additions
    }
  }
  if (kCount) {
    unsigned long long v = n_in;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(ctr + 1, v);
  }
}

// Per list entry: the number of partial slots (the source leaf's particles,
// none for the leaf against itself) and the sort key of the pass-2 grouping
// (the source leaf; nnodes for entries without partials, so they sort last).
__global__ void k_mut_prep(const uint64_t *__restrict__ lst, int64_t ne, const uint2 *__restrict__ range,
                           uint32_t nnodes, uint32_t *__restrict__ cnt, uint64_t *__restrict__ key,
                           uint32_t *__restrict__ val) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne) return;
  const uint64_t e = lst[t];
  const uint32_t a = pair_sink(e), b = pair_src(e);
  const bool self = a == b && pair_shift(e) == 13u;
  cnt[t] = self ? 0u : range[b].y;
  key[t] = self ? (uint64_t)nnodes : (uint64_t)b;
  val[t] = (uint32_t)t;
}

// Work of each sink leaf (its sink chunks times the source particles on its
// list) as a descending sort key, so the heaviest leaves are handed out first
// and the last warps to finish hold light ones.
__global__ void k_leaf_work(const uint32_t *__restrict__ leaves, int64_t nl, const uint2 *__restrict__ range,
                            const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                            const uint64_t *__restrict__ lst, uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const uint32_t a = leaves[t];
  uint64_t w = 0;
  for (uint32_t i = beg[a]; i < end[a]; ++i) w += range[pair_src(lst[i])].y;
  w *= (range[a].y + 31u) / 32u;
  key[t] = (w > 0xffffffffffull ? 0ull : 0xffffffffffull - w);  // 40-bit descending key
  val[t] = a;
}

// Bounds of each source leaf's run in the sorted keys.
__global__ void k_mut_bounds(const uint64_t *__restrict__ key, int64_t ne, uint32_t nnodes,
                             uint32_t *__restrict__ rbeg, uint32_t *__restrict__ rend) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const uint64_t k = key[i];
  if (k >= nnodes) return;
  if (i == 0 || key[i - 1] != k) rbeg[k] = (uint32_t)i;
  if (i == ne - 1 || key[i + 1] != k) rend[k] = (uint32_t)(i + 1);
}

// Pass 2: one warp per leaf B adds the partials of its entries (as a source), in
// the sorted order, to B's accelerations.
__global__ void __launch_bounds__(256) k_p2p_reactions(const uint32_t *__restrict__ leaves, int64_t nl,
                                                       const uint2 *__restrict__ range,
                                                       const uint32_t *__restrict__ rbeg,
                                                       const uint32_t *__restrict__ rend,
                                                       const uint32_t *__restrict__ ents,
                                                       const uint32_t *__restrict__ poff,
                                                       const float *__restrict__ part, uint64_t npart,
                                                       const uint32_t *__restrict__ perm, int64_t n, float G,
                                                       float *__restrict__ acc_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nl; t += nw) {
    const uint32_t b = leaves[t];
    const uint2 rb = range[b];
    const uint32_t lo = rbeg[b], hi = rend[b];
    float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, sx1 = 0.f, sy1 = 0.f, sz1 = 0.f;
    for (uint32_t i0 = lo; i0 < hi; i0 += 32) {
      // the partial offsets of the next 32 entries, one per lane, then broadcast
      uint32_t po = 0;
      if (i0 + lane < hi) po = poff[ents[i0 + lane]];
      const int m = hi - i0 < 32u ? (int)(hi - i0) : 32;
#pragma unroll 4
      for (int j = 0; j < m; ++j) {
        const uint64_t base = __shfl_sync(0xffffffffu, po, j);
        if ((uint32_t)lane < rb.y) {
          sx0 += part[base + lane];
          sy0 += part[npart + base + lane];
          sz0 += part[2 * npart + base + lane];
        }
        if ((uint32_t)lane + 32u < rb.y) {
          sx1 += part[base + lane + 32];
          sy1 += part[npart + base + lane + 32];
          sz1 += part[2 * npart + base + lane + 32];
        }
      }
    }
    if (hi > lo) {
      if ((uint32_t)lane < rb.y) {
        const uint32_t o = perm[rb.x + lane];
        acc_out[o] += G * sx0;
        acc_out[n + o] += G * sy0;
        acc_out[2 * n + o] += G * sz0;
      }
      if ((uint32_t)lane + 32u < rb.y) {
        const uint32_t o = perm[rb.x + lane + 32];
        acc_out[o] += G * sx1;
        acc_out[n + o] += G * sy1;
        acc_out[2 * n + o] += G * sz1;
      }
    }
  }
}

}  // namespace

cudaError_t p2p_pass_mutual(Ctx &c, float *acc, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  const int T = 256;
  const int64_t ne = c.np2p;
  const uint32_t nn = (uint32_t)c.nnodes;
  const size_t ne1 = (size_t)(ne > 0 ? ne : 1);
  TRY(ensure(c.mut_cnt, ne1 * 4));
  TRY(ensure(c.mut_poff, ne1 * 4));
  TRY(ensure(c.mut_key, ne1 * 8));
  TRY(ensure(c.mut_key_alt, ne1 * 8));
  TRY(ensure(c.mut_val, ne1 * 4));
  TRY(ensure(c.mut_val_alt, ne1 * 4));
  TRY(ensure(c.mut_bounds, ((size_t)nn + 1) * 8));
  TRY(ensure(c.mut_small, 64));
  uint32_t *rbeg = P<uint32_t>(c.mut_bounds), *rend = rbeg + nn + 1;
  TRY(cudaMemsetAsync(c.mut_bounds.p, 0, ((size_t)nn + 1) * 8, st));
  uint64_t npart = 0;
  if (ne > 0) {
    k_mut_prep<<<blocks_for(ne, T), T, 0, st>>>(P<uint64_t>(c.p2p), ne, P<uint2>(c.range), nn, P<uint32_t>(c.mut_cnt),
                                                P<uint64_t>(c.mut_key), P<uint32_t>(c.mut_val));
    note_launch();
    TRY(cudaGetLastError());
    uint64_t *tot = P<uint64_t>(c.mut_small);
    TRY(scan_u32(P<uint32_t>(c.mut_cnt), P<uint32_t>(c.mut_poff), tot, (size_t)ne, c.tmp, st));
    TRY(cudaMemcpyAsync(&npart, tot, 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (npart >= 0xffffffffull) return cudaErrorInvalidValue;  // 32-bit partial slots
    int bits = 1;
    while (((uint64_t)1 << bits) <= (uint64_t)nn) ++bits;
    bool alt = false;
    TRY(radix_sort_u64(P<uint64_t>(c.mut_key), P<uint32_t>(c.mut_val), P<uint64_t>(c.mut_key_alt),
                       P<uint32_t>(c.mut_val_alt), (size_t)ne, 0, bits, &alt, c.tmp, st));
    if (alt) {
      std::swap(c.mut_key, c.mut_key_alt);
      std::swap(c.mut_val, c.mut_val_alt);
    }
    k_mut_bounds<<<blocks_for(ne, T), T, 0, st>>>(P<uint64_t>(c.mut_key), ne, nn, rbeg, rend);
    note_launch();
    TRY(cudaGetLastError());
  }
  TRY(ensure(c.mut_part, (size_t)(npart > 0 ? npart : 1) * 12));
  // sink leaves in descending order of work (the sort reuses the pass-2 key buffers' alt copies)
  const size_t nl1 = (size_t)c.nleaves;
  TRY(ensure(c.mut_lkey, nl1 * 8 * 2));
  TRY(ensure(c.mut_lval, nl1 * 4 * 2));
  {
    uint64_t *lk = P<uint64_t>(c.mut_lkey);
    uint32_t *lv = P<uint32_t>(c.mut_lval);
    k_leaf_work<<<blocks_for(c.nleaves, T), T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint2>(c.range),
                                                        P<uint32_t>(c.p2p_beg), P<uint32_t>(c.p2p_end),
                                                        P<uint64_t>(c.p2p), lk, lv);
    note_launch();
    TRY(cudaGetLastError());
    bool alt = false;
    TRY(radix_sort_u64(lk, lv, lk + nl1, lv + nl1, nl1, 0, 40, &alt, c.tmp, st));
    c.mut_order = alt ? lv + nl1 : lv;
  }
  int dev = 0, nsm = 0;
  TRY(cudaGetDevice(&dev));
  TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = c.prm.tile_p2p_blocks > 0 ? c.prm.tile_p2p_blocks : 8;
  unsigned g = (unsigned)(nsm * per_sm);
  if ((size_t)g * 8 > (size_t)c.nleaves) g = blocks_for(c.nleaves, 8);
  const bool count = (c.prm.profile & 2) != 0, poly = c.prm.split == 1;
  auto kern = count ? (poly ? k_p2p_mut<true, 1> : k_p2p_mut<true, 0>)
                    : (poly ? k_p2p_mut<false, 1> : k_p2p_mut<false, 0>);
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 3);
  const PairFit2 fit2 = pair_fit2(c);
  const size_t dyn = (size_t)2 * 8 * kCapM * sizeof(float4);
  TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  TRY(cudaMemsetAsync(ctr, 0, 8, st));
  kern<<<g, T, dyn, st>>>(c.mut_order, c.nleaves, P<uint4>(c.cell), P<uint2>(c.range),
                          P<uint32_t>(c.p2p_beg), P<uint32_t>(c.p2p_end), P<uint64_t>(c.p2p), P<uint32_t>(c.mut_poff),
                          P<float4>(c.pm4), P<uint32_t>(c.idx), c.n, (float)c.prm.box, fit2, (float)c.prm.G, acc,
                          P<float>(c.mut_part), npart, ctr);
  note_launch();
  TRY(cudaGetLastError());
  if (npart > 0) {
    unsigned g2 = blocks_for(c.nleaves, 8);
    if (g2 > (unsigned)nsm * 16u) g2 = (unsigned)nsm * 16u;
    k_p2p_reactions<<<g2, T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint2>(c.range), rbeg, rend,
                                       P<uint32_t>(c.mut_val), P<uint32_t>(c.mut_poff), P<float>(c.mut_part), npart,
                                       P<uint32_t>(c.idx), c.n, (float)c.prm.G, acc);
    note_launch();
    TRY(cudaGetLastError());
  }
  return cudaSuccess;
#undef TRY
}

}  // namespace hfmm
