// Cut-off P2P over each sink leaf's P2P list (Sec. 2.1, the pair force
// f_(1)(r) r of Sec. 2.2, kept for 0 < r < R_c), added to the L2P accelerations
// already in the caller's particle order (the un-permute).
//
// One warp per work item: a chunk of up to 32 sinks of a leaf, taken from a
// global work counter in longest-first order (k_lpt_hist / k_lpt_place below).
// The source particles of all leaves on the sink's list are streamed through per-warp
// shared memory in fills of up to kCap particles.  A fill takes the next 32
// list entries (a prefix scan of their particle counts gives each candidate
// its slot, an entry cut at the buffer's end continues in the next fill; each
// entry marks its first slot and the marks are carried forward, so every slot
// knows its entry) and copies the candidates' particles asynchronously
// (cp.async) into a raw buffer;
// the next fill's copies are issued before the current fill is evaluated, so
// their latency hides behind the arithmetic.  Once a fill has landed it is
// transformed into the evaluation buffer: moved into the sink leaf's frame (the
// leaf-centre difference is an exact integer in half units), negated, and kept
// only if within R_c of the bounding box of the chunk's sinks (a margin of
// 2^-12 in r^2 keeps every source whose FP32 pair distance could come out
// below R_c; the others contribute nothing).  Lanes are split as (sink i,
// stream s): with cs sinks in the chunk, S = 32 / cs streams walk the buffer,
// so small leaves still keep the warp busy; the streams are added in a fixed
// order at the end (deterministic).  Chunks of 11, 12 or 17..20 sinks, where
// S = 32 / cs leaves many lanes idle, are split in two halves instead: each lane
// holds one sink of each half and evaluates both against every staged source
// pair, which doubles the streams.
//
// The evaluation buffer holds sources in pairs, {-x0, -x1, -y0, -y1}
// {-z0, -z1, -w0, -w1} (w = mass), so each lane evaluates two pairs per step
// with the packed FP32x2 add / multiply / fma of sm_100+ (half the FP32
// instructions; rsqrt and exp2 stay per element).  An odd tail is padded with a
// massless source far outside the cut-off.
//
// Pair force (Gaussian split): a = -m S(x) r / r^3, S(x) = erfc(x/2) + x e^(-x^2/4) / sqrt(pi),
// x = r / r_s, evaluated as S = exp2(-x^2 log2(e) / 4) * Q(r) with Q a degree-9
// polynomial interpolating e^(x^2/4) erfc(x/2) + x / sqrt(pi) at Chebyshev
// nodes on [0, R_c], expanded in powers of u = r - R_c / 2 (coefficients from
// the host, fit_pair_factor()).
#include "p2p_common.cuh"

namespace hfmm {
namespace {


// kCap: source particles per fill (even); dynamic shared memory: 2 x 8 x kCap float4.
// kSplit 0: the Gaussian truncation S(x) above; 1: the polynomial truncation of
// Sec. 5, a = -m (1/r^3 - 5 / (2 R_c^3) + 3 r^2 / (2 R_c^5)) r, no exp2 and no
// fitted factor (see hfmm_params.split).
template <bool kCount, int kCap, int kSplit>
__global__ void __launch_bounds__(256, 2) k_p2p(const uint32_t *__restrict__ items,
                                                const uint4 *__restrict__ cell, const uint2 *__restrict__ range,
                                                const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                                                const uint64_t *__restrict__ lst, const float4 *__restrict__ pm4,
                                                const uint32_t *__restrict__ perm, int64_t n, float box, PairFit2 fit,
                                                float G, float *__restrict__ acc_out,
                                                unsigned long long *__restrict__ ctr, const unsigned *__restrict__ n_items) {
  extern __shared__ float4 p2p_smem[];
  const int64_t nl = *n_items;  // work items: a leaf's chunk of up to 32 sinks (leaf index, chunk in bit 31)
  // per warp: the 32 list entries of the pending fill (first particle, exclusive
  // candidate offset, leaf-centre offset in the sink's frame), each candidate's
  // entry, and the chunk's sink bounding box (lo xyz, hi xyz)
  __shared__ uint32_t e_src[8][32], e_excl[8][32];
  __shared__ float4 e_off[8][32];  // per entry: leaf-centre offset (x, y, z, unused)
  __shared__ uint8_t e_own[8][kCap];
  __shared__ float e_box[8][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float4 *raw = p2p_smem + wid * kCap;            // the pending fill, as copied
  float4 *buf = p2p_smem + (8 + wid) * kCap;      // the fill being evaluated, in pairs
  float *bf = reinterpret_cast<float *>(buf);
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);
  // cull threshold: R_c^2 (1 + 2^-12), far above the FP32 rounding of either distance
  const float rc2_cull = fit.rc2 * (1.f + 1.f / 4096.f);
  const float half_unit = box / (float)kHalfBox;
  uint32_t n_in = 0;  // pairs inside the cut-off (profile mode only)
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= nl) break;
    const uint32_t item = items[t], k = item & 0x7fffffffu;
    const uint4 ca = cell[k];
    const uint2 r = range[k];
    const uint32_t tb = beg[k], te = end[k];
    if (tb == te) continue;  // no sources (in sink batches: a leaf of another batch)

    // the entry window at q + lane, prefetched in two steps: the list word
    // (fetch_lst, while the previous fill is evaluated), then the source leaf's
    // particle range and cell (fetch_src, while the pending fill lands)
    uint64_t pf_e = 0;
    uint2 pf_rb = make_uint2(0u, 0u);
    uint4 pf_cb = make_uint4(0u, 0u, 0u, 0u);
    auto fetch_lst = [&](uint32_t q) {
      if (q + lane < te) pf_e = lst[q + lane];
    };
    auto fetch_src = [&](uint32_t q) {
      if (q + lane < te) {
        const uint32_t b = pair_src(pf_e);
        pf_rb = range[b];
        pf_cb = cell[b];
      }
    };

    // issue the fill starting at list entry q (the first jq particles of that
    // entry already taken; its window prefetched): tables, async copies;
    // advances (q, jq) and starts fetching the next window; returns the number
    // of candidates
    auto issue = [&](uint32_t &q, uint32_t &jq) -> uint32_t {
      const uint32_t qi = q + lane;
      const bool valid = qi < te;
      uint32_t cnt = 0, first = 0;
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
      e_excl[wid][lane] = excl;  // non-decreasing in the lane index
      e_off[wid][lane] = make_float4(dx, dy, dz, 0.f);
      const uint32_t all = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t tot = all < (uint32_t)kCap ? all : (uint32_t)kCap;
      // candidate p belongs to the last entry whose offset is <= p: each
      // non-empty entry marks its first slot, and the marks are carried forward
      // (kPer slots per lane, then a prefix maximum over the lanes: the entries'
      // offsets increase with the lane)
      constexpr int kPer = kCap / 32;
      uint8_t *own_row = e_own[wid];
#pragma unroll
      for (int i = 0; i < kPer; ++i) own_row[lane * kPer + i] = 0xffu;
      __syncwarp();
      if (avail > 0 && excl < tot) own_row[excl] = (uint8_t)lane;
      __syncwarp();
      {
        uint8_t b[kPer];
        int lastm = -1;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          b[i] = own_row[lane * kPer + i];
          if (b[i] != 0xffu) lastm = b[i];
        }
        int pm = lastm;  // inclusive prefix maximum over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, pm, o);
          if (lane >= o && y > pm) pm = y;
        }
        int cur = __shfl_up_sync(0xffffffffu, pm, 1);  // the mark carried in from the lanes before
        if (lane == 0) cur = -1;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          if (b[i] != 0xffu) cur = b[i];
          b[i] = (uint8_t)cur;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kPer; ++i) own_row[lane * kPer + i] = b[i];
      }
      __syncwarp();
      // the copies, four candidates per lane per step
      for (uint32_t pb = 0; pb < tot; pb += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t p = pb + lane + 32 * u;
          if (p < tot) {
            const int o = own_row[p];
            const uint32_t idx = e_src[wid][o] + (p - e_excl[wid][o]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(raw_s + 16u * p), "l"(pm4 + idx)
                         : "memory");
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      // entries taken whole; an entry cut at the buffer's end continues next time
      const unsigned full = __ballot_sync(0xffffffffu, valid && incl <= (uint32_t)kCap);
      const int nfull = __popc(full);
      const uint32_t pex = __shfl_sync(0xffffffffu, excl, nfull & 31);
      const uint32_t pstart = nfull == 0 ? jq : 0u;
      const bool partial = nfull < 32 && q + nfull < te;
      jq = partial ? pstart + (pex < (uint32_t)kCap ? (uint32_t)kCap - pex : 0u) : 0u;
      q += nfull;
      fetch_lst(q);
      return tot;
    };

    const uint32_t cfirst = r.x + 32u * (item >> 31), cend = min(cfirst + 32u, r.x + r.y);
    for (uint32_t cbase = cfirst; cbase < cend; cbase += 32) {
      const uint32_t rem = r.x + r.y - cbase;
      const int cs = rem < 32 ? (int)rem : 32;
      // two sinks per lane (one from each half of the chunk) where that doubles the
      // streams: cs in {11, 12, 17..20}; otherwise one sink per lane
      const int c2 = (cs + 1) >> 1;
      const bool two = 2 * (32 / cs) < 32 / c2;
      const int cl = two ? c2 : cs;  // sinks per lane group
      const int S = 32 / cl, stream = lane / cl, il = lane % cl;
      const bool active = stream < S;
      const float4 xi = pm4[cbase + il];
      const bool hasb = two && il + c2 < cs;
      const float4 xib = hasb ? pm4[cbase + il + c2] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
      const float2 xx = f2(xi.x), xy = f2(xi.y), xz = f2(xi.z);
      const float2 bxx = f2(xib.x), bxy = f2(xib.y), bxz = f2(xib.z);
      {
        float lo0 = xi.x, lo1 = xi.y, lo2 = xi.z, hi0 = xi.x, hi1 = xi.y, hi2 = xi.z;
        if (hasb) {
          lo0 = fminf(lo0, xib.x);
          lo1 = fminf(lo1, xib.y);
          lo2 = fminf(lo2, xib.z);
          hi0 = fmaxf(hi0, xib.x);
          hi1 = fmaxf(hi1, xib.y);
          hi2 = fmaxf(hi2, xib.z);
        }
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
      float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);
      float2 bx = f2(0.f), by = f2(0.f), bz = f2(0.f);
      uint32_t q = tb, jq = 0;
      bool pending = q < te;
      fetch_lst(q);
      fetch_src(q);
      uint32_t tot = pending ? issue(q, jq) : 0u;
      while (pending) {
        fetch_src(q);
        // the pending fill has landed: into the sink's frame, cull, pair up
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        uint32_t kept = 0;
        {
          const float bx0 = e_box[wid][0], by0 = e_box[wid][1], bz0 = e_box[wid][2];
          const float bx1 = e_box[wid][3], by1 = e_box[wid][4], bz1 = e_box[wid][5];
          // four candidates per lane per step (independent chains), kept in
          // candidate order
          for (uint32_t pb = 0; pb < tot; pb += 128) {
            float4 v[4];
            int o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t p = pb + lane + 32 * u;
              const uint32_t pc = p < tot ? p : 0u;
              v[u] = raw[pc];
              o[u] = e_own[wid][pc];
            }
            bool keep[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 d = e_off[wid][o[u]];
              v[u].x += d.x;
              v[u].y += d.y;
              v[u].z += d.z;
              const float gx = fmaxf(fmaxf(bx0 - v[u].x, v[u].x - bx1), 0.f);
              const float gy = fmaxf(fmaxf(by0 - v[u].y, v[u].y - by1), 0.f);
              const float gz = fmaxf(fmaxf(bz0 - v[u].z, v[u].z - bz1), 0.f);
              keep[u] = pb + lane + 32 * u < tot && gx * gx + gy * gy + gz * gz <= rc2_cull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned kb = __ballot_sync(0xffffffffu, keep[u]);
              if (keep[u]) {
                const uint32_t slot = kept + (uint32_t)__popc(kb & ((1u << lane) - 1u));
                float *a = bf + (slot >> 1) * 8 + (slot & 1);  // pair slot/2: {x0 x1 y0 y1} {z0 z1 w0 w1}
                a[0] = -v[u].x;
                a[2] = -v[u].y;
                a[4] = -v[u].z;
                a[6] = -v[u].w;
              }
              kept += (uint32_t)__popc(kb);
            }
          }
        }
        if ((kept & 1) && lane == 0) {  // pad: massless, far beyond the cut-off
          float *a = bf + (kept >> 1) * 8 + 1;
          a[0] = -1e18f;
          a[2] = -1e18f;
          a[4] = -1e18f;
          a[6] = 0.f;
        }
        __syncwarp();  // the raw buffer and the entry tables are free again
        pending = q < te;
        if (pending) tot = issue(q, jq);  // in flight during the evaluation below
        // the pair force of two staged sources on one sink, added to (sx, sy, sz)
        auto pair2 = [&](float2 px, float2 py, float2 pz, const float4 &A, const float4 &B, float2 &sx, float2 &sy,
                         float2 &sz) {
          const float2 dx = __fadd2_rn(px, make_float2(A.x, A.y));
          const float2 dy = __fadd2_rn(py, make_float2(A.z, A.w));
          const float2 dz = __fadd2_rn(pz, make_float2(B.x, B.y));
          const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          const bool in0 = (r2.x < fit.rc2) && (r2.x > 0.f);
          const bool in1 = (r2.y < fit.rc2) && (r2.y > 0.f);
          if (kCount) n_in += (uint32_t)in0 + (uint32_t)in1;
          // outside (0, R_c) the values below may be inf/NaN; the selects discard them
          const float2 rinv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
          const float2 r3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
          float2 f;
          if constexpr (kSplit == 1) {
            // -m (1/r^3 - 5 / (2 R_c^3) + 3 r^2 / (2 R_c^5))
            f = __fmul2_rn(__fadd2_rn(r3, __ffma2_rn(r2, fit.pc1, fit.pc0)), make_float2(B.z, B.w));
          } else {
            const float2 tt = __ffma2_rn(r2, rinv, fit.nrmid);  // u = r - R_c / 2
            float2 qv = fit.c[9];
#pragma unroll
            for (int j = 8; j >= 0; --j) qv = __ffma2_rn(qv, tt, fit.c[j]);
            const float2 ea = __fmul2_rn(r2, fit.kexp);
            const float2 sfac = __fmul2_rn(make_float2(exp2_mufu(ea.x), exp2_mufu(ea.y)), qv);
            f = __fmul2_rn(__fmul2_rn(sfac, r3), make_float2(B.z, B.w));  // -S m / r^3
          }
          f.x = in0 ? f.x : 0.f;
          f.y = in1 ? f.y : 0.f;
          sx = __ffma2_rn(f, dx, sx);
          sy = __ffma2_rn(f, dy, sy);
          sz = __ffma2_rn(f, dz, sz);
        };
        if (active) {
          const int np = (int)((kept + 1) >> 1);
          if (two) {
#pragma unroll 4
            for (int kk = stream; kk < np; kk += S) {
              const float4 A = buf[2 * kk], B = buf[2 * kk + 1];
              pair2(xx, xy, xz, A, B, ax, ay, az);
              pair2(bxx, bxy, bxz, A, B, bx, by, bz);
            }
          } else {
#pragma unroll 8
            for (int kk = stream; kk < np; kk += S) {
              const float4 A = buf[2 * kk], B = buf[2 * kk + 1];
              pair2(xx, xy, xz, A, B, ax, ay, az);
            }
          }
        }
        __syncwarp();  // the evaluation buffer is rewritten by the next fill
      }
      // add the streams of each sink in a fixed order
      buf[lane] = make_float4(ax.x + ax.y, ay.x + ay.y, az.x + az.y, 0.f);
      buf[32 + lane] = make_float4(bx.x + bx.y, by.x + by.y, bz.x + bz.y, 0.f);
      __syncwarp();
      if (lane < cs) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        const int i0 = lane < cl ? lane : 32 + lane - cl;  // the sink's slot in the first group
        for (int s = 0; s < S; ++s) {
          const float4 v = buf[i0 + s * cl];
          sx += v.x;
          sy += v.y;
          sz += v.z;
        }
        const uint32_t o = perm[cbase + lane];
        acc_out[o] += G * sx;
        acc_out[n + o] += G * sy;
        acc_out[2 * n + o] += G * sz;
      }
      __syncwarp();
    }
  }
  if (kCount) {
    unsigned long long v = n_in;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(ctr + 1, v);
  }
}

// Longest-first order of the work (list scheduling: the persistent grid takes
// items in this order).  An item is one chunk of up to 32 sinks of a leaf
// (leaves of 33..64 particles give two, so the heaviest leaves' work is split
// between two warps; the chunks' sums are independent, so the forces do not
// change).  An item's work is about the leaf's list entries times its sinks;
// items are bucketed by the binary order of magnitude of that (coarse buckets
// already give the longest-first schedule its bound, the heaviest single item)
// and placed bucket by bucket, heaviest first.  Leaves with empty lists (other
// sink batches) give no item.  The order within a bucket does not matter: each
// item's sums are its own warp's.
constexpr int kLptBuckets = 64;

__global__ void k_lpt_hist(const uint32_t *__restrict__ leaves, int64_t nl, const uint2 *__restrict__ range,
                           const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                           uint8_t *__restrict__ bucket, unsigned *__restrict__ hist, unsigned *__restrict__ n_items,
                           const TreeState *tz) {
  __shared__ unsigned h[kLptBuckets];
  for (int i = threadIdx.x; i < kLptBuckets; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  nl = tree_leaves(tz, nl);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nl) {
    const uint32_t a = leaves[t];
    const uint32_t ent = end[a] - beg[a], cnt = range[a].y;
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c) {
      uint8_t b = 0xff;
      if (ent > 0 && 32u * c < cnt) {
        const uint32_t cs = min(32u, cnt - 32u * c);
        b = (uint8_t)__clzll((unsigned long long)ent * cs);  // heavier: smaller bucket index
        atomicAdd(&h[b], 1u);
      }
      bucket[2 * t + c] = b;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kLptBuckets; i += blockDim.x)
    if (h[i]) {
      atomicAdd(&hist[i], h[i]);
      atomicAdd(n_items, h[i]);
    }
}

// Ranks within a block from shared-memory counters, one global reservation per
// (block, bucket): the few heavy buckets take few global atomics.
__global__ void k_lpt_place(const uint32_t *__restrict__ leaves, int64_t nl, const uint8_t *__restrict__ bucket,
                            const unsigned *__restrict__ hist, unsigned *__restrict__ cursor,
                            uint32_t *__restrict__ order, const TreeState *tz) {
  __shared__ unsigned base[kLptBuckets], cnt[kLptBuckets];
  for (int i = threadIdx.x; i < kLptBuckets; i += blockDim.x) cnt[i] = 0u;
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int i = 0; i < kLptBuckets; ++i) {
      base[i] = run;
      run += hist[i];
    }
  }
  __syncthreads();
  nl = tree_leaves(tz, nl);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < nl;
  uint8_t b[2] = {0xff, 0xff};
  unsigned local[2] = {0u, 0u};
  if (valid) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      b[c] = bucket[2 * t + c];
      if (b[c] != 0xff) local[c] = atomicAdd(&cnt[b[c]], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kLptBuckets; i += blockDim.x)
    if (cnt[i]) base[i] += atomicAdd(&cursor[i], cnt[i]);
  __syncthreads();
  if (valid) {
    const uint32_t a = leaves[t];
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (b[c] != 0xff) order[base[b[c]] + local[c]] = a | ((uint32_t)c << 31);
  }
}

}  // namespace

cudaError_t p2p_pass(Ctx &c, float *acc, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  const int T = 256;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int per_sm = c.prm.tile_p2p_blocks > 0 ? c.prm.tile_p2p_blocks : 8;
  unsigned g = (unsigned)(nsm * per_sm);
  if ((size_t)g * 8 > (size_t)c.nleaves) g = blocks_for(c.nleaves, 8);
  const bool small = c.prm.tile_p2p_stage == 128, count = (c.prm.profile & 2) != 0;
  auto kern = c.prm.split == 1
                  ? (count ? (small ? k_p2p<true, 128, 1> : k_p2p<true, 256, 1>)
                           : (small ? k_p2p<false, 128, 1> : k_p2p<false, 256, 1>))
                  : (count ? (small ? k_p2p<true, 128, 0> : k_p2p<true, 256, 0>)
                           : (small ? k_p2p<false, 128, 0> : k_p2p<false, 256, 0>));
  // d_small[3] = work counter, d_small[4] = in-cut-off pair count (zeroed earlier when profiling)
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 3);
  const PairFit2 fit2 = pair_fit2(c);  // the context's fit as packed operand pairs
  // two buffers (raw copies, evaluation pairs) of kCap float4 per warp
  const size_t dyn = (size_t)2 * 8 * (small ? 128 : 256) * sizeof(float4);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 8, st);
  if (e != cudaSuccess) return e;
  // the leaves longest first
  const TreeState *tz = c.graph_tree ? P<TreeState>(c.tstate) : nullptr;
  if ((e = ensure(c.lpt_order, (size_t)c.nleaves * 8)) != cudaSuccess) return e;
  if ((e = ensure(c.lpt_tmp, (size_t)c.nleaves * 2 + (2 * kLptBuckets + 4) * sizeof(unsigned) + 64)) != cudaSuccess)
    return e;
  unsigned *hist = P<unsigned>(c.lpt_tmp), *cursor = hist + kLptBuckets, *n_items = cursor + kLptBuckets;
  uint8_t *bucket = reinterpret_cast<uint8_t *>(n_items + 4);
  if ((e = cudaMemsetAsync(hist, 0, (2 * kLptBuckets + 4) * sizeof(unsigned), st)) != cudaSuccess) return e;
  if (c.prm.leaf_max > 64) return cudaErrorInvalidValue;  // two chunks per leaf at most
  k_lpt_hist<<<blocks_for(c.nleaves, T), T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint2>(c.range),
                                                      P<uint32_t>(c.p2p_beg), P<uint32_t>(c.p2p_end), bucket, hist,
                                                      n_items, tz);
  k_lpt_place<<<blocks_for(c.nleaves, T), T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, bucket, hist, cursor,
                                                       P<uint32_t>(c.lpt_order), tz);
  note_launch(2);
  kern<<<g, T, dyn, st>>>(P<uint32_t>(c.lpt_order), P<uint4>(c.cell), P<uint2>(c.range), P<uint32_t>(c.p2p_beg),
                        P<uint32_t>(c.p2p_end), P<uint64_t>(c.p2p), P<float4>(c.pm4), P<uint32_t>(c.idx), c.n,
                        (float)c.prm.box, fit2, (float)c.prm.G, acc, ctr, n_items);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
