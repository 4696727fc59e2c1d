// C ABI of libhfmm (declared in include/hfmm.h): context lifecycle, argument
// checks, error mapping, phase orchestration, statistics and exports.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace hfmm;

namespace {

thread_local std::string g_create_err;

int fail(Ctx &c, int code, const std::string &msg) {
  c.err = msg;
  return code;
}

int cuda_fail(Ctx &c, cudaError_t e, const char *where) {
  int code = e == cudaErrorMemoryAllocation ? HFMM_ERR_OOM : HFMM_ERR_CUDA;
  c.err = std::string(where) + ": " + cudaGetErrorString(e);
  return code;
}

cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

bool valid_params(const hfmm_params &p, std::string &why) {
  if (!(p.box > 0)) return why = "box must be > 0", false;
  if (p.pm_grid < 1) return why = "pm_grid must be >= 1", false;
  if (!(p.rs_cells > 0)) return why = "rs_cells must be > 0", false;
  if (!(p.rcut_rs > 0)) return why = "rcut_rs must be > 0", false;
  if (!(p.theta >= 0) || p.theta > 1.0) return why = "theta must be in [0, 1]", false;
  if (p.order < 1 || p.order > kPMax) return why = "order must be in 1..8", false;
  if (p.leaf_max < 1 || p.leaf_max > 64) return why = "leaf_max must be in 1..64", false;
  if (p.mac_mode != 0 && p.mac_mode != 1) return why = "mac_mode must be 0 (geometric) or 1 (learned)", false;
  if (p.transition_rule != 0 && p.transition_rule != 1) return why = "transition_rule must be 0 or 1", false;
  if (p.size_rule != 0 && p.size_rule != 1) return why = "size_rule must be 0 or 1", false;
  if (p.m2l_precision < 0 || p.m2l_precision > 4) return why = "m2l_precision must be 0..4", false;
  if (p.m2l_precision != 0 && !m2l_tc_supported(p.order))
    return why = "m2l_precision 1..4 (3xTF32 / BF16x3 tensor cores) support orders 1..6", false;
  if (p.profile < 0 || p.profile > 3) return why = "profile must be 0..3", false;
  if (p.m2l_tables != 0 && p.m2l_tables != 1) return why = "m2l_tables must be 0 or 1", false;
  if (p.tile_p2p_stage != 0 && p.tile_p2p_stage != 128 && p.tile_p2p_stage != 256)
    return why = "tile_p2p_stage must be 0, 128 or 256", false;
  if (p.tile_p2p_blocks < 0 || p.tile_p2p_blocks > 8) return why = "tile_p2p_blocks must be in 0..8", false;
  if (p.tile_m2l_blocks < 0 || p.tile_m2l_blocks > 64) return why = "tile_m2l_blocks must be in 0..64", false;
  if (p.tile_trav_blocks < 0 || p.tile_trav_blocks > 4) return why = "tile_trav_blocks must be in 0..4", false;
  if (p.use_graph != 0 && p.use_graph != 1) return why = "use_graph must be 0 or 1", false;
  if (p.list_init < 0) return why = "list_init must be >= 0", false;
  if (p.sink_batches < 0 || p.sink_batches > 4096) return why = "sink_batches must be in 0..4096", false;
  if (p.tc_wait_polls < -1) return why = "tc_wait_polls must be >= -1", false;
  if (p.split != 0 && p.split != 1) return why = "split must be 0 (Gaussian) or 1 (polynomial)", false;
  if (p.split == 1 && (p.mac_mode != 0 || p.m2l_precision != 0 || p.m2l_tables != 0))
    return why = "split 1 needs mac_mode 0, m2l_precision 0 and m2l_tables 0", false;
  if (p.p2p_mutual != 0 && p.p2p_mutual != 1) return why = "p2p_mutual must be 0 or 1", false;
  if (p.p2p_mutual == 1 && (p.mac_mode != 0 || p.size_rule != 1))
    return why = "p2p_mutual 1 needs mac_mode 0 and size_rule 1", false;
  if (p.tree != 0 && p.tree != 1) return why = "tree must be 0 (Morton octree) or 1 (ORB / k-d tree)", false;
  if (p.tree == 1 && (p.mac_mode != 0 || p.m2l_precision != 0 || p.m2l_tables != 0 || p.p2p_mutual != 0 ||
                      p.order > 6))
    return why = "tree 1 needs mac_mode 0, m2l_precision 0, m2l_tables 0, p2p_mutual 0 and order <= 6", false;
  double rs = p.rs_cells * (p.box / (double)p.pm_grid);
  double rc = p.rcut_rs * rs;
  if (!(rc < 0.5 * p.box)) return why = "cut-off radius must be below half the box", false;
  return true;
}

}  // namespace

namespace hfmm {

// Integer forms of the acceptance tests (see Ctx::rc2i and Ctx::acc_thr).  The
// squared distances the traversal forms stay below 3 * 2^48, exact in FP64, so
// comparing the integers against these thresholds takes the FP64 decisions.
void mac_integer_thresholds(Ctx &c) {
  c.rc2i = (int64_t)std::floor(c.rc2h);
  const double smax = 3.0 * std::ldexp(1.0, 48);
  for (int l = 0; l <= kDepth; ++l) {
    const double w = std::ldexp(1.0, 44 - 2 * l);  // 4 w_l^2
    int64_t t = INT64_MAX;
    if (c.theta2 > 0 && w / c.theta2 < smax) {
      double x = std::ceil(w / c.theta2);
      // fl(theta2 * x) is non-decreasing in x: walk to the least x with fl(theta2 * x) >= w
      while (x > 0 && c.theta2 * (x - 1) >= w) x -= 1;
      while (c.theta2 * x < w) x += 1;
      t = (int64_t)x;
    }
    c.acc_thr[l] = t;
  }
}

PairFit fit_pair_factor(double rs, double rc) {
  constexpr int N = 10;
  const double pi = 3.14159265358979323846;
  const double xc = rc / rs;
  double fk[N], cj[N], T[N + 1][N], mono[N];
  for (int k = 0; k < N; ++k) {
    double t = 0.5 * (1.0 + std::cos(pi * (k + 0.5) / N));
    double x = xc * t;
    fk[k] = std::exp(0.25 * x * x) * std::erfc(0.5 * x) + x / std::sqrt(pi);
  }
  for (int j = 0; j < N; ++j) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += fk[k] * std::cos(pi * j * (k + 0.5) / N);
    cj[j] = (j == 0 ? 1.0 : 2.0) * s / N;
  }
  // T_j(s) as monomial coefficients in s = 2r / R_c - 1 (the interval's midpoint at 0)
  std::memset(T, 0, sizeof(T));
  T[0][0] = 1.0;
  T[1][1] = 1.0;
  for (int j = 1; j + 1 < N; ++j)
    for (int i = 0; i < N; ++i) T[j + 1][i] = (i ? 2.0 * T[j][i - 1] : 0.0) - T[j - 1][i];
  for (int i = 0; i < N; ++i) {
    mono[i] = 0.0;
    for (int j = 0; j < N; ++j) mono[i] += cj[j] * T[j][i];
  }
  // in powers of u = r - R_c / 2 (s = u * 2 / R_c): small coefficients, a well-conditioned Horner sum
  PairFit f;
  double sc = 1.0;
  for (int i = 0; i < N; ++i, sc *= 2.0 / rc) f.c[i] = (float)(mono[i] * sc);
  f.rmid = (float)(0.5 * rc);
  f.rc2 = (float)(rc * rc);
  f.kexp = (float)(-1.4426950408889634 / (4.0 * rs * rs));
  return f;
}

}  // namespace hfmm

namespace {

// Every device buffer of the context (the PM buffers apart).
template <class F>
void for_each_buffer(Ctx &c, F f) {
  DBuf *bufs[] = {&c.key, &c.key_alt, &c.idx, &c.idx_alt, &c.xs, &c.pm4, &c.perm, &c.cell, &c.range, &c.kids,
                  &c.leaves, &c.bounds, &c.nkids, &c.koff, &c.front, &c.front_next, &c.cls, &c.counts, &c.offs,
                  &c.m2l, &c.m2l_alt, &c.p2p, &c.p2p_alt, &c.m2l_beg, &c.m2l_end, &c.p2p_beg, &c.p2p_end, &c.M,
                  &c.L, &c.tmp, &c.tmp2, &c.d_small, &c.hpos, &c.hmass, &c.hacc, &c.m2l_mid, &c.tab,
                  &c.mlp_w, &c.cand, &c.mlp_scratch, &c.fseg, &c.fseg_next, &c.seg_a, &c.seg_b, &c.acc_a,
                  &c.acc_b, &c.segbase, &c.btot2, &c.rm_key, &c.rm_beg, &c.rm_cnt, &c.rp_key, &c.rp_beg,
                  &c.rp_cnt, &c.segpre, &c.ctot, &c.tstate, &c.rm_rank, &c.rp_rank, &c.rcnt_m, &c.rcnt_p,
                  &c.mut_cnt, &c.mut_poff, &c.mut_key, &c.mut_key_alt, &c.mut_val, &c.mut_val_alt,
                  &c.mut_bounds, &c.mut_small, &c.mut_part, &c.mut_lkey, &c.mut_lval, &c.lo_flag,
                  &c.lo_rank, &c.lo_meta, &c.lo_sink, &c.lo_tcnt, &c.lo_toff, &c.lo_scr,
                  &c.pacc, &c.tf_pairs, &c.tf_segs, &c.tf_sst, &c.lpt_order, &c.lpt_tmp, &c.kd.xw,
                  &c.kd.ord[0], &c.kd.ord[1], &c.kd.ord[2], &c.kd.ord2[0], &c.kd.ord2[1], &c.kd.ord2[2],
                  &c.kd.side, &c.kd.flag, &c.kd.scan, &c.kd.pnode, &c.kd.nflag, &c.kd.nscan, &c.kd.first,
                  &c.kd.count, &c.kd.child, &c.kd.parent, &c.kd.axis, &c.kd.box, &c.kd.geo, &c.kd.geof, &c.kd.hs,
                  &c.kd.ctr, &c.kd.lv};
  for (DBuf *b : bufs) f(*b);
}

}  // namespace

extern "C" {

void hfmm_default_params(hfmm_params *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->box = 1.0;
  o->pm_grid = 32;
  o->rs_cells = 1.25;
  o->rcut_rs = 4.5;
  o->G = 1.0;
  o->theta = 0.5;
  o->order = 4;
  o->leaf_max = 16;
  o->mac_mode = 0;
  o->transition_rule = 1;
  o->size_rule = 1;
  o->m2l_precision = 0;
  o->profile = 0;
  o->m2l_tables = 0;
}

int hfmm_create(const hfmm_params *params, hfmm_ctx **out) {
  if (!params || !out) {
    g_create_err = "null argument";
    return HFMM_ERR_ARG;
  }
  *out = nullptr;
  std::string why;
  if (!valid_params(*params, why)) {
    g_create_err = why;
    return HFMM_ERR_ARG;
  }
  hfmm_ctx *h = new (std::nothrow) hfmm_ctx();
  if (!h) {
    g_create_err = "host allocation failed";
    return HFMM_ERR_OOM;
  }
  Ctx &c = h->c;
  c.prm = *params;
  c.rs = params->rs_cells * (params->box / (double)params->pm_grid);
  c.rc = params->rcut_rs * c.rs;
  double t = c.rc * 4194304.0;
  t = t / params->box;
  c.rc2h = t * t;
  c.theta2 = params->theta * params->theta;
  mac_integer_thresholds(c);
  c.p = params->order;
  c.nc = ncoef(c.p);
  c.ldm = (c.nc + 3) & ~3;
  c.fit = fit_pair_factor(c.rs, c.rc);
  c.tab_k = m2l_table_extent(*params);
  cudaError_t e = cudaMallocHost(&c.h_pinned, 1024);
  if (e == cudaSuccess) e = ensure(c.d_small, 256);
  for (int i = 0; i < 16 && e == cudaSuccess; ++i) e = cudaEventCreate(&c.ev[i]);
  if (e != cudaSuccess) {
    g_create_err = std::string("CUDA: ") + cudaGetErrorString(e);
    hfmm_destroy(h);
    return e == cudaErrorMemoryAllocation ? HFMM_ERR_OOM : HFMM_ERR_CUDA;
  }
  c.ev_ready = true;
  *out = h;
  return HFMM_OK;
}

void hfmm_destroy(hfmm_ctx *h) {
  if (!h) return;
  Ctx &c = h->c;
  for_each_buffer(c, [](DBuf &b) { release(b); });
  pm_release(c);
  if (c.gexec) cudaGraphExecDestroy(c.gexec);
  if (c.gexec_step) cudaGraphExecDestroy(c.gexec_step);
  if (c.gstream) cudaStreamDestroy(c.gstream);
  if (c.gready) cudaEventDestroy(c.gready);
  if (c.h_pinned) cudaFreeHost(c.h_pinned);
  for (int i = 0; i < 16; ++i)
    if (c.ev[i]) cudaEventDestroy(c.ev[i]);
  delete h;
}

const char *hfmm_last_error(const hfmm_ctx *h) {
  if (!h) return g_create_err.c_str();
  return h->c.err.c_str();
}

int hfmm_build_tree(hfmm_ctx *h, const double *pos, const float *mass, int64_t n, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  c.have_tree = false;
  c.last_step_graph = false;
  c.lists_split = false;
  c.last_batches = 1;
  if (n < 0 || n > (int64_t)0x7fffffff) return fail(c, HFMM_ERR_ARG, "n must be in [0, 2^31)");
  if (n > 0 && (!pos || !mass)) return fail(c, HFMM_ERR_ARG, "null position or mass pointer");
  c.mass_ref = mass;
  cudaError_t e = c.prm.tree == 1 ? kd_build_tree(c, pos, mass, n, S(stream)) : build_tree(c, pos, mass, n, S(stream));
  if (e == cudaErrorInvalidValue && c.nnodes >= ((int64_t)1 << kSinkBits))
    return fail(c, HFMM_ERR_CAPACITY, "more than 2^27 tree nodes");
  if (e != cudaSuccess) return cuda_fail(c, e, "build_tree");
  return HFMM_OK;
}

namespace {

// The configurations the graphs cover: FP32 CUDA-core M2L without operator
// tables, the geometric acceptance, one-sided P2P and no pair counting.
bool graph_eligible(const Ctx &c) {
  return c.prm.use_graph && c.prm.tree == 0 && c.prm.m2l_precision == 0 && c.prm.mac_mode == 0 && !(c.prm.profile & 2) &&
         !c.prm.p2p_mutual && !c.prm.m2l_tables && sink_batches_for(c) == 1;
}

// The whole short-range call captured as one CUDA graph on the context's own
// stream and replayed on `st`: upward pass, the walk (its list sizes stay on
// the device: the lists have their capacities from the last call or the first
// guess), list grouping (run counts read on the device), M2L, L2L/L2P and P2P.
// Every buffer is sized before the capture.  After the graph, one read-back
// of the walk's state: *ok is false when a list overflowed (the caller then
// runs the direct path, which grows the lists).  With profiling the graph is
// timed as a whole.
cudaError_t whole_call_graph(Ctx &c, float *acc, cudaStream_t st, bool prof, bool *ok) {
  cudaError_t e;
  *ok = false;
  if (!c.gstream && (e = cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = traverse_graph_prepare(c)) != cudaSuccess) return e;
  if ((e = sort_lists_prepare(c)) != cudaSuccess) return e;
  // during the capture the list sizes are their capacities on the host
  c.nm2l = (int64_t)c.cap_m2l;
  c.np2p = (int64_t)c.cap_p2p;
  c.graph_walk = true;
  std::vector<void *> deferred;
  g_deferred_free = &deferred;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(c.gstream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t r = upward(c, c.gstream);
    if (r == cudaSuccess) r = traverse_graph_launch(c, c.gstream);
    if (r == cudaSuccess) r = sort_lists(c, c.gstream);
    if (r == cudaSuccess) r = m2l_all(c, c.gstream);
    if (r == cudaSuccess) r = downward(c, acc, c.gstream);
    if (r == cudaSuccess) r = p2p_pass(c, acc, c.gstream);
    e = cudaStreamEndCapture(c.gstream, &graph);
    if (r != cudaSuccess) e = r;
  }
  c.graph_walk = false;
  g_deferred_free = nullptr;
  for (void *p : deferred) cudaFree(p);  // allocations replaced during the capture (none expected)
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  if (c.gexec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(c.gexec, graph, &info) == cudaSuccess) {
      ++c.graph_updates;
    } else {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(c.gexec);
      c.gexec = nullptr;
    }
  }
  if (!c.gexec) {
    e = cudaGraphInstantiate(&c.gexec, graph, 0);
    if (e != cudaSuccess) {
      c.gexec = nullptr;
      cudaGraphDestroy(graph);
      return e;
    }
    ++c.graph_instantiations;
  }
  cudaGraphDestroy(graph);
  if (prof) cudaEventRecord(c.ev[3], st);
  e = cudaGraphLaunch(c.gexec, st);  // its kernels were counted as they were captured
  if (prof) cudaEventRecord(c.ev[9], st);
  if (e != cudaSuccess) return e;
  c.last_graph = true;
  return traverse_graph_finish(c, st, ok);
}

}  // namespace

constexpr const char *kWalkLimit = "traversal did not complete within its capacity retries and depth bound";

int hfmm_short_range_forces(hfmm_ctx *h, float *acc, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "short_range_forces before build_tree");
  if (c.prm.mac_mode == 1 && !c.have_mlp) return fail(c, HFMM_ERR_STATE, "learned acceptance without hfmm_load_mlp");
  if (c.n > 0 && !acc) return fail(c, HFMM_ERR_ARG, "null acceleration pointer");
  if (c.n == 0) return HFMM_OK;
  cudaStream_t st = S(stream);
  cudaError_t e;
  size_t eb = (size_t)c.nnodes * c.ldm * sizeof(float);
  if ((e = ensure(c.M, eb)) != cudaSuccess) return cuda_fail(c, e, "alloc M");
  if ((e = ensure(c.L, eb)) != cudaSuccess) return cuda_fail(c, e, "alloc L");
  if ((e = cudaMemsetAsync(c.L.p, 0, eb, st)) != cudaSuccess) return cuda_fail(c, e, "memset L");
  // the padding of each multipole row is read (as part of a float4) but never used: keep it finite
  if (c.ldm != c.nc && (e = cudaMemsetAsync(c.M.p, 0, eb, st)) != cudaSuccess) return cuda_fail(c, e, "memset M");
  bool prof = (c.prm.profile & 1) != 0;
  if ((c.prm.profile & 2) && (e = cudaMemsetAsync(P<uint64_t>(c.d_small) + 4, 0, 8, st)) != cudaSuccess)
    return cuda_fail(c, e, "memset counter");
  c.last_graph = false;
  c.last_batches = 1;
  c.lists_split = false;
  if (c.prm.tree == 1) {
    e = kd_short_range(c, acc, st);
    if (e == cudaErrorInvalidValue) return fail(c, HFMM_ERR_CAPACITY, "an interaction list above 2^32 - 1 entries");
    if (e != cudaSuccess) return cuda_fail(c, e, "k-d short range");
    return HFMM_OK;
  }
  if (const int nbatch = sink_batches_for(c); nbatch > 1) {
    if (prof) cudaEventRecord(c.ev[3], st);
    if ((e = upward(c, st)) != cudaSuccess) return cuda_fail(c, e, "upward");
    if (prof) cudaEventRecord(c.ev[4], st);
    if (c.prm.m2l_precision != 0 &&
        (e = cudaMemsetAsync(P<uint64_t>(c.d_small) + 6, 0, 8, st)) != cudaSuccess)
      return cuda_fail(c, e, "m2l status");
    e = short_range_batched(c, acc, nbatch, st);
    if (e == cudaErrorInvalidValue) return fail(c, HFMM_ERR_CAPACITY, kWalkLimit);
    if (e != cudaSuccess) return cuda_fail(c, e, "sink batches");
    if (prof) cudaEventRecord(c.ev[9], st);
    if (c.prm.m2l_precision != 0) {
      int *status = reinterpret_cast<int *>(P<uint64_t>(c.d_small) + 6);
      if ((e = cudaMemcpyAsync(c.h_pinned + 31, status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "m2l status");
      if (*reinterpret_cast<int *>(c.h_pinned + 31) != 0)
        return fail(c, HFMM_ERR_TIMEOUT, "tensor-core M2L: a bounded wait for MMA completion gave up");
    }
    return HFMM_OK;
  }
  if (graph_eligible(c)) {
    bool ok = false;
    e = whole_call_graph(c, acc, st, prof, &ok);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph");
    if (ok) {
      if (c.nm2l > (int64_t)UINT32_MAX || c.np2p > (int64_t)UINT32_MAX)
        return fail(c, HFMM_ERR_CAPACITY, "an interaction list above 2^32 - 1 entries");
      return HFMM_OK;
    }
    // a list overflowed inside the graph: start again directly (the walk grows the lists)
    c.last_graph = false;
    if ((e = cudaMemsetAsync(c.L.p, 0, eb, st)) != cudaSuccess) return cuda_fail(c, e, "memset L");
  }
  if (prof) cudaEventRecord(c.ev[3], st);
  if ((e = upward(c, st)) != cudaSuccess) return cuda_fail(c, e, "upward");
  if (prof) cudaEventRecord(c.ev[4], st);
  e = traverse(c, st);
  if (e == cudaErrorInvalidValue) return fail(c, HFMM_ERR_CAPACITY, kWalkLimit);
  if (e != cudaSuccess) return cuda_fail(c, e, "traverse");
  // the sink-grouped lists are addressed through 32-bit CSR bounds
  if (c.nm2l > (int64_t)UINT32_MAX || c.np2p > (int64_t)UINT32_MAX)
    return fail(c, HFMM_ERR_CAPACITY, "an interaction list above 2^32 - 1 entries");
  if (prof) cudaEventRecord(c.ev[5], st);
  if ((e = sort_lists(c, st)) != cudaSuccess) return cuda_fail(c, e, "sort_lists");
  if (prof) cudaEventRecord(c.ev[6], st);
  if (c.prm.m2l_precision != 0 &&
      (e = cudaMemsetAsync(P<uint64_t>(c.d_small) + 6, 0, 8, st)) != cudaSuccess)
    return cuda_fail(c, e, "m2l status");
  if ((e = m2l_all(c, st)) != cudaSuccess) return cuda_fail(c, e, "m2l");
  if (c.prm.m2l_precision != 0 && c.nm2l > 0) {
    int *status = reinterpret_cast<int *>(P<uint64_t>(c.d_small) + 6);
    if ((e = cudaMemcpyAsync(c.h_pinned + 31, status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(c, e, "m2l status");
    if (*reinterpret_cast<int *>(c.h_pinned + 31) != 0)
      return fail(c, HFMM_ERR_TIMEOUT, "tensor-core M2L: a bounded wait for MMA completion gave up");
  }
  if (prof) cudaEventRecord(c.ev[7], st);
  if ((e = downward(c, acc, st)) != cudaSuccess) return cuda_fail(c, e, "l2l/l2p");
  if (prof) cudaEventRecord(c.ev[8], st);
  e = c.prm.p2p_mutual ? p2p_pass_mutual(c, acc, st) : p2p_pass(c, acc, st);
  if (e == cudaErrorInvalidValue && c.prm.p2p_mutual)
    return fail(c, HFMM_ERR_CAPACITY, "mutual P2P: more than 2^32 - 1 partial sums");
  if (e != cudaSuccess) return cuda_fail(c, e, "p2p");
  if (prof) cudaEventRecord(c.ev[9], st);
  return HFMM_OK;
}

int hfmm_pm_long_range(hfmm_ctx *h, float *acc, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "pm_long_range before build_tree");
  if (c.n > 0 && !acc) return fail(c, HFMM_ERR_ARG, "null acceleration pointer");
  if (c.prm.pm_grid < 2 || c.prm.pm_grid > 1024) return fail(c, HFMM_ERR_ARG, "pm_grid must be in 2..1024");
  cudaError_t e = pm_long_range(c, acc, S(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "pm_long_range");
  return HFMM_OK;
}

namespace {

// What a captured step depends on besides the parameters (fixed for the
// context): every buffer address, the capacities, the arguments.  Equal
// signatures before a step and after the last capture: the graph is replayed
// as it is (each host-side swap of ping-pong buffers made during the capture
// is part of the state it left).
std::vector<uint64_t> step_signature(Ctx &c, const double *pos, const float *vel, const float *acc, double dt) {
  std::vector<uint64_t> v;
  v.reserve(192);
  for_each_buffer(c, [&](DBuf &b) {
    v.push_back((uint64_t)(uintptr_t)b.p);
    v.push_back((uint64_t)b.cap);
  });
  DBuf *pmb[] = {&c.pm_q, &c.pm_rho, &c.pm_mk, &c.pm_ak, &c.pm_a, &c.pm_gtab};
  for (DBuf *b : pmb) v.push_back((uint64_t)(uintptr_t)b->p);
  uint64_t dtb;
  std::memcpy(&dtb, &dt, 8);
  const uint64_t rest[] = {(uint64_t)c.n, c.cap_nodes, (uint64_t)c.cap_levels, c.cap_front, c.cap_m2l, c.cap_p2p,
                           c.cap_seg, c.cap_run, (uint64_t)c.pm_plan_r2c, (uint64_t)c.pm_plan_c2r,
                           (uint64_t)(uintptr_t)pos, (uint64_t)(uintptr_t)vel, (uint64_t)(uintptr_t)acc,
                           (uint64_t)(uintptr_t)c.mass_ref, dtb};
  v.insert(v.end(), rest, rest + sizeof(rest) / sizeof(rest[0]));
  return v;
}

// The kick-drift-kick step as one CUDA graph (Sec. 4's synchronised step):
// first kick, drift, the octree build (its sizes stay on the device), the
// short-range call (upward pass, walk, list grouping, M2L, L2L/L2P, P2P), the
// PM long range and the second kick.  Kernels after the build read the tree's
// extent from the device state and treat an overflowed tree as empty; the
// second kick runs only when the tree and the walk fitted.  Buffers are sized
// before the capture from the node capacity, the last tree's level count and
// the list capacities, and the graph is captured again only when an address, a
// capacity or an argument changed.  One read-back after the graph: *done is
// false when something overflowed, and the step then continues directly from
// the drifted positions (the first kick and the drift have been applied).
cudaError_t step_graph(Ctx &c, double *pos, float *vel, float *acc, double dt, cudaStream_t st, bool prof,
                       bool *done) {
  cudaError_t e;
  *done = false;
  const int64_t n = c.n;
  if (!c.gstream && (e = cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = build_tree_prepare(c, n)) != cudaSuccess) return e;
  // while the step is captured the tree's sizes on the host are the node capacity
  c.nnodes = c.nleaves = (int64_t)c.cap_nodes;
  const size_t eb = (size_t)c.cap_nodes * c.ldm * sizeof(float);
  if ((e = ensure(c.M, eb)) != cudaSuccess) return e;
  if ((e = ensure(c.L, eb)) != cudaSuccess) return e;
  if ((e = traverse_graph_prepare(c)) != cudaSuccess) return e;
  if ((e = sort_lists_prepare(c)) != cudaSuccess) return e;
  if ((e = pm_prepare(c)) != cudaSuccess) return e;
  std::vector<uint64_t> sig = step_signature(c, pos, vel, acc, dt);
  if (!c.gexec_step || sig != c.step_sig) {
    c.nm2l = (int64_t)c.cap_m2l;
    c.np2p = (int64_t)c.cap_p2p;
    c.graph_walk = c.graph_tree = true;
    std::vector<void *> deferred;
    g_deferred_free = &deferred;
    cudaGraph_t graph = nullptr;
    const long long l0 = g_launches.load();
    cudaStream_t gs = c.gstream;
    e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t r = kick(vel, acc, n, 0.5 * dt, gs);
      if (r == cudaSuccess) r = drift(pos, vel, n, dt, c.prm.box, gs);
      if (r == cudaSuccess) r = build_tree_launch(c, pos, c.mass_ref, n, gs);
      if (r == cudaSuccess) r = cudaMemsetAsync(c.L.p, 0, eb, gs);
      // the padding of each multipole row is read (as part of a float4) but never used: keep it finite
      if (r == cudaSuccess && c.ldm != c.nc) r = cudaMemsetAsync(c.M.p, 0, eb, gs);
      if (r == cudaSuccess) r = upward(c, gs);
      if (r == cudaSuccess) r = traverse_graph_launch(c, gs);
      if (r == cudaSuccess) r = sort_lists(c, gs);
      if (r == cudaSuccess) r = m2l_all(c, gs);
      if (r == cudaSuccess) r = downward(c, acc, gs);
      if (r == cudaSuccess) r = p2p_pass(c, acc, gs);
      if (r == cudaSuccess) r = pm_long_range(c, acc, gs);
      if (r == cudaSuccess) r = kick_guarded(vel, acc, n, 0.5 * dt, step_guard(c), gs);
      e = cudaStreamEndCapture(gs, &graph);
      if (r != cudaSuccess) e = r;
    }
    c.graph_walk = c.graph_tree = false;
    g_deferred_free = nullptr;
    for (void *p : deferred) cudaFree(p);  // allocations replaced during the capture (none expected)
    c.step_kernels = g_launches.load() - l0;
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (c.gexec_step) cudaGraphExecDestroy(c.gexec_step);
      c.gexec_step = nullptr;
      return e;
    }
    if (c.gexec_step) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(c.gexec_step, graph, &info) == cudaSuccess) {
        ++c.graph_updates;
      } else {
        (void)cudaGetLastError();
        cudaGraphExecDestroy(c.gexec_step);
        c.gexec_step = nullptr;
      }
    }
    if (!c.gexec_step) {
      e = cudaGraphInstantiate(&c.gexec_step, graph, 0);
      if (e != cudaSuccess) {
        c.gexec_step = nullptr;
        cudaGraphDestroy(graph);
        return e;
      }
      ++c.graph_instantiations;
    }
    cudaGraphDestroy(graph);
    c.step_sig = step_signature(c, pos, vel, acc, dt);  // the state the capture left
  } else {
    g_launches.fetch_add(c.step_kernels, std::memory_order_relaxed);  // the graph's kernels, counted per replay
  }
  if (prof) cudaEventRecord(c.ev[3], st);
  if ((e = cudaGraphLaunch(c.gexec_step, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c.ev[9], st);
  c.last_graph = c.last_step_graph = true;
  ++c.step_graphs;
  // the tree's state beside the walk's (both land in one synchronisation)
  unsigned char *hp = reinterpret_cast<unsigned char *>(c.h_pinned);
  if ((e = cudaMemcpyAsync(hp + 512, c.tstate.p, sizeof(TreeState), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  bool walk_ok = false;
  if ((e = traverse_graph_finish(c, st, &walk_ok)) != cudaSuccess) return e;
  TreeState ts;
  std::memcpy(&ts, hp + 512, sizeof(TreeState));
  if (!build_tree_finish(c, ts)) {
    c.have_tree = false;
    return cudaSuccess;
  }
  *done = walk_ok;
  return cudaSuccess;
}

}  // namespace

int hfmm_step(hfmm_ctx *h, double *pos, float *vel, float *acc, double dt, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "step before build_tree");
  if (c.n > 0 && (!pos || !vel || !acc || !c.mass_ref)) return fail(c, HFMM_ERR_ARG, "null particle array");
  if (!std::isfinite(dt)) return fail(c, HFMM_ERR_ARG, "dt must be finite");
  if (c.prm.pm_grid < 2 || c.prm.pm_grid > 1024) return fail(c, HFMM_ERR_ARG, "pm_grid must be in 2..1024");
  cudaStream_t st = S(stream);
  const int64_t n = c.n;
  cudaError_t e;
  bool drifted = false;
  // (node indices of the graph's walk are bounded by the node capacity: keep it below the sink field)
  const uint64_t cap_guess = std::max<uint64_t>(c.cap_nodes, (uint64_t)(2 * n / std::max(c.prm.leaf_max, 1) + 64));
  if (graph_eligible(c) && n > 0 && cap_guess < ((uint64_t)1 << kSinkBits)) {
    bool done = false;
    e = step_graph(c, pos, vel, acc, dt, st, (c.prm.profile & 1) != 0, &done);
    if (e != cudaSuccess) {
      c.have_tree = false;  // the host's tree sizes may be the capture's placeholders
      return cuda_fail(c, e, "step graph");
    }
    if (done) {
      if (c.nm2l > (int64_t)UINT32_MAX || c.np2p > (int64_t)UINT32_MAX)
        return fail(c, HFMM_ERR_CAPACITY, "an interaction list above 2^32 - 1 entries");
      return HFMM_OK;
    }
    drifted = true;  // an overflow: the step goes on directly from the drifted positions
    c.last_graph = c.last_step_graph = false;
  }
  if (!drifted) {
    if ((e = kick(vel, acc, n, 0.5 * dt, st)) != cudaSuccess) return cuda_fail(c, e, "kick");
    if ((e = drift(pos, vel, n, dt, c.prm.box, st)) != cudaSuccess) return cuda_fail(c, e, "drift");
  }
  int rc = hfmm_build_tree(h, pos, c.mass_ref, n, stream);
  if (rc != HFMM_OK) return rc;
  if ((rc = hfmm_short_range_forces(h, acc, stream)) != HFMM_OK) return rc;
  if ((rc = hfmm_pm_long_range(h, acc, stream)) != HFMM_OK) return rc;
  if ((e = kick(vel, acc, n, 0.5 * dt, st)) != cudaSuccess) return cuda_fail(c, e, "kick");
  return HFMM_OK;
}

int hfmm_short_range_forces_host(hfmm_ctx *h, const double *pos, const float *mass, int64_t n, float *acc,
                                 void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (n < 0 || n > (int64_t)0x7fffffff) return fail(c, HFMM_ERR_ARG, "n must be in [0, 2^31)");
  if (n > 0 && (!pos || !mass || !acc)) return fail(c, HFMM_ERR_ARG, "null host pointer");
  cudaStream_t st = S(stream);
  cudaError_t e;
  if ((e = ensure(c.hpos, (size_t)(n ? n : 1) * 24)) != cudaSuccess) return cuda_fail(c, e, "alloc pos");
  if ((e = ensure(c.hmass, (size_t)(n ? n : 1) * 4)) != cudaSuccess) return cuda_fail(c, e, "alloc mass");
  if ((e = ensure(c.hacc, (size_t)(n ? n : 1) * 12)) != cudaSuccess) return cuda_fail(c, e, "alloc acc");
  if (n > 0) {
    if ((e = cudaMemcpyAsync(c.hpos.p, pos, n * 24, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(c, e, "copy pos");
    if ((e = cudaMemcpyAsync(c.hmass.p, mass, n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(c, e, "copy mass");
  }
  int rc = hfmm_build_tree(h, P<double>(c.hpos), P<float>(c.hmass), n, stream);
  if (rc != HFMM_OK) return rc;
  rc = hfmm_short_range_forces(h, P<float>(c.hacc), stream);
  if (rc != HFMM_OK) return rc;
  if (n > 0 && (e = cudaMemcpyAsync(acc, c.hacc.p, n * 12, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(c, e, "copy acc");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "synchronize");
  return HFMM_OK;
}

int hfmm_interaction_counts(hfmm_ctx *h, int conventional, int64_t *out, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (!out) return fail(c, HFMM_ERR_ARG, "null output pointer");
  if (conventional != 0 && conventional != 1) return fail(c, HFMM_ERR_ARG, "conventional must be 0 or 1");
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "interaction_counts before build_tree");
  for (int i = 0; i < 4; ++i) out[i] = 0;
  if (c.n == 0) return HFMM_OK;
  cudaStream_t st = S(stream);
  if (c.prm.tree == 1) {
    c.lists_split = false;
    cudaError_t e = kd_interaction_counts(c, conventional != 0, out, st);
    if (e == cudaErrorInvalidValue) return fail(c, HFMM_ERR_CAPACITY, "k-d walk: buffers outgrown 16 times");
    if (e != cudaSuccess) return cuda_fail(c, e, "k-d walk");
    return HFMM_OK;
  }
  c.lists_split = false;
  c.count_walk = conventional ? 2 : 1;
  cudaError_t e = traverse(c, st);
  c.count_walk = 0;
  if (e == cudaErrorInvalidValue) return fail(c, HFMM_ERR_CAPACITY, kWalkLimit);
  if (e != cudaSuccess) return cuda_fail(c, e, "traverse");
  int64_t pp = 0;
  if ((e = p2p_list_particle_pairs(c, st, &pp)) != cudaSuccess) return cuda_fail(c, e, "count pairs");
  out[0] = c.nm2l;
  out[1] = c.np2p;
  out[2] = pp;
  out[3] = c.frontier_items;
  return HFMM_OK;
}

int hfmm_get_stats(hfmm_ctx *h, hfmm_stats *o) {
  if (!h || !o) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  std::memset(o, 0, sizeof(*o));
  o->n = c.n;
  o->nnodes = c.nnodes;
  o->nleaves = c.nleaves;
  o->nlevels = c.nlevels;
  o->traverse_iters = c.traverse_iters;
  o->np2p = c.np2p;
  o->nm2l = c.nm2l;
  o->p2p_particle_pairs = c.p2p_particle_pairs;
  o->nm2l_table = c.nm2l_table;
  o->frontier_pairs = c.frontier_items;
  o->traverse_walks = c.traverse_walks;
  o->step_graphs = c.step_graphs;
  o->graph_captures = c.graph_updates + c.graph_instantiations;
  o->sink_batches = c.last_batches;
  o->p2p_useful_pairs = -1;
  if ((c.prm.profile & 2) && c.n > 0) {
    unsigned long long u = 0;
    if (cudaMemcpy(&u, P<uint64_t>(c.d_small) + 4, 8, cudaMemcpyDeviceToHost) == cudaSuccess)
      o->p2p_useful_pairs = (int64_t)u;
  }
  o->launches = (int64_t)g_launches.load();
  float *t[] = {&o->t_keys_sort, &o->t_tree, &o->t_upward, &o->t_traverse, &o->t_lists, &o->t_m2l, &o->t_l2l,
                &o->t_p2p};
  const int ev_pairs[][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {7, 8}, {8, 9}};
  const int ev_graph[][2] = {{0, 1}, {1, 2}, {3, 9}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
  for (int i = 0; i < 8; ++i) {
    *t[i] = -1.f;
    if (c.last_step_graph && i < 2) continue;  // the build ran inside the step's graph
    if (c.lists_split && i >= 2) {  // sink batches: upward, then everything else as one span
      const int pr[2][2] = {{3, 4}, {4, 9}};
      if (i <= 3 && (c.prm.profile & 1) && c.n > 0) {
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, c.ev[pr[i - 2][0]], c.ev[pr[i - 2][1]]) == cudaSuccess) *t[i] = ms;
      }
      continue;
    }
    if (c.last_graph && ev_graph[i][0] >= 0 && (c.prm.profile & 1) && c.n > 0) {
      float ms = -1.f;
      if (cudaEventElapsedTime(&ms, c.ev[ev_graph[i][0]], c.ev[ev_graph[i][1]]) == cudaSuccess) *t[i] = ms;
      continue;
    }
    if (c.last_graph) continue;
    if ((c.prm.profile & 1) && c.n > 0) {
      float ms = -1.f;
      if (cudaEventElapsedTime(&ms, c.ev[ev_pairs[i][0]], c.ev[ev_pairs[i][1]]) == cudaSuccess) *t[i] = ms;
    }
  }
  cudaGetLastError();
  return HFMM_OK;
}

int hfmm_export(hfmm_ctx *h, int what, void *buf, size_t *bytes) {
  if (!h || !bytes) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "nothing to export before build_tree");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  size_t need = 0;
  if (c.lists_split &&
      (what == HFMM_EXPORT_P2P || what == HFMM_EXPORT_M2L || what == HFMM_EXPORT_M2L_ORDER))
    return fail(c, HFMM_ERR_STATE, "the last call ran in sink batches: its lists were not kept");
  const bool kd = c.prm.tree == 1;
  if (kd && (what == HFMM_EXPORT_KEYS || what == HFMM_EXPORT_NODES))
    return fail(c, HFMM_ERR_ARG, "keys and octree nodes do not exist on the k-d tree (tree 1)");
  if (!kd && (what == HFMM_EXPORT_KD_NODES || what == HFMM_EXPORT_KD_BOXES))
    return fail(c, HFMM_ERR_ARG, "k-d nodes exist with tree 1 only");
  switch (what) {
    case HFMM_EXPORT_KD_NODES: need = c.nnodes * 40; break;
    case HFMM_EXPORT_KD_BOXES: need = c.nnodes * 48; break;
    case HFMM_EXPORT_KEYS: need = c.n * 8; break;
    case HFMM_EXPORT_PERM: need = c.n * 4; break;
    case HFMM_EXPORT_NODES: need = c.nnodes * 64; break;
    case HFMM_EXPORT_P2P: need = c.np2p * 24; break;
    case HFMM_EXPORT_M2L: need = c.nm2l * 24; break;
    case HFMM_EXPORT_MULTIPOLES:
    case HFMM_EXPORT_LOCALS: need = (size_t)c.nnodes * c.nc * 4; break;
    case HFMM_EXPORT_M2L_ORDER: need = c.nm2l * 8; break;
    case HFMM_EXPORT_CANDIDATES: need = c.ncand_last * 24; break;
    default: return fail(c, HFMM_ERR_ARG, "unknown export");
  }
  if (!buf) {
    *bytes = need;
    return HFMM_OK;
  }
  if (*bytes < need) return fail(c, HFMM_ERR_ARG, "export buffer too small");
  *bytes = need;
  if (need == 0) return HFMM_OK;
  switch (what) {
    case HFMM_EXPORT_KEYS: e = cudaMemcpy(buf, c.key.p, need, cudaMemcpyDeviceToHost); break;
    case HFMM_EXPORT_PERM: e = cudaMemcpy(buf, c.idx.p, need, cudaMemcpyDeviceToHost); break;
    case HFMM_EXPORT_MULTIPOLES:
    case HFMM_EXPORT_LOCALS:  // rows of nc values out of the padded device rows
      e = cudaMemcpy2D(buf, c.nc * sizeof(float), (what == HFMM_EXPORT_LOCALS ? c.L : c.M).p, c.ldm * sizeof(float),
                       c.nc * sizeof(float), c.nnodes, cudaMemcpyDeviceToHost);
      break;
    case HFMM_EXPORT_NODES: {
      std::vector<uint4> cell(c.nnodes);
      std::vector<uint2> range(c.nnodes);
      std::vector<int2> kids(c.nnodes);
      e = cudaMemcpy(cell.data(), c.cell.p, c.nnodes * sizeof(uint4), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(range.data(), c.range.p, c.nnodes * sizeof(uint2), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(kids.data(), c.kids.p, c.nnodes * sizeof(int2), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      int64_t *o = static_cast<int64_t *>(buf);
      for (int64_t k = 0; k < c.nnodes; ++k) {
        int64_t *r = o + 8 * k;
        r[0] = cell[k].w; r[1] = cell[k].x; r[2] = cell[k].y; r[3] = cell[k].z;
        r[4] = range[k].x; r[5] = range[k].y;
        r[6] = kids[k].y ? kids[k].x : -1;
        r[7] = kids[k].y;
      }
      break;
    }
    case HFMM_EXPORT_KD_NODES: {
      const size_t nn = (size_t)c.nnodes;
      std::vector<uint32_t> first(nn), count(nn);
      std::vector<int> child(nn), axis(nn);
      e = cudaMemcpy(first.data(), c.kd.first.p, nn * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(count.data(), c.kd.count.p, nn * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(child.data(), c.kd.child.p, nn * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(axis.data(), c.kd.axis.p, nn * 4, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      int64_t *o = static_cast<int64_t *>(buf);
      int lev = 0;
      for (size_t k = 0; k < nn; ++k) {
        while ((int64_t)k >= c.kd.level_start[lev + 1]) ++lev;
        int64_t *r = o + 5 * k;
        r[0] = lev; r[1] = first[k]; r[2] = count[k]; r[3] = child[k]; r[4] = axis[k];
      }
      break;
    }
    case HFMM_EXPORT_KD_BOXES: {
      const size_t nn = (size_t)c.nnodes;
      std::vector<double> b(6 * nn);
      for (int q = 0; q < 6 && e == cudaSuccess; ++q)
        e = cudaMemcpy(b.data() + q * nn, P<double>(c.kd.box) + q * c.kd.cap, nn * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      double *o = static_cast<double *>(buf);
      for (size_t k = 0; k < nn; ++k)
        for (int q = 0; q < 6; ++q) o[6 * k + q] = b[q * nn + k];
      break;
    }
    case HFMM_EXPORT_CANDIDATES: {
      std::vector<uint64_t> v(c.ncand_last);
      e = cudaMemcpy(v.data(), c.cand.p, c.ncand_last * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      int64_t *o = static_cast<int64_t *>(buf);
      for (int64_t t = 0; t < c.ncand_last; ++t) {
        o[3 * t] = pair_sink(v[t]);
        o[3 * t + 1] = pair_src(v[t]);
        o[3 * t + 2] = pair_shift(v[t]);
      }
      break;
    }
    case HFMM_EXPORT_M2L_ORDER: {
      std::vector<uint64_t> v(c.nm2l);
      e = cudaMemcpy(v.data(), c.m2l.p, c.nm2l * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      int64_t *o = static_cast<int64_t *>(buf);
      for (int64_t t = 0; t < c.nm2l; ++t) o[t] = pair_order(v[t]);
      break;
    }
    case HFMM_EXPORT_P2P:
    case HFMM_EXPORT_M2L: {
      int64_t cnt = what == HFMM_EXPORT_P2P ? c.np2p : c.nm2l;
      std::vector<uint64_t> v(cnt);
      e = cudaMemcpy(v.data(), (what == HFMM_EXPORT_P2P ? c.p2p : c.m2l).p, cnt * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      int64_t *o = static_cast<int64_t *>(buf);
      for (int64_t t = 0; t < cnt; ++t) {
        o[3 * t] = pair_sink(v[t]);
        o[3 * t + 1] = pair_src(v[t]);
        o[3 * t + 2] = pair_shift(v[t]);
      }
      break;
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "export copy");
  return HFMM_OK;
}

int hfmm_load_mlp(hfmm_ctx *h, const void *weights_bf16, size_t bytes) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  const size_t need = (size_t)kMlpWeights * 2;
  if (!weights_bf16 || bytes != need) return fail(c, HFMM_ERR_ARG, "weights must be 5512 BF16 values (11024 bytes)");
  cudaError_t e = ensure(c.mlp_w, need);
  if (e == cudaSuccess) e = cudaMemcpy(c.mlp_w.p, weights_bf16, need, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "load_mlp");
  c.have_mlp = true;
  return HFMM_OK;
}

int hfmm_collect_training_pairs(hfmm_ctx *h, int64_t max_pairs, uint32_t sample_mod, float *features, float *errors,
                                int64_t *count, void *stream) {
  if (!h || !count) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  *count = 0;
  if (!c.have_tree) return fail(c, HFMM_ERR_STATE, "collect_training_pairs before build_tree");
  if (c.p != kPMax) return fail(c, HFMM_ERR_ARG, "training pairs need a context of order 8");
  if (max_pairs < 1 || !features || !errors) return fail(c, HFMM_ERR_ARG, "need max_pairs >= 1 and device buffers");
  cudaError_t e = collect_pairs(c, max_pairs, sample_mod, features, errors, count, S(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "collect_training_pairs");
  return HFMM_OK;
}

int hfmm_mlp_infer(const void *weights_bf16, const float *features, int64_t n, float *logits, int32_t *classes,
                   void *stream) {
  if (n < 0 || (n > 0 && (!weights_bf16 || !features))) return HFMM_ERR_ARG;
  return mlp_infer(weights_bf16, features, n, logits, classes, S(stream)) == cudaSuccess ? HFMM_OK : HFMM_ERR_CUDA;
}

int hfmm_mlp_grad(hfmm_ctx *h, const float *weights, const float *features, const int32_t *labels,
                  const float *class_weights, int64_t n, float *grad, float *loss, void *stream) {
  if (!h) return HFMM_ERR_ARG;
  Ctx &c = h->c;
  if (n < 1 || !weights || !features || !labels || !grad) return fail(c, HFMM_ERR_ARG, "bad training arguments");
  cudaError_t e = ensure(c.mlp_scratch, mlp_train_scratch_bytes());
  if (e == cudaSuccess) e = mlp_grad(weights, features, labels, class_weights, n, grad, loss, c.mlp_scratch.p, S(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "mlp_grad");
  return HFMM_OK;
}

int hfmm_mlp_adam(const float *grad, float lr, int step, float *weights, float *m1, float *m2, void *weights_bf16,
                  void *stream) {
  if (!grad || !weights || !m1 || !m2 || step < 1) return HFMM_ERR_ARG;
  return mlp_adam(weights, m1, m2, grad, lr, step, weights_bf16, S(stream)) == cudaSuccess ? HFMM_OK : HFMM_ERR_CUDA;
}

}  // extern "C"
