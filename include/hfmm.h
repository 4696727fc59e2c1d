/*
 * hfmm.h - C ABI of libhfmm.so, a GB300 (sm_103a) implementation of the
 * Gaussian-truncated short-range fast multipole method of Wang, "A Hybrid Fast
 * Multipole Method for Cosmological N-body Simulations" (Secs. 2.1-2.3), with a
 * plain particle-mesh long-range part (Sec. 2.2, PM filter).
 *
 * Problem (Sec. 2.2): N particles with masses m_j and positions x_j in a
 * periodic cube of side L.  Gravity is split at the scale r_s; this library
 * computes the short-range acceleration
 *     a_i = G sum_{j != i, 0 < |r_ij| < R_c} m_j f_(1)(|r_ij|) r_ij,
 *     f_(1)(r) = -[erfc(r / 2r_s) + r / (r_s sqrt(pi)) exp(-r^2 / 4r_s^2)] / r^3,
 * r_ij the minimum-image separation x_i - x_j, approximated by a truncated FMM:
 * Morton octree (or, with hfmm_params.tree = 1, the ORB / k-d tree of Sec. 2.1
 * and Sec. 4), P2M/M2M (Eqs. p2m, m2m), dual-tree traversal with the
 * three-rule acceptance criterion (Sec. 2.3), M2L with the derivative tensors
 * of erfc(r/2r_s)/r (Eq. m2l and the general-order prefactors of Sec. 2.2),
 * L2L/L2P (Eqs. l2l, l2p) and a cut-off P2P sum.
 *
 * Conventions for every entry point:
 *  - Return value: HFMM_OK (0) or a negative HFMM_ERR_* code; no exception or
 *    abort crosses the ABI.  hfmm_last_error() gives a message.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls may synchronise the stream where
 *    their documentation says so (data-dependent sizes).
 *  - Device pointers belong to the caller, must stay valid until the call's
 *    work on `stream` has completed, and are never freed by the library.
 *    Library workspaces (tree, lists, expansions) belong to the context and
 *    grow on demand; they are released by hfmm_destroy().
 *  - Positions are FP64 structure-of-arrays [3][n] (x block, y block, z
 *    block); masses FP32 [n]; accelerations FP32 SoA [3][n], in the caller's
 *    particle order.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef HFMM_H
#define HFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HFMM_OK = 0,
  HFMM_ERR_ARG = -1,      /* invalid argument (null pointer, bad size or parameter) */
  HFMM_ERR_OOM = -2,      /* device or host allocation failed */
  HFMM_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  HFMM_ERR_CAPACITY = -4, /* an index format limit was exceeded (more than 2^27 tree nodes; an
                             interaction list above 2^32 - 1 entries) */
  HFMM_ERR_STATE = -5,    /* call out of order (e.g. forces before build_tree) */
  HFMM_ERR_TIMEOUT = -6   /* a bounded device-side wait gave up */
};

/* Solver parameters.  r_s = rs_cells * box / pm_grid (Sec. 2.2: r_s ~ 1.2 grid
 * cells), R_c = rcut_rs * r_s (Sec. 2.2: cut-off ~ 5 r_s), R_c < box / 2. */
typedef struct {
  double box;          /* L, side of the periodic cube */
  int pm_grid;         /* N_g, PM mesh cells per side */
  double rs_cells;     /* r_s in PM cells */
  double rcut_rs;      /* R_c in units of r_s */
  double G;            /* gravitational constant */
  double theta;        /* opening angle theta_MAC of Sec. 2.3 (0 = never accept M2L) */
  int order;           /* expansion order p, 1..8 (total order |n| + |m| <= p) */
  int leaf_max;        /* a cell is split while it holds more than leaf_max particles (1..64) */
  int mac_mode;        /* 0 = geometric acceptance (Sec. 2.3); 1 = learned acceptance: rules 1
                          and 3 of Sec. 2.3 unchanged, and in place of rule 2 a network chooses,
                          for each pair with L / S_c <= theta (theta is then a safety bound),
                          between opening the pair and M2L at an order q in 2..order
                          (needs hfmm_load_mlp; order 8 recommended) */
  int transition_rule; /* 0: open iff S_c > R_c >= S_m (Sec. 2.3 as printed);
                          1: open iff S_max > R_c >= S_m (every M2L pair lies within R_c) */
  int size_rule;       /* L in theta = L / S_c: 0 = side of the source cell (as printed),
                          1 = larger side of the two cells */
  int m2l_precision;   /* 0 = FP32 on CUDA cores; split products hi*hi + hi*lo + lo*hi on the
                          tcgen05 tensor cores with FP32 accumulation in tensor memory
                          (orders 1..6): 1 = 3xTF32, 2 = BF16x3 (lo = bf16(x - bf16(x)),
                          about 2^-16 relative per product) */
  int profile;         /* bit 0: record per-phase CUDA-event timings; bit 1: count P2P
                          particle pairs (extra work; for statistics runs only) */
  int m2l_tables;      /* 1 = same-level M2L pairs whose integer cell offset o satisfies
                          |o_d| <= 2 floor(1/theta) + 1 read their translation operator
                          T_c = D_c(-o h) h^(|c|+1) (Eq. m2l with the truncated D of Sec. 2.2)
                          from a per-(level, offset) table built once in FP64 on the device;
                          other pairs evaluate D per pair.  0 (default) = every pair
                          evaluates D: on the 2M-particle clustered set (leaf 48, theta 0.35,
                          p 6) loading a table row per pair costs more than evaluating D
                          (2.79 vs 1.90 ms of M2L).  Used by m2l_precision 0 only. */
  /* Launch shapes (0 = built-in default; results do not depend on them beyond
     FP32 summation order).  The autotuner (autotune.py) picks them per GPU and
     workload and stores them in a JSON cache. */
  int tile_p2p_stage;  /* P2P source particles staged per warp: 128 or 256 (default 256) */
  int tile_p2p_blocks; /* P2P grid: blocks of 256 threads per SM, 1..8 (default 8; the kernel is
                          persistent and at most 2 of them are resident per SM) */
  int tile_m2l_blocks; /* cap on M2L blocks of 128 threads, per SM, 1..64 (default 64) */
  int tile_trav_blocks;/* traversal blocks of 256 threads per SM, 1..4 (default 4; capped by occupancy) */
  int use_graph;       /* 1 = hfmm_short_range_forces runs as one CUDA graph (captured on a library
                          stream, launched on the caller's): upward pass, the walk, list grouping,
                          M2L, L2L/L2P and P2P, with no host read-back inside; the lists take their
                          capacities from the last call (or the first guess), their sizes stay on
                          the device, and one read-back after the graph checks them: if a list
                          overflowed, the call runs again directly (growing the lists), so the
                          result is the same.  The executable graph is updated in place while the
                          launch sequence keeps its shape, else re-instantiated.  hfmm_step then
                          runs the whole kick-drift-kick step as one graph (see hfmm_step).
                          Geometric acceptance, m2l_precision 0, m2l_tables 0, p2p_mutual 0,
                          profile bit 1 off; otherwise ignored. */
  int tc_wait_polls;   /* m2l_precision 1 and 2: polls of the bounded wait for each chunk's MMAs before the
                          call gives up with HFMM_ERR_TIMEOUT (0 = 2^22; -1 = no poll at all, so that
                          every chunk gives up at once: a test of the error path).  After a give-up
                          every CTA waits again, with the full 2^22 polls, for the MMAs it issued
                          before it frees its tensor memory. */
  int split;           /* truncation of the force split: 0 = the Gaussian one of Sec. 2.2 (short-range
                          kernel erfc(r / 2r_s) / r); 1 = a polynomial one, which Sec. 5 allows in place
                          of it: kernel 1/r - P(r) for r < R_c and 0 beyond, P(r) = (15 - 10 w^2 +
                          3 w^4) / (8 R_c), w = r / R_c (the even quartic that makes the kernel and its
                          first two derivatives vanish at R_c; R_c = rcut_rs r_s is its only scale).
                          The pair force is then m (-1/r^3 + 5 / (2 R_c^3) - 3 r^2 / (2 R_c^5)) r, the
                          M2L prefactors the Newtonian ones minus those of P (none beyond the second),
                          and the PM Green function 4 pi / k^2 minus the transform of the kernel.
                          Split 1 needs mac_mode 0, m2l_precision 0 and m2l_tables 0. */
  int p2p_mutual;      /* 1 = mutual P2P (Newton's third law): the walk keeps one of the two ordered
                          leaf pairs (A, B, s) and (B, A, -s): the one whose sink A is the deeper
                          leaf; at equal depth the one with A < B if A + B is odd, A > B if even
                          (A = B: s at or below the unshifted index 13); the kernel evaluates each particle pair of
                          it once and adds the reaction on B's particles to per-entry partial sums,
                          which a second pass adds to B's accelerations in list order (the result
                          does not depend on scheduling).  A leaf against itself stays one-sided.
                          Needs mac_mode 0 and size_rule 1 (the walk is then symmetric); ignores
                          use_graph.  The partials take 12 bytes per (entry, source particle). */
  int list_init;       /* initial capacity, in entries, of every traversal list (frontier, M2L, P2P,
                          segments, runs) of a new context: 0 = a guess scaled with n and leaf_max;
                          a small value makes the walk overflow and repeat with grown lists (the
                          lists come out the same either way) */
  int sink_batches;    /* hfmm_short_range_forces in batches of sinks (0 = automatic: one batch
                          while the first guess of the P2P list stays below 2^28 entries, else
                          batches of about 2^27 guessed entries; 1..4096 = that many).  The walk
                          takes the top levels once (4, 5 or 6 of them as the batches grow),
                          then each batch of sink cells (a contiguous Morton range, about equal
                          particle counts) walks to the
                          leaves, and its lists are grouped and evaluated before the next batch
                          reuses the list memory, so memory and the 32-bit list bounds apply per
                          batch.  The lists hold the same entries, split by sink; a leaf above
                          the split level sums its entries in two groups (rounding differs from
                          one batch in the last bits).  Not in graph mode; after a call in more than one
                          batch the P2P / M2L lists cannot be exported. */
  int tree;            /* 0 = Morton octree (the default; every option above applies);
                          1 = the ORB / k-d tree of Sec. 2.1 (Fig. 1) and Sec. 4: a node of more than
                          leaf_max particles gives the first floor(n / 2) of them, in the order of
                          (coordinate, input index) along the longest axis of their bounding box, to its
                          first child and the rest to its second (the lowest axis on a tie); nodes are
                          numbered breadth first, and a leaf's particles are in (x, input index) order.
                          The geometry of a node is its particles' bounding box: expansions about its
                          centre, the rules of Sec. 2.3 on the boxes in FP64 (S_c between the centres,
                          S_m and S_max from per-axis gaps and spans, side = largest extent; a pair with
                          theta S_c = 0 is never accepted), the walk opening the node of larger side.
                          hfmm_build_tree synchronises `stream` once (the level extents); the walk is
                          one cooperative launch, followed by one read-back (repeated with grown
                          buffers when a list or the frontier outgrew its buffer).  Needs mac_mode 0,
                          m2l_precision 0, m2l_tables 0, p2p_mutual 0 and order <= 6 (either split);
                          use_graph and sink_batches are ignored, and
                          HFMM_EXPORT_KEYS and HFMM_EXPORT_NODES are octree only
                          (HFMM_EXPORT_KD_NODES and _KD_BOXES describe this tree).  The conventional
                          walk of hfmm_interaction_counts uses the same boxes and opening order. */
} hfmm_params;

/* Counters and timings of the last build_tree / short_range_forces call. */
typedef struct {
  int64_t n, nnodes, nleaves;
  int32_t nlevels, traverse_iters;
  int64_t np2p;           /* P2P leaf pairs */
  int64_t nm2l;           /* M2L cell pairs */
  int64_t p2p_particle_pairs; /* particle pairs evaluated by P2P incl. masked (profile bit 1, else -1) */
  int64_t p2p_useful_pairs;   /* pairs with 0 < r < R_c (profile bit 1, else -1) */
  int64_t launches;           /* kernels launched by this library in this process so far */
  /* milliseconds, filled when profile bit 0 is set (else -1); t_l2l covers L2L and L2P.
     After a call in graph mode t_upward covers the whole graph (upward pass to P2P) and
     t_traverse, t_lists, t_m2l, t_l2l, t_p2p are -1; after a step run as one graph
     t_upward covers the whole step and t_keys_sort, t_tree are -1 too; after a call in
     sink batches t_traverse covers everything after the upward pass and t_lists .. t_p2p
     are -1. */
  float t_keys_sort, t_tree, t_upward, t_traverse, t_lists, t_m2l, t_l2l, t_p2p;
  int64_t nm2l_table;         /* M2L pairs served by the operator table (profile bit 1, else -1) */
  int64_t frontier_pairs;     /* cell pairs the traversal classified, over all levels */
  int64_t traverse_walks;     /* walks the last traversal took (1 + repeats after a list overflowed) */
  int64_t step_graphs;        /* hfmm_step calls launched as one graph by this context */
  int64_t graph_captures;     /* graphs this context captured and instantiated or updated */
  int64_t sink_batches;       /* batches the last short-range call took */
} hfmm_stats;

typedef struct hfmm_ctx hfmm_ctx;

/* Default parameters of the small uniform workload: box 1, PM 32^3, r_s 1.25
 * cells, R_c 4.5 r_s, G 1, theta 0.5, p 4, 16 particles per leaf. */
void hfmm_default_params(hfmm_params *out);

/* Create a context on the current CUDA device.  Validates *params
 * (HFMM_ERR_ARG on a bad value).  *out receives the context. */
int hfmm_create(const hfmm_params *params, hfmm_ctx **out);

/* Release every library-owned buffer.  NULL is accepted. */
void hfmm_destroy(hfmm_ctx *ctx);

/* Message of the last failing call on ctx (or of hfmm_create when ctx is NULL). */
const char *hfmm_last_error(const hfmm_ctx *ctx);

/*
 * Build the octree (Sec. 2.1; a Morton-key octree): wrap positions into the
 * box (x - L floor(x / L)), 63-bit Morton keys on a 2^21 grid per side, stable
 * sort by (key, input index), split cells holding more than leaf_max particles
 * (depth cap 21), per-particle FP32 offsets from the geometric leaf centre.
 * pos_soa: device FP64 [3][n], finite values (any finite position is wrapped;
 * a NaN or infinite coordinate is not checked and lands in an arbitrary cell);
 * mass: device FP32 [n]; n >= 0 (n = 0 gives an empty tree).  The levels are built in one cooperative launch; `stream` is
 * synchronised once to read the node and level counts back (again if the node
 * capacity had to grow).  The library keeps no reference to pos/mass after the
 * call returns.
 */
int hfmm_build_tree(hfmm_ctx *ctx, const double *pos_soa, const float *mass, int64_t n, void *stream);

/*
 * Short-range accelerations of the particles of the last hfmm_build_tree:
 * P2M, M2M, dual-tree traversal with the hybrid acceptance rules, M2L, L2L,
 * L2P and the cut-off P2P (Secs. 2.1-2.3).  acc_soa: device FP32 [3][n], input
 * particle order, overwritten.  HFMM_ERR_STATE before any build_tree;
 * HFMM_ERR_OOM when the interaction lists do not fit in device memory (list
 * capacities start from a guess scaled with leaf_max and only lists that
 * overflow are grown, the walk then repeated); HFMM_ERR_CAPACITY when the M2L
 * or the P2P list exceeds 2^32 - 1 entries (the lists grouped by sink are
 * addressed through 32-bit bounds).  The traversal is one
 * cooperative launch; `stream` is synchronised once after it to read the list
 * sizes back, and once more after a tensor-core M2L to read its status word.
 */
int hfmm_short_range_forces(hfmm_ctx *ctx, float *acc_soa, void *stream);

/*
 * The same computation on HOST buffers: copies pos_soa (FP64 [3][n]) and mass
 * (FP32 [n]) to library-owned device memory, builds the tree, computes the
 * short-range accelerations and copies them to acc_soa (host FP32 [3][n]).
 * Returns after the result is on the host.  Pinned host memory gives
 * asynchronous copies; pageable memory works too.
 */
int hfmm_short_range_forces_host(hfmm_ctx *ctx, const double *pos_soa, const float *mass, int64_t n,
                                 float *acc_soa, void *stream);

/*
 * Long-range accelerations of the force split (Sec. 2.2: 1/r = erfc(r/2r_s)/r +
 * erf(r/2r_s)/r; the erf part on the PM mesh of the same section; with split 1 the
 * complement of the polynomial kernel, Green function 4 pi / k^2 minus the kernel's
 * transform, tabulated in FP64 per integer |k|^2 on the mesh), ADDED to acc_soa
 * (device float32 [3][n], input order) for the particles of the last
 * hfmm_build_tree.  Mesh: pm_grid^3 points x_g = g L / pm_grid; cloud-in-cell
 * assignment and interpolation; cuFFT; Green function 4 pi G exp(-k^2 r_s^2) / k^2
 * divided by the squared CIC window; spectral gradient i k with the Nyquist plane
 * of each component set to zero; k = 0 dropped.  The mass mesh is accumulated in
 * 64-bit fixed point, so the result does not depend on the order of the atomic
 * additions.  Library-owned mesh buffers (about 24 pm_grid^3 bytes) are kept
 * between calls.  pm_grid must be in 2..1024.  Errors: HFMM_ERR_STATE before
 * hfmm_build_tree, HFMM_ERR_ARG for a null acc_soa or a pm_grid outside 2..1024,
 * HFMM_ERR_CUDA for a failed launch or transform.
 */
int hfmm_pm_long_range(hfmm_ctx *ctx, float *acc_soa, void *stream);

/*
 * One kick-drift-kick leapfrog step of length dt in a static periodic box
 * (the synchronised global step of Sec. 4, without cosmological
 * factors), for the particles and masses of the last hfmm_build_tree:
 *   vel += acc dt/2;  pos += vel dt, wrapped into [0, L);  hfmm_build_tree(pos);
 *   acc = short range + long range at the new positions;  vel += acc dt/2.
 * pos_soa (device float64 [3][n]), vel_soa and acc_soa (device float32 [3][n])
 * are the caller's and are updated in place; on entry acc_soa must hold the
 * total acceleration at pos_soa (hfmm_short_range_forces then
 * hfmm_pm_long_range, or the previous step).  The mass array given to
 * hfmm_build_tree must stay valid.  Errors as for the calls it makes.
 * With use_graph (and the configurations it covers) the whole step is one CUDA
 * graph with no host read-back inside: the tree's sizes stay on the device
 * (nodes up to a capacity kept in the context, levels up to the last tree's
 * plus two), the lists take their capacities from the last call, and the
 * second kick runs only when all of them fitted.  One read-back after the graph
 * checks them; after an overflow the step goes on directly from the drifted
 * positions (rebuilding the tree, growing what overflowed), so the result is
 * the same.  The graph is captured again only when a buffer address, a
 * capacity or an argument changed since the last capture.
 */
int hfmm_step(hfmm_ctx *ctx, double *pos_soa, float *vel_soa, float *acc_soa, double dt, void *stream);

/* Counters and timings of the last calls (synchronises the context's work). */
int hfmm_get_stats(hfmm_ctx *ctx, hfmm_stats *out);

/*
 * Interaction counts of the comparison of Sec. 3 (Figs. 5-6: the P2P and M2L
 * kernel counts of the truncated FMM against a conventional FMM; the counts
 * depend only on the tree and the acceptance criterion).  Runs the dual-tree
 * walk alone (no expansions, no forces) on the tree of the last
 * hfmm_build_tree (the octree, or with tree = 1 the k-d tree and its boxes), with
 *   conventional = 0: the hybrid acceptance of Sec. 2.3 with the context's
 *     theta, transition_rule and size_rule and geometric decisions (also on a
 *     mac_mode 1 context), from the root against its 27 nearest periodic
 *     images, exactly the walk of hfmm_short_range_forces;
 *   conventional = 1: a conventional FMM's acceptance, the opening-angle test
 *     of Sec. 2.3 alone (accept M2L iff L / S_c <= theta with the context's
 *     size_rule; otherwise open the larger cell, both on a tie; two leaves give
 *     P2P), with no cut-off skip and no transition region, from the single pair
 *     (root, root) of the primary box: the walk a conventional FMM performs
 *     before treating the periodic images by Ewald summation.
 * out: host int64 [4]: M2L cell pairs, P2P leaf pairs, particle pairs on the
 * P2P lists (sum over P2P entries of n_sink n_source, a leaf against itself
 * included), cell pairs classified over all levels.  Replaces the context's
 * interaction lists (hfmm_get_stats and hfmm_export then report this walk's;
 * the next hfmm_short_range_forces walks again); list capacities grown by
 * the walk are kept.  Synchronises the stream.  HFMM_ERR_ARG for a null out or
 * conventional outside {0, 1}; HFMM_ERR_STATE before any build_tree;
 * HFMM_ERR_OOM when the lists do not fit in device memory.
 */
int hfmm_interaction_counts(hfmm_ctx *ctx, int conventional, int64_t *out, void *stream);

/*
 * Copy an internal array to host memory for inspection.  With host_buf NULL,
 * *bytes receives the size needed; otherwise at most *bytes are copied and
 * *bytes receives the size.  Synchronises the device.  Formats:
 *  HFMM_EXPORT_KEYS     uint64 [n]      Morton keys in sorted order
 *  HFMM_EXPORT_PERM     uint32 [n]      input index of each sorted particle
 *  HFMM_EXPORT_NODES    int64 [nnodes][8] level, ix, iy, iz, first, count,
 *                                       first child (-1 for a leaf), child count;
 *                                       breadth-first, key order within a level
 *  HFMM_EXPORT_P2P      int64 [np2p][3]  sink node, source node, shift index
 *  HFMM_EXPORT_M2L      int64 [nm2l][3]  (shift index s: (sx+1)*9+(sy+1)*3+(sz+1),
 *                                       the source is displaced by s * L)
 *  HFMM_EXPORT_MULTIPOLES float [nnodes][ncoef(p)]  M_m / h^|m|   (h = cell side)
 *  HFMM_EXPORT_LOCALS     float [nnodes][ncoef(p)]  L_n * h^(|n|+1)
 *                       (tree 1: h = the node's scale, the power of two L 2^-j at or above
 *                       its side, j <= 21)
 * Multi-index order: for k = 0..p, nx = k..0, ny = k-nx..0, nz = k-nx-ny.
 */
enum {
  HFMM_EXPORT_KEYS = 0,
  HFMM_EXPORT_PERM = 1,
  HFMM_EXPORT_NODES = 2,
  HFMM_EXPORT_P2P = 3,
  HFMM_EXPORT_M2L = 4,
  HFMM_EXPORT_MULTIPOLES = 5,
  HFMM_EXPORT_LOCALS = 6,
  HFMM_EXPORT_M2L_ORDER = 7, /* int64 [nm2l] expansion order of each M2L entry, list order */
  HFMM_EXPORT_CANDIDATES = 8, /* int64 [n][3] pairs of the last hfmm_collect_training_pairs (row order) */
  HFMM_EXPORT_KD_NODES = 9,   /* tree 1: int64 [nnodes][5] level, first, count, first child (-1 for a
                                 leaf; the second child follows it), split axis (-1 for a leaf) */
  HFMM_EXPORT_KD_BOXES = 10   /* tree 1: double [nnodes][6] bounding box lo x y z, hi x y z */
};
int hfmm_export(hfmm_ctx *ctx, int what, void *host_buf, size_t *bytes);

/*
 * Learned acceptance (an addition to the paper's Sec. 2.3 criterion).
 * The network maps 12 pair features to 8 classes {open, M2L at order 2..8}:
 * 12 -> 64 -> ReLU -> 64 -> ReLU -> 8, BF16 weights, FP32 accumulation.
 * Weight blob: 5512 BF16 values, W1[64][12], b1[64], W2[64][64], b2[64],
 * W3[8][64], b3[8].  Features (half units; all dimensionless): S_c/r_s,
 * S_m/r_s, S_max/R_c, h_A/S_c, h_B/S_c, max(h_A,h_B)/S_c, (level_A-level_B)/8,
 * log2(1+n_A)/16, log2(1+n_B)/16, |dipole of B|/|M_0|, |quadrupole of B|/|M_0|
 * (scaled multipoles), S_c/R_c.
 */
/* Copy the network's weights (host pointer, 11024 bytes) to the context. */
int hfmm_load_mlp(hfmm_ctx *ctx, const void *weights_bf16, size_t bytes);

/*
 * Training data, measured by the method itself: after hfmm_build_tree on an
 * order-8 context, visit every cell pair (every pair opened), and for a
 * hash-sampled 1/sample_mod of the candidate pairs (rules 1 and 3 passed,
 * L / S_c <= theta) write the 12 features (device FP32 [n][12]) and the error
 * of M2L at orders 2..8 against the pair's own direct sum, measured on up to
 * 32 particles of the sink cell (device FP32 [n][7]:
 * |a_M2L - a_direct|_2 / |a_direct|_2).  At most max_pairs rows; *count
 * receives n.  Synchronises the stream.
 */
int hfmm_collect_training_pairs(hfmm_ctx *ctx, int64_t max_pairs, uint32_t sample_mod, float *features,
                                float *errors, int64_t *count, void *stream);

/* Network inference on the tensor cores (device pointers): logits [n][8]
 * and/or classes [n] (argmax, ties to the lower class); either may be NULL. */
int hfmm_mlp_infer(const void *weights_bf16, const float *features, int64_t n, float *logits, int32_t *classes,
                   void *stream);

/*
 * Mean softmax cross-entropy over n samples and its gradient (device
 * pointers): weights = FP32 master copy [5512] (rounded to BF16 in the
 * forward pass, as the inference does), labels [n] in 0..7, class_weights
 * [8] or NULL; grad [5512] and loss [1] are written.  Uses ctx's scratch.
 */
int hfmm_mlp_grad(hfmm_ctx *ctx, const float *weights, const float *features, const int32_t *labels,
                  const float *class_weights, int64_t n, float *grad, float *loss, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected at `step` >= 1)
 * on the FP32 master weights; writes the BF16 copy when weights_bf16 != NULL. */
int hfmm_mlp_adam(const float *grad, float lr, int step, float *weights, float *m1, float *m2, void *weights_bf16,
                  void *stream);

/*
 * Throughput probe for the roofline denominators of the ALU-bound kernels (the
 * P2P pair sum and the CUDA-core M2L).  The paper has no counterpart: it is a
 * measurement aid.  kind 0 = FP32 fused multiply-add (2 flop each), 1 = packed
 * FP32x2 fused multiply-add (4 flop each), 2 = ex2.approx, 3 = rsqrt.approx
 * (1 operation each).  Launches 8 blocks of 256 threads per SM, each thread
 * running 16 independent chains for iters x 8 steps, once untimed and once
 * timed with CUDA events on `stream`.  scratch: device FP32 buffer of
 * 2048 x (SM count) values (overwritten).  *rate receives flop/s (kinds 0, 1)
 * or operations/s (kinds 2, 3); *ms (may be NULL) the timed launch in
 * milliseconds.  Synchronises the stream.  HFMM_ERR_ARG for a bad kind, iters
 * < 1 or a null scratch or rate; HFMM_ERR_CUDA if a launch or an event fails.
 */
int hfmm_alu_peak(int kind, int iters, float *scratch, double *rate, double *ms, void *stream);

/*
 * Allocation-free Morton keys + sort.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory at the point of
 * the call - for example a host runtime that plans all GPU memory up front and
 * forbids further cudaMalloc, or code that must not risk the implicit device
 * synchronisation cudaMalloc/cudaFree can cause.  It computes what the first
 * steps of hfmm_build_tree compute: wrap into [0, box), 63-bit Morton keys on a
 * 2^21 grid per side, stable sort by (key, input index).
 *  pos_soa  device FP64 [3][n] (caller's)       keys_out device uint64 [n] (caller's)
 *  perm_out device uint32 [n]: input index of each sorted key (caller's)
 * Scratch: one file-scope device array of fixed size (about 6.5 MB, enough for
 * HFMM_NOALLOC_MAX_N particles) that every GPU loading the library holds until
 * the process exits.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call in each CUDA context looks up that array's device
 * address (cudaGetSymbolAddress) with the context current, so make the first
 * call on a device before any stream capture.  The address is kept per context
 * (keyed by the context's process-unique id), so a call from another context on
 * the same device, or from the primary context re-created after
 * cudaDeviceReset, looks the address up again rather than reusing a stale one.
 * Every call on a device shares the array:
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  Nothing in the array is
 * assumed to start at zero: each call writes every word before reading it.
 * Returns HFMM_OK; HFMM_ERR_CAPACITY if n > HFMM_NOALLOC_MAX_N; HFMM_ERR_ARG
 * for n < 0, box <= 0 or a null pointer with n > 0; HFMM_ERR_CUDA if a launch
 * fails, or, without launching anything, if a CUDA error of an earlier call
 * was already pending on entry (that error is left pending for the caller).
 * Work is enqueued on `stream`; the call does not synchronise.
 */
#define HFMM_NOALLOC_MAX_N 524288
int hfmm_morton_sort_noalloc(const double *pos_soa, int64_t n, double box, uint64_t *keys_out, uint32_t *perm_out,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HFMM_H */
