"""FP64 CPU oracle for the Gaussian-truncated short-range FMM (Wang, "A Hybrid
Fast Multipole Method for Cosmological N-body Simulations").

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  Nothing in the product
package imports this module, and this module imports nothing from it.

The C sources ``orc.c`` (Morton octree) and ``orc_kd.c`` (the ORB / k-d tree
variant) hold the arithmetic (FP64, OpenMP); this file only compiles them with
gcc and marshals numpy arrays through ctypes.

Parity status of each function (what pins it is in ``tests/test_oracle_*.py``):
  prefactors, derivative tensor, P2M/M2M/M2L/L2L/L2P, direct sum, tree,
  traversal (hybrid and conventional), interaction counts, FMM forces, the
  network's forward and gradient, its forward with the FP32 error bound, the
  pair features of the learned acceptance, the learned walk, the k-d tree, its
  walk and its FMM forces: pinned (closed forms, symbolic derivatives,
  exact identities, brute force, textbook interaction lists, special cases).
Sibling modules: ``pm.py`` (PM long range and the KDK step) and
``poly_split.py`` (a polynomial truncation of the split), both numpy FP64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = [os.path.join(_HERE, "orc.c"), os.path.join(_HERE, "orc_kd.c")]
_lock = threading.Lock()
_lib = None

# gcc flags: no FMA contraction and no fast-math, so the integer acceptance
# decisions and the wrap come out identical on x86-64 and aarch64.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile ``orc.c`` and ``orc_kd.c`` into ``oracle/_build/liborc.so`` (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *_SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            d, i64, i32 = C.c_double, C.c_int64, C.c_int
            P = C.c_void_p
            L.orc_ncoef.argtypes = [i32]
            L.orc_ncoef.restype = i32
            L.orc_multi_index.argtypes = [i32, P]
            L.orc_prefactors.argtypes = [d, d, i32, P]
            L.orc_deriv_tensor.argtypes = [P, d, i32, P]
            L.orc_p2m.argtypes = [i64, P, P, P, i32, P]
            L.orc_m2m.argtypes = [P, P, i32, P]
            L.orc_m2l.argtypes = [P, P, d, i32, P]
            L.orc_l2l.argtypes = [P, P, i32, P]
            L.orc_l2p.argtypes = [P, P, i32, d, P, P]
            L.orc_direct_sr.argtypes = [i64, P, P, d, d, d, d, i64, P, P]
            L.orc_create.argtypes = [d, d, d, d, d, i32, i32, i32, i32]
            L.orc_create.restype = P
            L.orc_destroy.argtypes = [P]
            L.orc_build_tree.argtypes = [P, i64, P, P]
            L.orc_traverse.argtypes = [P]
            L.orc_traverse_conventional.argtypes = [P]
            L.orc_upward.argtypes = [P]
            L.orc_m2l_pass.argtypes = [P]
            L.orc_downward.argtypes = [P, P]
            L.orc_p2p_pass.argtypes = [P, P]
            L.orc_fmm_forces.argtypes = [P, P]
            L.orc_size.argtypes = [P, i32]
            L.orc_size.restype = i64
            L.orc_export_particles.argtypes = [P, P, P, P]
            L.orc_export_nodes.argtypes = [P, P]
            L.orc_export_list.argtypes = [P, i32, P]
            L.orc_export_expansions.argtypes = [P, i32, P]
            L.orc_num_threads.restype = i32
            L.orc_bf16.argtypes = [d]
            L.orc_bf16.restype = d
            L.orc_mlp_forward.argtypes = [P, P, i64, i32, P]
            L.orc_mlp_loss_grad.argtypes = [P, P, P, P, i64, i32, P, P]
            L.orc_set_lists.argtypes = [P, P, i64, P, P, i64]
            L.orc_fmm_forces_given_lists.argtypes = [P, P]
            L.orc_pair_error.argtypes = [P, i64, i64, i32, i32]
            L.orc_pair_error.restype = d
            L.orc_find_node.argtypes = [P, i32, C.c_uint32, C.c_uint32, C.c_uint32]
            L.orc_find_node.restype = i64
            L.orc_pair_features.argtypes = [P, i64, i64, i32, P]
            L.orc_prefactors_poly.argtypes = [d, d, i32, P]
            L.orc_deriv_tensor_split.argtypes = [P, d, d, i32, i32, P]
            L.orc_direct_sr_split.argtypes = [i64, P, P, d, d, d, i32, d, i64, P, P]
            L.orc_set_split.argtypes = [P, i32]
            L.orc_mlp_forward_bound.argtypes = [P, P, P, i64, P, P, P, P]
            L.orc_traverse_learned.argtypes = [P, P, P, P, P, i64, P]
            L.orc_export_m2l_orders.argtypes = [P, P]
            L.orc_kd_create.argtypes = [d, d, d, d, d, i32, i32, i32, i32]
            L.orc_kd_create.restype = P
            L.orc_kd_destroy.argtypes = [P]
            L.orc_kd_build.argtypes = [P, i64, P, P]
            L.orc_kd_traverse.argtypes = [P]
            L.orc_kd_set_split.argtypes = [P, i32]
            L.orc_kd_traverse_conventional.argtypes = [P]
            L.orc_kd_upward.argtypes = [P]
            L.orc_kd_m2l_pass.argtypes = [P]
            L.orc_kd_downward.argtypes = [P, P]
            L.orc_kd_p2p_pass.argtypes = [P, P]
            L.orc_kd_forces.argtypes = [P, P]
            L.orc_kd_size.argtypes = [P, i32]
            L.orc_kd_size.restype = i64
            L.orc_kd_export.argtypes = [P, P, P, P]
            L.orc_kd_export_list.argtypes = [P, i32, P]
            L.orc_kd_set_lists.argtypes = [P, P, i64, P, i64]
            L.orc_kd_forces_given_lists.argtypes = [P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def ncoef(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def multi_indices(p: int) -> np.ndarray:
    """Graded multi-index order used by every expansion array: [ncoef(p)][3]."""
    out = np.zeros((ncoef(p), 3), dtype=np.int32)
    L = lib()
    for c in range(ncoef(p)):
        _check(L.orc_multi_index(c, _p(out[c])), "multi_index")
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- kernels
def prefactors(r: float, rs: float, p: int) -> np.ndarray:
    """f_(0..p)(r); rs <= 0 selects the Newtonian prefactors."""
    f = np.zeros(p + 1)
    _check(lib().orc_prefactors(float(r), float(rs), int(p), _p(f)), "prefactors")
    return f


def prefactors_poly(r: float, rc: float, p: int) -> np.ndarray:
    """f_(0..p)(r) of the polynomial truncation (Sec. 5 reading): 1/r - P(r) inside R_c."""
    f = np.zeros(p + 1)
    _check(lib().orc_prefactors_poly(float(r), float(rc), int(p), _p(f)), "prefactors_poly")
    return f


SPLITS = {"gauss": 0, "poly": 1}


def deriv_tensor(R, rs: float, p: int, split="gauss", rc=0.0) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64)
    D = np.zeros(ncoef(p))
    if split == "gauss":
        _check(lib().orc_deriv_tensor(_p(R), float(rs), int(p), _p(D)), "deriv_tensor")
    else:
        _check(lib().orc_deriv_tensor_split(_p(R), float(rs), float(rc), SPLITS[split], int(p), _p(D)),
               "deriv_tensor_split")
    return D


def p2m(x, mu, z, p):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    M = np.zeros(ncoef(p))
    _check(lib().orc_p2m(len(mu), _p(x), _p(mu), _p(z), p, _p(M)), "p2m")
    return M


def m2m(M, x, p):
    M = np.ascontiguousarray(M, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(ncoef(p))
    _check(lib().orc_m2m(_p(M), _p(x), p, _p(out)), "m2m")
    return out


def m2l(M, R, rs, p, L=None):
    M = np.ascontiguousarray(M, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.zeros(ncoef(p)) if L is None else np.ascontiguousarray(L, dtype=np.float64).copy()
    _check(lib().orc_m2l(_p(M), _p(R), float(rs), p, _p(L)), "m2l")
    return L


def l2l(L, x, p):
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(ncoef(p))
    _check(lib().orc_l2l(_p(L), _p(x), p, _p(out)), "l2l")
    return out


def l2p(L, u, p, G=1.0):
    L = np.ascontiguousarray(L, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    phi = np.zeros(1)
    a = np.zeros(3)
    _check(lib().orc_l2p(_p(L), _p(u), p, float(G), _p(phi), _p(a)), "l2p")
    return float(phi[0]), a


# ---------------------------------------------------------------- direct sum
def direct_sr(pos, mass, box, rs, rc, G=1.0, sinks=None, split="gauss") -> np.ndarray:
    """Minimum-image direct truncated sum; pos [3][n] -> acc [3][nsink] (FP64).
    split: "gauss" (Sec. 2.2) or "poly" (the polynomial truncation of Sec. 5)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = pos.shape[1]
    if sinks is None:
        ns, sp = n, None
    else:
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        ns, sp = len(sinks), sinks
    acc = np.zeros((3, ns))
    _check(lib().orc_direct_sr_split(n, _p(pos), _p(mass), box, rs, rc, SPLITS[split], G, ns, _p(sp), _p(acc)),
           "direct_sr")
    return acc


# ---------------------------------------------------------------- network
MLP_WEIGHTS = 5512


def bf16(x: float) -> float:
    return float(lib().orc_bf16(float(x)))


def mlp_forward(w, x, rnd=1) -> np.ndarray:
    """Logits [n][8] of the learned-acceptance network (weights as doubles, blob order)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 12)
    out = np.zeros((x.shape[0], 8))
    _check(lib().orc_mlp_forward(_p(w), _p(x), x.shape[0], int(rnd), _p(out)), "mlp_forward")
    return out


def mlp_forward_bound(w, x, xtol=None):
    """The network at its rounding points (BF16 inputs and hidden activations,
    exact sums) with a bound on the logits of any FP32 evaluation of it.
    x [n][12]; xtol [n][12] or None: how far the evaluated features may be
    from x before their BF16 rounding.  Returns (logits [n][8], bound [n][8],
    class [n], mask [n]): the class is the argmax of the logits (ties to the
    lower class), the mask has bit k set for every class the bound lets an
    evaluation's argmax take."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 12)
    n = x.shape[0]
    xt = None if xtol is None else np.ascontiguousarray(np.broadcast_to(xtol, x.shape), dtype=np.float64)
    lo = np.zeros((n, 8))
    el = np.zeros((n, 8))
    cls = np.zeros(n, dtype=np.int32)
    mask = np.zeros(n, dtype=np.uint32)
    _check(lib().orc_mlp_forward_bound(_p(w), _p(x), _p(xt), n, _p(lo), _p(el), _p(cls), _p(mask)),
           "mlp_forward_bound")
    return lo, el, cls, mask


def mlp_loss_grad(w, x, labels, class_weights=None, rnd=1):
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 12)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    cw = None if class_weights is None else np.ascontiguousarray(class_weights, dtype=np.float64)
    g = np.zeros(MLP_WEIGHTS)
    loss = np.zeros(1)
    _check(lib().orc_mlp_loss_grad(_p(w), _p(x), _p(lab), _p(cw), x.shape[0], int(rnd), _p(g), _p(loss)),
           "mlp_loss_grad")
    return float(loss[0]), g


# ---------------------------------------------------------------- FMM
class FMM:
    """FP64 truncated FMM with the same tree, MAC and lists as the GPU library."""

    def __init__(self, box=1.0, rs=None, rc=None, G=1.0, theta=0.5, order=4, leaf_max=16,
                 transition_rule=1, size_rule=1, split="gauss"):
        self._c = lib().orc_create(box, rs, rc, G, theta, order, leaf_max, transition_rule, size_rule)
        if not self._c:
            raise ValueError("invalid oracle parameters")
        _check(lib().orc_set_split(self._c, SPLITS[split]), "set_split")
        self.split = split
        self.box, self.rs, self.rc, self.G, self.theta = box, rs, rc, G, theta
        self.order, self.leaf_max, self.rule, self.size_rule = order, leaf_max, transition_rule, size_rule
        self.n = 0

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            lib().orc_destroy(c)
            self._c = None

    def build_tree(self, pos, mass):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = pos.shape[1]
        _check(lib().orc_build_tree(self._c, self.n, _p(pos), _p(mass)), "build_tree")

    def size(self, what):
        return int(lib().orc_size(self._c, {"n": 0, "nodes": 1, "levels": 2, "p2p": 3, "m2l": 4}[what]))

    def traverse(self, conventional=False):
        """The hybrid walk of Sec. 2.3, or (conventional=True) the conventional-FMM
        walk the interaction counts of Sec. 3 are compared against: the opening-angle
        test alone, from (root, root) of the primary box."""
        if conventional:
            _check(lib().orc_traverse_conventional(self._c), "traverse_conventional")
        else:
            _check(lib().orc_traverse(self._c), "traverse")

    def counts(self):
        """Interaction counts of the current lists (Sec. 3): M2L cell pairs, P2P leaf
        pairs, and particle pairs on the P2P lists (sum of n_sink n_source)."""
        nodes = self.nodes()
        p2p, m2l = self.lists()
        cnt = nodes[:, 5]
        pp = int((cnt[p2p[:, 0]] * cnt[p2p[:, 1]]).sum()) if len(p2p) else 0
        return {"m2l": len(m2l), "p2p": len(p2p), "p2p_particle_pairs": pp}

    def forces(self) -> np.ndarray:
        acc = np.zeros((3, self.n))
        _check(lib().orc_fmm_forces(self._c, _p(acc)), "fmm_forces")
        return acc

    def particles(self):
        n = self.n
        key = np.zeros(n, dtype=np.uint64)
        perm = np.zeros(n, dtype=np.int64)
        xs = np.zeros((n, 3))
        lib().orc_export_particles(self._c, _p(key), _p(perm), _p(xs))
        return key, perm, xs

    def nodes(self) -> np.ndarray:
        out = np.zeros((self.size("nodes"), 8), dtype=np.int64)
        lib().orc_export_nodes(self._c, _p(out))
        return out

    def lists(self):
        p2p = np.zeros((self.size("p2p"), 3), dtype=np.int64)
        m2l = np.zeros((self.size("m2l"), 3), dtype=np.int64)
        lib().orc_export_list(self._c, 0, _p(p2p))
        lib().orc_export_list(self._c, 1, _p(m2l))
        return p2p, m2l

    def expansions(self, which):
        out = np.zeros((self.size("nodes"), ncoef(self.order)))
        _check(lib().orc_export_expansions(self._c, {"M": 0, "L": 1}[which], _p(out)), "export_expansions")
        return out

    def forces_given_lists(self, p2p, m2l, orders=None):
        """FMM forces on the given lists (P2P and M2L rows: sink, source, shift; optional order per M2L row)."""
        p2p = np.ascontiguousarray(p2p, dtype=np.int64).reshape(-1, 3)
        m2l = np.ascontiguousarray(m2l, dtype=np.int64).reshape(-1, 3)
        o = None if orders is None else np.ascontiguousarray(orders, dtype=np.int64)
        _check(lib().orc_set_lists(self._c, _p(p2p), len(p2p), _p(m2l), _p(o), len(m2l)), "set_lists")
        acc = np.zeros((3, self.n))
        _check(lib().orc_fmm_forces_given_lists(self._c, _p(acc)), "fmm_forces_given_lists")
        return acc

    def pair_features(self, pairs) -> np.ndarray:
        """The 12 learned-acceptance features [n][12] of (sink, source, shift) rows;
        computes the multipoles first when they are missing."""
        pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)
        out = np.zeros((len(pairs), 12))
        for i, (a, b, sh) in enumerate(pairs):
            rc = lib().orc_pair_features(self._c, int(a), int(b), int(sh), _p(out[i]))
            if rc != 0:
                self.upward()
                _check(lib().orc_pair_features(self._c, int(a), int(b), int(sh), _p(out[i])), "pair_features")
        return out

    def traverse_learned(self, w, ftol_rel, ftol_abs, ref_m2l=None, ref_orders=None) -> dict:
        """The walk with the learned acceptance (the network in place of the
        opening-angle rule, theta the safety bound).  ftol_rel, ftol_abs [12]:
        feature tolerance of the evaluation the lists are compared with.  With
        ref_m2l / ref_orders (an evaluation's M2L list and orders) a candidate
        whose class the bound leaves open takes that list's decision."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        tr = np.ascontiguousarray(np.broadcast_to(ftol_rel, (12,)), dtype=np.float64)
        ta = np.ascontiguousarray(np.broadcast_to(ftol_abs, (12,)), dtype=np.float64)
        ref = None
        nref = 0
        if ref_m2l is not None:
            r = np.concatenate([np.asarray(ref_m2l, dtype=np.int64).reshape(-1, 3),
                                np.asarray(ref_orders, dtype=np.int64).reshape(-1, 1)], axis=1)
            ref = np.ascontiguousarray(r[np.lexsort((r[:, 2], r[:, 1], r[:, 0]))])
            nref = len(ref)
        st = np.zeros(6)
        _check(lib().orc_traverse_learned(self._c, _p(w), _p(tr), _p(ta), _p(ref), nref, _p(st)), "traverse_learned")
        return {"candidates": int(st[0]), "ambiguous": int(st[1]), "resolved": int(st[2]),
                "outside_bound": int(st[3]), "max_bound": float(st[4])}

    def m2l_orders(self) -> np.ndarray:
        out = np.zeros(self.size("m2l"), dtype=np.int64)
        lib().orc_export_m2l_orders(self._c, _p(out))
        return out

    def pair_error(self, a, b, s, q):
        return float(lib().orc_pair_error(self._c, int(a), int(b), int(s), int(q)))

    def find_node(self, lev, ix, iy, iz):
        return int(lib().orc_find_node(self._c, int(lev), int(ix), int(iy), int(iz)))

    # phase-by-phase access for the tests
    def upward(self):
        _check(lib().orc_upward(self._c), "upward")

    def m2l_pass(self):
        _check(lib().orc_m2l_pass(self._c), "m2l_pass")

    def downward(self):
        a = np.zeros((self.n, 3))
        _check(lib().orc_downward(self._c, _p(a)), "downward")
        return a

    def p2p_pass(self):
        a = np.zeros((self.n, 3))
        _check(lib().orc_p2p_pass(self._c, _p(a)), "p2p_pass")
        return a


class KdFMM:
    """FP64 truncated FMM on the ORB / k-d tree of Sec. 2.1 (Fig. 1) and Sec. 4:
    nodes split at the particle-count median along the longest axis of their
    particles' bounding box, boxes as cell geometry (the readings are in orc_kd.c)."""

    def __init__(self, box=1.0, rs=None, rc=None, G=1.0, theta=0.5, order=4, leaf_max=16,
                 transition_rule=1, size_rule=1, split="gauss"):
        self._c = lib().orc_kd_create(box, rs, rc, G, theta, order, leaf_max, transition_rule, size_rule)
        if not self._c:
            raise ValueError("invalid oracle parameters")
        _check(lib().orc_kd_set_split(self._c, SPLITS[split]), "kd_set_split")
        self.split = split
        self.box, self.rs, self.rc, self.G, self.theta = box, rs, rc, G, theta
        self.order, self.leaf_max, self.rule, self.size_rule = order, leaf_max, transition_rule, size_rule
        self.n = 0

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            lib().orc_kd_destroy(c)
            self._c = None

    def build_tree(self, pos, mass):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = pos.shape[1]
        _check(lib().orc_kd_build(self._c, self.n, _p(pos), _p(mass)), "kd_build")

    def size(self, what):
        return int(lib().orc_kd_size(self._c, {"n": 0, "nodes": 1, "levels": 2, "p2p": 3, "m2l": 4}[what]))

    def traverse(self, conventional=False):
        """The hybrid walk of Sec. 2.3 on the k-d boxes, or (conventional=True) the
        conventional FMM's: the opening-angle test alone, from (root, root) of the
        primary box."""
        if conventional:
            _check(lib().orc_kd_traverse_conventional(self._c), "kd_traverse_conventional")
        else:
            _check(lib().orc_kd_traverse(self._c), "kd_traverse")

    def counts(self):
        """Interaction counts of the current lists (Sec. 3): M2L cell pairs, P2P leaf
        pairs, and particle pairs on the P2P lists (sum of n_sink n_source)."""
        nodes, _, _ = self.tree()
        p2p, m2l = self.lists()
        cnt = nodes[:, 2]
        pp = int((cnt[p2p[:, 0]] * cnt[p2p[:, 1]]).sum()) if len(p2p) else 0
        return {"m2l": len(m2l), "p2p": len(p2p), "p2p_particle_pairs": pp}

    def forces(self) -> np.ndarray:
        acc = np.zeros((3, self.n))
        _check(lib().orc_kd_forces(self._c, _p(acc)), "kd_forces")
        return acc

    def tree(self):
        """(nodes [nnodes][5] int64: level, first, count, first child or -1, split axis or -1;
        boxes [nnodes][6] float64: lo xyz, hi xyz; perm [n] int64: input index in tree order)."""
        k = self.size("nodes")
        nodes = np.zeros((k, 5), dtype=np.int64)
        boxes = np.zeros((k, 6))
        perm = np.zeros(self.n, dtype=np.int64)
        lib().orc_kd_export(self._c, _p(nodes), _p(boxes), _p(perm))
        return nodes, boxes, perm

    def lists(self):
        p2p = np.zeros((self.size("p2p"), 3), dtype=np.int64)
        m2l = np.zeros((self.size("m2l"), 3), dtype=np.int64)
        lib().orc_kd_export_list(self._c, 0, _p(p2p))
        lib().orc_kd_export_list(self._c, 1, _p(m2l))
        return p2p, m2l

    def forces_given_lists(self, p2p, m2l):
        p2p = np.ascontiguousarray(p2p, dtype=np.int64).reshape(-1, 3)
        m2l = np.ascontiguousarray(m2l, dtype=np.int64).reshape(-1, 3)
        _check(lib().orc_kd_set_lists(self._c, _p(p2p), len(p2p), _p(m2l), len(m2l)), "kd_set_lists")
        acc = np.zeros((3, self.n))
        _check(lib().orc_kd_forces_given_lists(self._c, _p(acc)), "kd_forces_given_lists")
        return acc
