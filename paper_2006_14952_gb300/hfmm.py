"""ctypes binding of libhfmm.so (include/hfmm.h).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step of the solver runs in the library's CUDA kernels.
There is no CPU fallback: if the library has not been built, or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

HFMM_OK = 0
ERRORS = {-1: "HFMM_ERR_ARG", -2: "HFMM_ERR_OOM", -3: "HFMM_ERR_CUDA", -4: "HFMM_ERR_CAPACITY",
          -5: "HFMM_ERR_STATE", -6: "HFMM_ERR_TIMEOUT"}
EXPORT = {"keys": 0, "perm": 1, "nodes": 2, "p2p": 3, "m2l": 4, "multipoles": 5, "locals": 6, "m2l_order": 7,
          "candidates": 8, "kd_nodes": 9, "kd_boxes": 10}
MLP_WEIGHTS = 5512

# Every symbol include/hfmm.h declares.
SYMBOLS = ["hfmm_default_params", "hfmm_create", "hfmm_destroy", "hfmm_last_error", "hfmm_build_tree",
           "hfmm_short_range_forces", "hfmm_short_range_forces_host", "hfmm_get_stats", "hfmm_export",
           "hfmm_load_mlp", "hfmm_collect_training_pairs", "hfmm_mlp_infer", "hfmm_mlp_grad", "hfmm_mlp_adam",
           "hfmm_morton_sort_noalloc", "hfmm_pm_long_range", "hfmm_step", "hfmm_interaction_counts",
           "hfmm_alu_peak"]


class Params(C.Structure):
    _fields_ = [("box", C.c_double), ("pm_grid", C.c_int), ("rs_cells", C.c_double), ("rcut_rs", C.c_double),
                ("G", C.c_double), ("theta", C.c_double), ("order", C.c_int), ("leaf_max", C.c_int),
                ("mac_mode", C.c_int), ("transition_rule", C.c_int), ("size_rule", C.c_int),
                ("m2l_precision", C.c_int), ("profile", C.c_int), ("m2l_tables", C.c_int),
                ("tile_p2p_stage", C.c_int), ("tile_p2p_blocks", C.c_int), ("tile_m2l_blocks", C.c_int),
                ("tile_trav_blocks", C.c_int), ("use_graph", C.c_int), ("tc_wait_polls", C.c_int),
                ("split", C.c_int), ("p2p_mutual", C.c_int), ("list_init", C.c_int),
                ("sink_batches", C.c_int), ("tree", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnodes", C.c_int64), ("nleaves", C.c_int64), ("nlevels", C.c_int32),
                ("traverse_iters", C.c_int32), ("np2p", C.c_int64), ("nm2l", C.c_int64),
                ("p2p_particle_pairs", C.c_int64), ("p2p_useful_pairs", C.c_int64), ("launches", C.c_int64),
                ("t_keys_sort", C.c_float), ("t_tree", C.c_float),
                ("t_upward", C.c_float), ("t_traverse", C.c_float), ("t_lists", C.c_float), ("t_m2l", C.c_float),
                ("t_l2l", C.c_float), ("t_p2p", C.c_float), ("nm2l_table", C.c_int64), ("frontier_pairs", C.c_int64),
                ("traverse_walks", C.c_int64), ("step_graphs", C.c_int64), ("graph_captures", C.c_int64),
                ("sink_batches", C.c_int64)]


class HfmmError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhfmm.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise HfmmError(f"{path} is missing: build it with paper_2006_14952_gb300.build.build()")
            _build.build()
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        L.hfmm_default_params.argtypes = [C.POINTER(Params)]
        L.hfmm_default_params.restype = None
        L.hfmm_create.argtypes = [C.POINTER(Params), C.POINTER(vp)]
        L.hfmm_create.restype = i32
        L.hfmm_destroy.argtypes = [vp]
        L.hfmm_destroy.restype = None
        L.hfmm_last_error.argtypes = [vp]
        L.hfmm_last_error.restype = C.c_char_p
        L.hfmm_build_tree.argtypes = [vp, vp, vp, i64, vp]
        L.hfmm_build_tree.restype = i32
        L.hfmm_short_range_forces.argtypes = [vp, vp, vp]
        L.hfmm_short_range_forces.restype = i32
        L.hfmm_short_range_forces_host.argtypes = [vp, vp, vp, i64, vp, vp]
        L.hfmm_short_range_forces_host.restype = i32
        L.hfmm_pm_long_range.argtypes = [vp, vp, vp]
        L.hfmm_pm_long_range.restype = i32
        L.hfmm_step.argtypes = [vp, vp, vp, vp, C.c_double, vp]
        L.hfmm_step.restype = i32
        L.hfmm_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.hfmm_get_stats.restype = i32
        L.hfmm_export.argtypes = [vp, i32, vp, C.POINTER(C.c_size_t)]
        L.hfmm_export.restype = i32
        L.hfmm_load_mlp.argtypes = [vp, vp, C.c_size_t]
        L.hfmm_load_mlp.restype = i32
        L.hfmm_collect_training_pairs.argtypes = [vp, i64, C.c_uint32, vp, vp, C.POINTER(i64), vp]
        L.hfmm_collect_training_pairs.restype = i32
        L.hfmm_mlp_infer.argtypes = [vp, vp, i64, vp, vp, vp]
        L.hfmm_mlp_infer.restype = i32
        L.hfmm_mlp_grad.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.hfmm_mlp_grad.restype = i32
        L.hfmm_mlp_adam.argtypes = [vp, C.c_float, i32, vp, vp, vp, vp, vp]
        L.hfmm_mlp_adam.restype = i32
        L.hfmm_interaction_counts.argtypes = [vp, i32, C.POINTER(i64), vp]
        L.hfmm_interaction_counts.restype = i32
        L.hfmm_alu_peak.argtypes = [i32, i32, vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.hfmm_alu_peak.restype = i32
        _lib = L
        return L


def default_params() -> Params:
    p = Params()
    load().hfmm_default_params(C.byref(p))
    return p


def _stream_handle(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def mlp_infer(weights_bf16, x, stream=None):
    """Network logits [n][8] and classes [n] (CUDA tensors in, CUDA tensors out)."""
    import torch

    n = x.shape[0]
    logits = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    cls = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = load().hfmm_mlp_infer(C.c_void_p(weights_bf16.data_ptr()), C.c_void_p(x.data_ptr()), n,
                               C.c_void_p(logits.data_ptr()), C.c_void_p(cls.data_ptr()), _stream_handle(stream))
    if rc != HFMM_OK:
        raise HfmmError(f"hfmm_mlp_infer: {ERRORS.get(rc, rc)}")
    return logits, cls


ALU_KINDS = {"ffma": 0, "ffma2": 1, "ex2": 2, "rsqrt": 3}


def alu_peak(kind: str, iters: int = 4096, stream=None):
    """Measured throughput of one ALU instruction kind over the whole GPU:
    (rate, ms); rate in flop/s for "ffma"/"ffma2", operations/s for "ex2"/"rsqrt"."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    scratch = torch.empty(2048 * sms, dtype=torch.float32, device="cuda")
    rate, ms = C.c_double(0.0), C.c_double(0.0)
    rc = load().hfmm_alu_peak(ALU_KINDS[kind], int(iters), C.c_void_p(scratch.data_ptr()), C.byref(rate),
                              C.byref(ms), _stream_handle(stream))
    if rc != HFMM_OK:
        raise HfmmError(f"hfmm_alu_peak: {ERRORS.get(rc, rc)}")
    return rate.value, ms.value


def mlp_adam(grad, lr, step, weights, m1, m2, weights_bf16=None, stream=None):
    wb = C.c_void_p(weights_bf16.data_ptr()) if weights_bf16 is not None else None
    rc = load().hfmm_mlp_adam(C.c_void_p(grad.data_ptr()), float(lr), int(step), C.c_void_p(weights.data_ptr()),
                              C.c_void_p(m1.data_ptr()), C.c_void_p(m2.data_ptr()), wb, _stream_handle(stream))
    if rc != HFMM_OK:
        raise HfmmError(f"hfmm_mlp_adam: {ERRORS.get(rc, rc)}")


class Solver:
    """One hfmm context: build_tree, short_range_forces, get_stats, export."""

    def __init__(self, **kw):
        self._lib = load()
        p = default_params()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        h = C.c_void_p()
        rc = self._lib.hfmm_create(C.byref(p), C.byref(h))
        if rc != HFMM_OK:
            raise HfmmError(f"hfmm_create: {ERRORS.get(rc, rc)}: {self._lib.hfmm_last_error(None).decode()}")
        self._h = h
        self.n = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hfmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != HFMM_OK:
            msg = self._lib.hfmm_last_error(self._h).decode()
            raise HfmmError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")

    @property
    def rs(self) -> float:
        p = self.params
        return p.rs_cells * (p.box / p.pm_grid)

    @property
    def rc(self) -> float:
        return self.params.rcut_rs * self.rs

    def build_tree(self, pos, mass, stream=None):
        """pos: CUDA float64 [3][n] contiguous; mass: CUDA float32 [n]."""
        import torch

        assert pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous() and pos.shape[0] == 3
        assert mass.is_cuda and mass.dtype == torch.float32 and mass.is_contiguous()
        n = pos.shape[1]
        assert mass.shape[0] == n
        self.n = n
        self._check(self._lib.hfmm_build_tree(self._h, C.c_void_p(pos.data_ptr()), C.c_void_p(mass.data_ptr()), n,
                                              _stream_handle(stream)), "hfmm_build_tree")

    def short_range_forces(self, acc=None, stream=None):
        """Returns (or fills) a CUDA float32 [3][n] tensor of accelerations."""
        import torch

        if acc is None:
            acc = torch.empty((3, self.n), dtype=torch.float32, device="cuda")
        assert acc.is_cuda and acc.dtype == torch.float32 and acc.is_contiguous()
        self._check(self._lib.hfmm_short_range_forces(self._h, C.c_void_p(acc.data_ptr()), _stream_handle(stream)),
                    "hfmm_short_range_forces")
        return acc

    def pm_long_range(self, acc=None, stream=None):
        """Adds the long-range (PM) accelerations into a CUDA float32 [3][n] tensor (zeros if None)."""
        import torch

        if acc is None:
            acc = torch.zeros((3, self.n), dtype=torch.float32, device="cuda")
        assert acc.is_cuda and acc.dtype == torch.float32 and acc.is_contiguous()
        self._check(self._lib.hfmm_pm_long_range(self._h, C.c_void_p(acc.data_ptr()), _stream_handle(stream)),
                    "hfmm_pm_long_range")
        return acc

    def step(self, pos, vel, acc, dt, stream=None):
        """One KDK step in place: pos CUDA float64 [3][n]; vel, acc CUDA float32 [3][n]
        (acc must hold the total acceleration at pos on entry)."""
        import torch

        assert pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()
        for t in (vel, acc):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.shape == pos.shape
        self._check(self._lib.hfmm_step(self._h, C.c_void_p(pos.data_ptr()), C.c_void_p(vel.data_ptr()),
                                        C.c_void_p(acc.data_ptr()), float(dt), _stream_handle(stream)), "hfmm_step")

    def short_range_forces_host(self, pos, mass, acc=None, stream=None):
        """Host numpy (or pinned CPU torch) buffers in and out."""
        n = pos.shape[1]
        if acc is None:
            acc = np.empty((3, n), dtype=np.float32)
        ptr = (lambda a: C.c_void_p(a.data_ptr())) if hasattr(pos, "data_ptr") else (
            lambda a: a.ctypes.data_as(C.c_void_p))
        self.n = n
        self._check(self._lib.hfmm_short_range_forces_host(self._h, ptr(pos), ptr(mass), n, ptr(acc),
                                                           _stream_handle(stream)), "hfmm_short_range_forces_host")
        return acc

    def get_stats(self) -> dict:
        s = Stats()
        self._check(self._lib.hfmm_get_stats(self._h, C.byref(s)), "hfmm_get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def interaction_counts(self, conventional=False, stream=None) -> dict:
        """Kernel counts of Sec. 3 on the current tree: the hybrid walk, or the
        conventional FMM's (opening-angle test alone, primary box)."""
        out = (C.c_int64 * 4)()
        self._check(self._lib.hfmm_interaction_counts(self._h, 1 if conventional else 0, out,
                                                      _stream_handle(stream)), "hfmm_interaction_counts")
        return {"m2l": out[0], "p2p": out[1], "p2p_particle_pairs": out[2], "frontier_pairs": out[3]}

    def load_mlp(self, weights_bf16):
        """weights_bf16: numpy uint16 [5512] holding BF16 bit patterns."""
        w = np.ascontiguousarray(weights_bf16, dtype=np.uint16)
        assert w.size == MLP_WEIGHTS
        self._check(self._lib.hfmm_load_mlp(self._h, w.ctypes.data_as(C.c_void_p), w.nbytes), "hfmm_load_mlp")

    def collect_training_pairs(self, max_pairs, sample_mod=1, stream=None):
        """Features [n][12] and M2L errors at orders 2..8 [n][7] (CUDA float32 tensors)."""
        import torch

        feat = torch.empty((max_pairs, 12), dtype=torch.float32, device="cuda")
        err = torch.empty((max_pairs, 7), dtype=torch.float32, device="cuda")
        cnt = C.c_int64(0)
        self._check(self._lib.hfmm_collect_training_pairs(self._h, max_pairs, sample_mod,
                                                          C.c_void_p(feat.data_ptr()), C.c_void_p(err.data_ptr()),
                                                          C.byref(cnt), _stream_handle(stream)),
                    "hfmm_collect_training_pairs")
        return feat[:cnt.value], err[:cnt.value]

    def mlp_grad(self, weights, x, labels, class_weights=None, stream=None):
        """Gradient and loss of the mean cross-entropy (CUDA tensors)."""
        import torch

        grad = torch.empty(MLP_WEIGHTS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        cw = C.c_void_p(class_weights.data_ptr()) if class_weights is not None else None
        self._check(self._lib.hfmm_mlp_grad(self._h, C.c_void_p(weights.data_ptr()), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(labels.data_ptr()), cw, x.shape[0], C.c_void_p(grad.data_ptr()),
                                            C.c_void_p(loss.data_ptr()), _stream_handle(stream)), "hfmm_mlp_grad")
        return grad, loss

    def export(self, what: str) -> np.ndarray:
        code = EXPORT[what]
        nb = C.c_size_t(0)
        self._check(self._lib.hfmm_export(self._h, code, None, C.byref(nb)), "hfmm_export")
        dtype, cols = {"keys": (np.uint64, 0), "perm": (np.uint32, 0), "nodes": (np.int64, 8), "p2p": (np.int64, 3),
                       "m2l": (np.int64, 3), "multipoles": (np.float32, -1), "locals": (np.float32, -1),
                       "m2l_order": (np.int64, 0), "candidates": (np.int64, 3), "kd_nodes": (np.int64, 5),
                       "kd_boxes": (np.float64, 6)}[what]
        out = np.empty(nb.value // np.dtype(dtype).itemsize, dtype=dtype)
        if nb.value:
            self._check(self._lib.hfmm_export(self._h, code, out.ctypes.data_as(C.c_void_p), C.byref(nb)),
                        "hfmm_export")
        if cols > 0:
            out = out.reshape(-1, cols)
        elif cols < 0:
            nc = (self.params.order + 1) * (self.params.order + 2) * (self.params.order + 3) // 6
            out = out.reshape(-1, nc)
        return out
