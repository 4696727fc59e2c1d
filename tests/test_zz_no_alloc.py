"""The allocation-free Morton sort (hfmm_morton_sort_noalloc), called through
the C ABI, against the keys and permutation of hfmm_build_tree on the same
input and against the FP64 oracle's keys.  Calls in a row with different
inputs check that the shared fixed scratch array carries nothing over from one
call to the next; one call uses exactly the largest size the array holds and a
box side that is not a power of two (the exact-division path of the wrap).
Some callers of this library cannot allocate device memory when they call it
(a runtime that owns all GPU memory, or code that must avoid the
synchronisation an allocation may cause); this entry point serves them."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

MAX_N = 524288  # HFMM_NOALLOC_MAX_N


def _lib():
    from paper_2006_14952_gb300 import hfmm

    L = hfmm.load()
    f = L.hfmm_morton_sort_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return hfmm, f


def _reference(hfmm, pos_np, mass_np, box):
    import torch

    s = hfmm.Solver(pm_grid=32, box=box)
    s.build_tree(torch.from_numpy(pos_np).cuda(), torch.from_numpy(mass_np).cuda())
    torch.cuda.synchronize()
    return s.export("keys"), s.export("perm")


def _inputs():
    from paper_2006_14952_gb300 import workloads as W

    a = W.nfw_clustered(300001, 40, 0.7, 77)
    a[0][:, :3] = [[-0.25, 1.0, 2.5], [0.0, 0.999999999, -1e-18], [1.0 - 1e-17, 0.5, 3.0]]
    b = W.uniform(123457, 78)
    # the largest size, box side 3 (not a power of two), some positions outside [0, 3)
    pos, mass = W.nfw_clustered(MAX_N, 60, 0.6, 79)
    pos = pos * 3.0
    rng = np.random.default_rng(80)
    out = rng.choice(MAX_N, 2000, replace=False)
    pos[:, out] += rng.integers(-2, 3, (3, 2000)) * 3.0 + rng.uniform(-0.5, 0.5, (3, 2000))
    pos[:, out[:3]] = [[3.0, -3.0, 6.0 - 1e-15], [0.0, 3.0 - 1e-16, -1e-300], [2.9999999999999996, 9.0, -6.0]]
    return [(a[0], a[1], 1.0), (b[0], b[1], 1.0), (pos, mass, 3.0), (b[0], b[1], 1.0)]


def test_noalloc_sort_matches_build_tree_and_oracle_on_calls_in_a_row():
    import torch

    hfmm, f = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for pos, mass, box in _inputs():
        pos = np.ascontiguousarray(pos)
        n = pos.shape[1]
        dpos = torch.from_numpy(pos).cuda()
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rc = f(ctypes.c_void_p(dpos.data_ptr()), n, box, ctypes.c_void_p(keys.data_ptr()),
               ctypes.c_void_p(perm.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got_keys, got_perm = keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32)
        ref_keys, ref_perm = _reference(hfmm, pos, mass, box)
        np.testing.assert_array_equal(got_keys, ref_keys)
        np.testing.assert_array_equal(got_perm, ref_perm)
        o = oracle.FMM(box=box, rs=0.01 * box, rc=0.045 * box, leaf_max=16)
        o.build_tree(pos, mass)
        okey, operm, _ = o.particles()
        np.testing.assert_array_equal(got_keys, okey)
        np.testing.assert_array_equal(got_perm.astype(np.int64), operm)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    hfmm, f = _lib()
    assert f(None, MAX_N + 1, 1.0, None, None, None) == -4  # HFMM_ERR_CAPACITY
    assert f(None, -1, 1.0, None, None, None) == -1
    assert f(None, 0, 1.0, None, None, None) == 0
