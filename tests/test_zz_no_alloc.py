"""The allocation-free Morton sort (hfmm_morton_sort_noalloc), called through
the C ABI, against the keys and permutation of hfmm_build_tree on the same
input.  Two calls in a row with different inputs check that the shared fixed
scratch array carries nothing over from one call to the next.  Some callers
of this library cannot allocate device memory when they call it (a runtime
that owns all GPU memory, or code that must avoid the synchronisation an
allocation may cause); this entry point serves them."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2006_14952_gb300 import hfmm

    L = hfmm.load()
    f = L.hfmm_morton_sort_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return hfmm, f


def _reference(hfmm, pos_np, mass_np):
    import torch

    s = hfmm.Solver(pm_grid=32)
    s.build_tree(torch.from_numpy(pos_np).cuda(), torch.from_numpy(mass_np).cuda())
    torch.cuda.synchronize()
    return s.export("keys"), s.export("perm")


def test_noalloc_sort_matches_build_tree_twice_in_a_row():
    import torch

    from paper_2006_14952_gb300 import workloads as W

    hfmm, f = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    inputs = [W.nfw_clustered(300001, 40, 0.7, 77), W.uniform(123457, 78)]
    inputs[0][0][:, :3] = [[-0.25, 1.0, 2.5], [0.0, 0.999999999, -1e-18], [1.0 - 1e-17, 0.5, 3.0]]
    for pos, mass in inputs:
        n = pos.shape[1]
        dpos = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rc = f(ctypes.c_void_p(dpos.data_ptr()), n, 1.0, ctypes.c_void_p(keys.data_ptr()),
               ctypes.c_void_p(perm.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        ref_keys, ref_perm = _reference(hfmm, np.ascontiguousarray(pos), mass)
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), ref_keys)
        np.testing.assert_array_equal(perm.cpu().numpy().view(np.uint32), ref_perm)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    hfmm, f = _lib()
    assert f(None, 524288 + 1, 1.0, None, None, None) == -4  # HFMM_ERR_CAPACITY
    assert f(None, -1, 1.0, None, None, None) == -1
    assert f(None, 0, 1.0, None, None, None) == 0
