"""Graph mode: the post-traversal sequence captured as one CUDA graph gives the
same forces, bit for bit, as direct launches; repeated calls update the
executable graph in place; a different particle set re-captures it."""
import numpy as np
import pytest

from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(s, pos, mass, acc=None):
    import torch

    s.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
    a = s.short_range_forces(acc)
    torch.cuda.synchronize()
    return a.cpu().numpy()


@pytest.mark.parametrize("order", [4, 6])
def test_graph_mode_is_bit_identical(order):
    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(50000, 50, 0.7, 61)
    direct = hfmm.Solver(pm_grid=32, theta=0.4, order=order)
    graph = hfmm.Solver(pm_grid=32, theta=0.4, order=order, use_graph=1, profile=1)
    ref = run(direct, pos, mass)
    for _ in range(3):  # first call instantiates, later ones update in place
        np.testing.assert_array_equal(run(graph, pos, mass), ref)
    st = graph.get_stats()
    assert st["t_lists"] > 0 and st["t_p2p"] == -1  # the graph is timed as a whole
    # another set: new sizes, new capture
    pos2, mass2 = W.uniform(30001, 62)
    np.testing.assert_array_equal(run(graph, pos2, mass2), run(direct, pos2, mass2))
