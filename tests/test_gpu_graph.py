"""Graph mode: the whole short-range call (upward pass, the walk, list
grouping, M2L, L2L/L2P, P2P) captured as one CUDA graph gives the same forces
and the same lists, bit for bit, as direct launches; repeated calls update the
executable graph in place; a different particle set re-captures it; when a
list outgrows its capacity inside the graph the call runs again directly and
still gives the same result."""
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


def same_lists(a, b):
    for what in ("p2p", "m2l"):
        np.testing.assert_array_equal(a.export(what), b.export(what))


@pytest.mark.parametrize("order", [4, 6])
def test_graph_mode_is_bit_identical(order):
    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(50000, 50, 0.7, 61)
    direct = hfmm.Solver(pm_grid=32, theta=0.4, order=order)
    graph = hfmm.Solver(pm_grid=32, theta=0.4, order=order, use_graph=1, profile=1)
    ref = run(direct, pos, mass)
    for _ in range(3):  # first call instantiates, later ones update in place
        np.testing.assert_array_equal(run(graph, pos, mass), ref)
        same_lists(graph, direct)
    st, sd = graph.get_stats(), direct.get_stats()
    assert st["t_upward"] > 0 and st["t_p2p"] == -1 and st["t_traverse"] == -1  # timed as a whole
    assert st["nm2l"] == sd["nm2l"] and st["np2p"] == sd["np2p"] and st["traverse_walks"] == 1
    # another set: new sizes, new capture
    pos2, mass2 = W.uniform(30001, 62)
    np.testing.assert_array_equal(run(graph, pos2, mass2), run(direct, pos2, mass2))
    same_lists(graph, direct)


def test_graph_mode_falls_back_when_a_list_overflows():
    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(40000, 50, 0.7, 63)
    direct = hfmm.Solver(pm_grid=32, theta=0.5, order=4)
    ref = run(direct, pos, mass)
    graph = hfmm.Solver(pm_grid=32, theta=0.5, order=4, use_graph=1, list_init=256)
    np.testing.assert_array_equal(run(graph, pos, mass), ref)  # overflow in the graph, then direct
    assert graph.get_stats()["traverse_walks"] > 1
    np.testing.assert_array_equal(run(graph, pos, mass), ref)  # the grown lists fit: the graph alone
    assert graph.get_stats()["traverse_walks"] == 1
    same_lists(graph, direct)
    # a larger set than the capacities were grown for
    pos3, mass3 = W.nfw_clustered(120000, 80, 0.8, 64)
    np.testing.assert_array_equal(run(graph, pos3, mass3), run(direct, pos3, mass3))
