"""The kick-drift-kick step as one CUDA graph (use_graph): positions,
velocities and accelerations identical, bit for bit, to the step run by direct
launches; later steps replay the graph without capturing it again; when the
tree (its node or level capacity) or a list outgrows its capacity inside the
graph, the step goes on directly from the drifted positions and still gives the
same result."""
import numpy as np
import pytest

from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a, dt):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def start(s, pos, mass, vel):
    """Device state with acc = total acceleration at pos (what hfmm_step expects)."""
    p, m, v = dev(pos, np.float64), dev(mass, np.float32), dev(vel, np.float32)
    s.build_tree(p, m)
    a = s.short_range_forces()
    s.pm_long_range(a)
    return p, m, v, a


def steps(s, state, k, dt):
    import torch

    p, m, v, a = state
    for _ in range(k):
        s.step(p, v, a, dt)
    torch.cuda.synchronize()
    return p.cpu().numpy(), v.cpu().numpy(), a.cpu().numpy()


def assert_same(out, ref):
    for x, y in zip(out, ref):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("order", [4, 6])
def test_step_graph_is_bit_identical_and_replays_without_capture(order):
    from paper_2006_14952_gb300 import hfmm

    rng = np.random.default_rng(70)
    pos, mass = W.nfw_clustered(40000, 40, 0.7, 71)
    vel = 0.05 * rng.normal(size=(3, pos.shape[1]))
    kw = dict(pm_grid=32, theta=0.4, order=order)
    direct = hfmm.Solver(**kw)
    graph = hfmm.Solver(use_graph=1, **kw)
    sd, sg = start(direct, pos, mass, vel), start(graph, pos, mass, vel)
    c0 = graph.get_stats()["graph_captures"]
    assert_same(steps(graph, sg, 4, 2e-3), steps(direct, sd, 4, 2e-3))
    st, s0 = graph.get_stats(), direct.get_stats()
    assert st["step_graphs"] == 4 and s0["step_graphs"] == 0
    assert st["graph_captures"] - c0 < 4  # at least one step replayed the graph as it was
    assert st["nnodes"] == s0["nnodes"] and st["nlevels"] == s0["nlevels"]
    assert st["np2p"] == s0["np2p"] and st["nm2l"] == s0["nm2l"]
    for what in ("p2p", "m2l"):
        np.testing.assert_array_equal(graph.export(what), direct.export(what))


def test_step_graph_falls_back_when_the_tree_outgrows_its_capacities():
    """A uniform start (a shallow tree) and velocities that gather every particle
    into a ball 100 times smaller within one drift: the new tree is several
    levels deeper than the last one plus two, so the graph's tree overflows and
    the step is finished directly; the next step captures a graph for the deep
    tree and runs it."""
    from paper_2006_14952_gb300 import hfmm

    n, dt = 30000, 1e-2
    pos, mass = W.uniform(n, 72)
    target = 0.5 + 0.01 * (pos - 0.5)
    vel = (target - pos) / dt
    kw = dict(pm_grid=32, theta=0.5, order=4)
    direct = hfmm.Solver(**kw)
    graph = hfmm.Solver(use_graph=1, **kw)
    sd, sg = start(direct, pos, mass, vel), start(graph, pos, mass, vel)
    shallow = graph.get_stats()["nlevels"]
    assert_same(steps(graph, sg, 1, dt), steps(direct, sd, 1, dt))
    st = graph.get_stats()
    assert st["step_graphs"] == 1 and st["nlevels"] >= shallow + 3
    assert st["nlevels"] == direct.get_stats()["nlevels"]
    assert_same(steps(graph, sg, 1, 1e-4), steps(direct, sd, 1, 1e-4))
    assert graph.get_stats()["step_graphs"] == 2


def test_step_graph_falls_back_when_a_list_overflows():
    """List capacities grown on a small set (list_init makes them start tiny),
    then a step on a clustered set 15 times larger: the walk inside the graph
    overflows, the step is finished directly (the walk grows the lists and
    repeats), and the next step runs as one graph with the grown lists."""
    from paper_2006_14952_gb300 import hfmm

    rng = np.random.default_rng(73)
    pos, mass = W.nfw_clustered(30000, 30, 0.7, 74)
    vel = 0.05 * rng.normal(size=(3, pos.shape[1]))
    kw = dict(pm_grid=32, theta=0.5, order=4)
    direct = hfmm.Solver(**kw)
    graph = hfmm.Solver(use_graph=1, list_init=256, **kw)
    sp, sm = W.uniform(2000, 77)
    graph.build_tree(dev(sp, np.float64), dev(sm, np.float32))
    graph.short_range_forces()
    sd = start(direct, pos, mass, vel)
    pg, mg, vg = dev(pos, np.float64), dev(mass, np.float32), dev(vel, np.float32)
    graph.build_tree(pg, mg)
    sg = (pg, mg, vg, sd[3].clone())  # the same starting accelerations
    assert_same(steps(graph, sg, 1, 2e-3), steps(direct, sd, 1, 2e-3))
    st = graph.get_stats()
    assert st["step_graphs"] == 1 and st["traverse_walks"] > 1
    assert_same(steps(graph, sg, 1, 2e-3), steps(direct, sd, 1, 2e-3))
    st = graph.get_stats()
    assert st["step_graphs"] == 2 and st["traverse_walks"] == 1


def test_step_graph_profile_times_the_whole_step():
    from paper_2006_14952_gb300 import hfmm

    rng = np.random.default_rng(75)
    pos, mass = W.nfw_clustered(20000, 20, 0.7, 76)
    vel = 0.05 * rng.normal(size=(3, pos.shape[1]))
    graph = hfmm.Solver(pm_grid=32, theta=0.5, order=4, use_graph=1, profile=1)
    sg = start(graph, pos, mass, vel)
    steps(graph, sg, 2, 2e-3)
    st = graph.get_stats()
    assert st["step_graphs"] == 2
    assert st["t_upward"] > 0 and st["t_tree"] == -1 and st["t_keys_sort"] == -1 and st["t_p2p"] == -1
