"""Pins of the tree geometry (Sec. 3.1)."""
import pytest

from oracle.tree import Tree


def test_shapes_4x4_m8():
    t = Tree(16, 8)
    shapes = sorted(set(t.shape))
    assert [t.shape.count(s) for s in [(2, 2, 4), (4, 4, 8), (8, 8, 8)]] == [8, 4, 2]
    assert t.nL == 3 and t.n_nodes == 14


def test_shapes_32x32_m128():
    t = Tree(1024, 128)
    from collections import Counter
    c = Counter(t.shape)
    assert c[(2, 2, 4)] == 512 and c[(4, 4, 16)] == 256 and c[(16, 16, 128)] == 128
    assert c[(128, 128, 128)] == 126


@pytest.mark.parametrize("N,m", [(16, 8), (64, 32), (256, 64)])
def test_regions_partition_sites(N, m):
    t = Tree(N, m)
    for n in range(t.n_nodes):
        regs = [t.region(n, s) for s in range(3)]
        assert sum(len(r) for r in regs) == N
        assert set().union(*regs) == set(range(N))


def test_post_order_and_paths():
    t = Tree(64, 16)
    order = t.post_order()
    assert sorted(order) == list(range(t.n_nodes))
    t0, t1 = t.top_nodes()
    assert order.index(t0) == t.n_nodes // 2 - 1 and order[-1] == t1
    for a, b in zip(order[:-1], order[1:]):
        p = t.path(a, b)
        for x, y in zip(p[:-1], p[1:]):
            t.slot_towards(x, y)  # adjacent
