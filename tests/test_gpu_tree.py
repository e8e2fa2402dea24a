"""The quadtree of Sec. 2.1 / Remark (tree) built on the device (Morton keys,
the library's own stable radix sort, the breadth-first box table) against the
oracle's tree (lexsort and a host breadth-first split): the point order and
every box must agree exactly (integer work, bit-exact)."""
import numpy as np
import pytest

from oracle.tree import Tree as OTree
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_08057_gb300 import build
    build.build()
    from paper_1603_08057_gb300 import binding
    return binding


def _cases():
    yield "uniform 100000", W.uniform(100000, 1001)
    yield "mixture 262144", W.mixture(262144, 3)
    yield "grid 256^2", W.grid(256)
    yield "one point", W.uniform(1, 1002)
    yield "65 points", W.uniform(65, 1003)
    # duplicates: 200 copies of one location split down to the deepest level
    x = W.uniform(3000, 1004)
    x[:200] = x[0]
    yield "duplicates", x
    # a ragged tail of radix tiles (2048 per tile) and ties across tiles
    x = np.repeat(W.uniform(1500, 1005), 3, axis=0)
    yield "repeated points", x


@pytest.mark.parametrize("name,x", list(_cases()), ids=[c[0] for c in _cases()])
def test_tree_matches_oracle_exactly(B, name, x):
    t = B.Tree(torch.tensor(x, dtype=torch.float64, device="cuda"))
    perm, boxes = t.export()
    ref = OTree(x, 64)
    np.testing.assert_array_equal(perm, ref.perm)
    assert boxes.shape[0] == len(ref.level)
    np.testing.assert_array_equal(boxes[:, 0], ref.level)
    np.testing.assert_array_equal(boxes[:, 1], ref.start)
    np.testing.assert_array_equal(boxes[:, 2], ref.count)
    np.testing.assert_array_equal(boxes[:, 3], ref.parent)
    np.testing.assert_array_equal(boxes[:, 4], ref.slot)
    assert np.all(boxes[:, 5] == 0)
