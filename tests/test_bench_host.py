"""Host logic of bench.py: the count of tensor-core flops the FP32 factorisation issues,
against schedules counted by hand (no GPU)."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHUNK = 12 * 2 * 128 * 128 * 8   # one 32-column chunk of a 128 x 128 tile, split TF32


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Fronts:
    """Stands in for a context: one Oseen system with the given fronts (m, p, children)."""

    def __init__(self, rows):
        self.rows = np.array(rows, np.int32)

    def front_table(self, j):
        return self.rows if j == 0 else None


def test_small_front_tiles():
    # m = 200, p = 100, one CTA: after the pivot blocks ending at 32, 64, 96, 100 the trailing
    # orders 168, 136, 104, 100 take 2 x 2, 2 x 2, 1 and 1 tiles of one chunk each
    f = _Fronts([[200, 100, 0, -1, 0, -1, -1]])
    assert _bench().issued_tensor_flops(f) == 10 * CHUNK


def test_large_front_schedule():
    # m = 600, p = 300 (order >= 256): groups [0, 128), [128, 256), [256, 300)
    #   group 0, blocks 0, 32, 64: panels 5 + 4, 5 + 4, 4 + 4 tiles; after block 96: strips
    #     4 x 2 + 2 x 3 tiles of 4 chunks
    #   group 1, blocks 128, 160, 192: 4 + 3, 4 + 3, 3 + 3; after block 224: 3 x 1 + 1 x 3 tiles
    #     of 4 chunks
    #   group 2, block 256: 3 + 3; block 288 ends the pivots (12 columns): nothing
    #   Schur block [300, 600): 3 x 3 tiles of 10 chunks
    units = 9 + 9 + 8 + 14 * 4 + 7 + 7 + 6 + 6 * 4 + 6 + 9 * 10
    f = _Fronts([[600, 300, 0, -1, 0, -1, -1]])
    assert _bench().issued_tensor_flops(f) == units * CHUNK


def test_ancestor_of_a_large_front_takes_the_large_path():
    # a parent of order 200 above a child of order 300 is factored by the large-front path too
    child = [300, 100, 0, 1, 0, -1, -1]
    parent = [200, 200, 1, -1, 1, 0, -1]
    b = _bench()
    both = b.issued_tensor_flops(_Fronts([child, parent]))
    alone = b.issued_tensor_flops(_Fronts([child]))
    # parent, large path (m = p = 200): group 0 panels after blocks 0, 32, 64: 2 + 1, 2 + 1,
    # 1 + 1 tiles (trailing orders 168, 136, 104; row panels [128, 200)); after block 96 the
    # strip rows and columns [128, 200), one tile of 4 chunks; group 1 ends at the front's
    # order, so after blocks 128, 160 only the column panels (1 tile each; block 192 ends the
    # pivots); no Schur block
    parent_units = 3 + 3 + 2 + 1 * 4 + 1 + 1
    assert both - alone == parent_units * CHUNK
