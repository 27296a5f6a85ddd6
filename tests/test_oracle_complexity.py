"""Pin of the operation counts against the numbers Table 2 prints (Sec. III-B)."""
import json
import os

from oracle import complexity as cx

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_complexity.json")))


def test_table2_operation_counts():
    n = GOLD["n"]
    assert round(cx.flashmp_flops(n) / 1e9, 2) == GOLD["flashmp_ops_G"]
    assert round(cx.direct_flops(n) / 1e9, 1) == GOLD["direct_ops_G"]
    assert round(cx.direct_bytes(n) / 1e9, 1) == GOLD["direct_memory_GB"]


def test_boundary_rank_counts():
    # Sec. III-A Step 4: 2n^2 - n nonzeros of Lambda per component, 6n^2 - 3n in total.
    for n in (2, 5, 32):
        assert cx.boundary_rank(n) == 6 * n * n - 3 * n


def test_transform_flops_per_box_is_nine_tensor_products_each_way():
    # Sec. III-B: one tensor product costs 2 n^4 on a cube; G and G^{-1} are 9 each.
    n = 32
    assert cx.transform_flops_box(n, n, n) == 36 * n ** 4
