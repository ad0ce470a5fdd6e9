"""Host logic of bench.py's byte model: visits per level of a mu-cycle (Alg. 4's
recursion, with the hybrid rule) and the bytes of a solve built from them."""
import bench


def test_cycle_visits_follow_the_recursion():
    sizes = [1 << 24, 1 << 21, 1 << 18, 1 << 15, 1 << 12]
    assert bench.cycle_visits(sizes, 1) == [1, 1, 1, 1, 1]
    assert bench.cycle_visits(sizes, 2) == [1, 2, 4, 8, 16]
    # hybrid: mu visits only into levels of at least 2^20 cells, once below
    assert bench.cycle_visits(sizes, 2, 1 << 20) == [1, 2, 2, 2, 2]


def test_model_bytes_per_solve():
    sizes = [1000, 125]
    n_tree = 1125
    v = bench.model_bytes(sizes, n_tree, 3, "mixed", fused_first=False)
    assert v == 3 * (bench.LEVEL_VISIT_BYTES * (1000 + 125) + bench.OUTER_BYTES["mixed"] * n_tree)
    # the mixed solve's cycles take their first sweep from the update (or the projection)
    vf = bench.model_bytes(sizes, n_tree, 3, "mixed")
    assert vf == v - 3 * bench.FIRST_SWEEP_SAVED_BYTES * 1000
    w = bench.model_bytes(sizes, n_tree, 3, "fp32", mu=2)
    assert w == 3 * (bench.LEVEL_VISIT_BYTES * (1000 + 2 * 125) + bench.OUTER_BYTES["fp32"] * n_tree)
