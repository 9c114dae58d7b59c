"""The benchmark's byte accounting for the roofline of a plan (host logic,
no GPU): the unfused per-plan count against the worked figures of the
512x512, depth-3, K = 4 configuration at its level capacities
[1, 20, 400, 8000] with 1 MiB beliefs -- 862 belief-sized transfers with
the factorised leaf values (2 + 20 at the root, 20 (2 + 20) at level 1, one
read of each of the 400 leaf parents), 17,262 with materialised leaves
(each of the 8,000 leaves written and read back)."""
import bench


def test_survey_bytes_fused_worked_example():
    N = 512 * 512
    assert bench.survey_bytes([1, 20, 400, 8000], N, 3, "fused") == 862 * 4 * N


def test_survey_bytes_materialised_worked_example():
    N = 512 * 512
    assert bench.survey_bytes([1, 20, 400, 8000], N, 3, "materialise") == (22 + 440 + 800 + 8000 + 8000) * 4 * N


def test_survey_bytes_small_cases():
    # depth 0: the root's one read; depth 1: the root is the leaf parent
    assert bench.survey_bytes([1], 10, 0, "fused") == 40
    assert bench.survey_bytes([1, 7], 10, 1, "fused") == 40
    assert bench.survey_bytes([1, 7], 10, 1, "materialise") == (2 + 7 + 7) * 40


def test_support_cells_dilate_and_clip():
    import numpy as np
    occ = np.zeros((10, 12), np.uint8)
    b = np.zeros((10, 12), np.float32)
    b[4:7, 5:8] = 1.0           # a 3x3 block in the middle
    assert bench.support_cells(b, occ, 1)[:3] == [9, 25, 49]
    b[:] = 0.0
    b[0, 0] = 1.0               # a corner: the window is clipped by the grid
    assert bench.support_cells(b, occ, 2) == [1, 4, 9, 16]
    b[:] = 0.0                  # no mass at all: empty windows
    assert bench.support_cells(b, occ, 0) == [0, 0]


def test_window_bytes_reduce_to_the_dense_count_on_full_windows():
    N = 37 * 40
    for nodes, depth in (([1, 7, 30, 90], 3), ([1, 5], 1), ([1], 0)):
        for mode in ("fused", "materialise"):
            assert bench.window_bytes(nodes, [N] * (depth + 2), depth, mode) == \
                bench.survey_bytes(nodes, N, depth, mode)


def test_expand_flops_per_level():
    # depth 2, fused: the root (no child formation) over the level-1 window,
    # then level 1 in the contraction form over its own window: per child
    # and cell, per parent (the root) and cell, and the planes per cell
    base = bench.FLOPS_STENCIL + bench.FLOPS_SUMS
    got = bench.expand_flops([1, 6, 40], [100, 110, 121, 130], 2, "fused")
    assert got == 1 * 110 * base + 110 * (6 * bench.FLOPS_CTR_CHILD + 1 * bench.FLOPS_STENCIL + bench.FLOPS_CTR_PLANES)
    # depth 1, fused: the root's own pass with the Q-weighted sums (no contraction form)
    got = bench.expand_flops([1, 6], [100, 110, 121], 1, "fused")
    assert got == 1 * 110 * (base + bench.FLOPS_QSUMS)
    got = bench.expand_flops([1, 6, 40], [100, 110, 121, 130], 2, "materialise")
    assert got == 1 * 110 * base + 6 * 121 * (base + bench.FLOPS_CHILD)
    # 152 SMs at 2070 MHz: 152 * 128 * 2 * 2.07e9 = 80.55 TFLOP/s
    assert abs(bench.alu_peak_tflops(152) - 80.55) < 0.01
