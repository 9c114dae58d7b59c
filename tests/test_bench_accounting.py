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
