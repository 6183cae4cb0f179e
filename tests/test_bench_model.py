"""Host checks of the benchmark's byte model and launch mirror (no GPU).

The byte model must reproduce the compulsory traffic written out by hand for
the workloads (pull SpMV of the 27-point stencil on 256^3 and of the scale-22
R-MAT PageRank step), take the least of the three patterns as a product's
work, and the launch mirror must give the launches per call that the
profiler's launch list of one benchmark step shows per call class."""
import bench


def test_dense_pull_bytes_of_the_stencil_and_pagerank():
    m = n = 256 ** 3
    nnz = 766 ** 3  # interior 27-point rows plus the truncated boundary rows
    assert nnz == 449_455_096
    # rowptr, (index + value) per entry, x, y -- each element once, FP32
    assert bench.useful_bytes(0, m, n, nnz, n, nnz, m, 4, 4, 4, False, False) == 3_796_967_364
    m = n = 1 << 22
    nnz = 128_305_302
    b = bench.useful_bytes(1, m, n, nnz, n, nnz, m, 4, 4, 4, False, False)
    assert b == 4 * (m + 1) + 8 * nnz + 4 * n + 4 * m
    assert abs(b / 1e9 - 1.077) < 0.001


def test_push_and_validated_pull_bytes():
    m, n, nnz = 1000, 2000, 50_000
    nnz_x, nnz_s, nnz_y = 30, 700, 400
    push = bench.useful_bytes(6, m, n, nnz, nnz_x, nnz_s, nnz_y, 4, 4, 4, True, True)
    assert push == nnz_x * 8 + 8 * nnz_x + nnz_s * 8 + nnz_y * 8 + 8
    mpull = bench.useful_bytes(3, m, n, nnz, nnz_x, nnz_s, nnz_y, 4, 4, 4, True, True)
    assert mpull == 4 * (m + 1) + 4 * nnz + nnz_s * 4 + n / 8 + nnz_x * 8 + nnz_y * 8 + 8
    # Boolean: no values anywhere
    bpush = bench.useful_bytes(8, m, n, nnz, nnz_x, nnz_s, nnz_y, 0, 0, 0, True, True)
    assert bpush == nnz_x * 4 + 8 * nnz_x + nnz_s * 4 + nnz_y * 4 + 8
    w = bench.work_bytes(m, n, nnz, nnz_x, nnz_s, nnz_y, 4, 4, 4, True, True)
    assert w == min(push, mpull, bench.useful_bytes(0, m, n, nnz, nnz_x, nnz_s, nnz_y, 4, 4, 4, True, True))


def test_launch_mirror_matches_the_profiled_step():
    # launches per call of each class in the committed launch list of one
    # step (Boolean list in / list out; PageRank dense, forced in the replay);
    # the replay launches the recorded choice directly, so no direct chain
    K = {name: i for i, name in enumerate(("pull_thread", "pull_warp", "pull_bal", "mpull_thread", "mpull_warp",
                                          "mpull_bal", "push_thread_atom", "push_warp_atom", "push_bal_atom"))}
    long_flags = 2  # long-row pass and its second pass, no fix-up for a Boolean list output
    # features, scatter, the fused long-row + thread pass, the second pass, compaction (2), clear
    assert bench.launches(K["pull_thread"], True, True, auto=False, long_extra=long_flags, bool_fused=True) == 105 // 15
    assert bench.launches(K["push_bal_atom"], True, True, auto=False) == 96 // 16
    assert bench.launches(K["push_thread_atom"], True, True, auto=False) == 48 // 12
    assert bench.launches(K["push_warp_atom"], True, True, auto=False) == 52 // 13
    # the replay of the PageRank call skips the feature pass (3 launches): the
    # selector-driven call adds it and the warp push's direct chain (4)
    assert bench.launches(K["pull_warp"], False, False, auto=False, long_extra=2) == 3 + 1
    assert bench.launches(K["pull_warp"], False, False, long_extra=2) == 3 + 1 + 4
    # a selector-driven call that picks the warp push launches its chain only
    assert bench.launches(K["push_warp_atom"], True, True) == bench.launches(K["push_warp_atom"], True, True, auto=False)


def test_launch_mirror_matches_the_profiled_stencil_step():
    # launches per call in the committed launch list of the stencil step
    # (per density: x listed -> y listed, x dense -> y dense)
    K = {"pull_thread": 0, "push_warp_atom": 7}
    assert bench.launches(K["push_warp_atom"], True, True, auto=False) == 4  # features, push, compaction (2)
    # features, x compaction (2), push, write-out
    assert bench.launches(K["push_warp_atom"], False, False, auto=False) == 5
    # features, scatter, pull, compaction (2), clear
    assert bench.launches(K["pull_thread"], True, True, auto=False) == 6
    assert bench.launches(K["pull_thread"], False, False, auto=False) == 2  # features, pull
    # selector-driven: the pulls also launch the warp push's chain (3 and 4 kernels)
    assert bench.launches(K["pull_thread"], True, True) == 6 + 3
    assert bench.launches(K["pull_thread"], False, False) == 2 + 4
