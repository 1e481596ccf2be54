"""Host-side pieces of the benchmark that need no GPU: the product-count
comparison of Sec. 5.2 (Fig. 7) recomputed exactly for FP64 words."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fig7_product_counts_follow_the_papers_comparison():
    """Sec. 5.2 for FP64 words: the multimodular count is at least the lower
    bound of eq. numprodMM, and whenever the best multiword variant has
    u + v <= 4 it needs no more products than the multimodular approach."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_07508_b300 import inputs
    k = 4096
    counts = bench.product_counts(k)
    assert set(counts) == {str(b) for b in range(20, 53)}
    for b, row in counts.items():
        lp = math.log2(inputs.largest_prime_below_pow2(int(b)))
        for lam, c in row.items():
            lower = math.ceil((4 * lp + 2 * math.log2(k)) / (53 - math.log2(int(lam))))
            assert c["multimodular"] >= lower - 1  # eq. numprodMM, up to the rounding of the prime bound
            u, v = c["uv"]
            if u + v <= 4:
                assert c["multiword"] <= c["multimodular"], (b, lam, c)
    assert counts["52"]["1"] == {"multiword": 4, "uv": [2, 2], "multimodular": 5}


def test_committed_traffic_profile_matches_the_kernel_source():
    """The bench line's roofline traffic comes from the committed ncu summary
    of the word-product kernels, which is valid only for the kernel source
    whose hash it records: the committed summary and source must agree, so
    that the line carries measured DRAM bytes rather than null, one value
    per sweep bitsize and each at least the launch's algorithmic bytes."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_07508_b300 import inputs
    traffic = bench.profile_traffic()
    assert traffic is not None, "profiles/gemm_tc_sweep4096.md was taken on another gemm_tc.cu"
    assert sorted(traffic) == sorted(inputs.SWEEP_BITS)
    n = 4096
    for b, t in traffic.items():
        u = math.ceil(b / 9) if math.ceil(b / 9) < math.ceil(b / 8) else math.ceil(b / 8)  # digits a side
        algorithmic = 2 * u * n * n * 2 + (2 * u - 1) * n * n * 4  # words read once, sums written once
        assert t >= 0.9 * algorithmic, (b, t, algorithmic)
