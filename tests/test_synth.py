"""Seeded input generators shared by the oracle and the GPU path."""
import numpy as np

from paper_2101_03240_gb300 import synth as S


def test_mixed_edge_matches_the_image():
    for i in range(6):
        img = S.mixed_image(i, 123, 8, 20)
        assert img.shape == (S.mixed_edge(i, 123, 8, 20),) * 3


def test_request_stream_edges_match_the_images():
    reqs = S.c5_requests(n=3, lo=8, hi=16)
    for j, (t, L, kind) in enumerate(reqs):
        assert S.mixed_edge(j, 5000, 8, 16) == L
        assert kind == j % 2
    assert [r[0] for r in reqs] == sorted(r[0] for r in reqs)


def test_bench_generates_the_batch_in_a_pool():
    """bench.py builds the 256-image batch in a process pool; the images are
    those of synth.c4_batch."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    a = bench.batch_images(4)
    b = S.c4_batch(4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
