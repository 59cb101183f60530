"""The serving workspace pool's size classes (host logic): a class holds the request
and exceeds it by at most an eighth."""
import random

from paper_2606_30620_b300.serve import WorkspacePool


def test_size_class_bounds():
    rng = random.Random(3)
    sizes = [1, 2, 7, 8, 9, 15, 16, 17, 1023, 1024, 1025, 4096, 10_000_000] + \
        [rng.randint(1, 1 << 36) for _ in range(20000)]
    for n in sizes:
        c = WorkspacePool.size_class(n)
        assert n <= c <= n + n // 8 + 1, (n, c)


def test_size_classes_are_few():
    # sizes 1 MB .. 1 GB fall into at most 8 classes per power of two
    classes = {WorkspacePool.size_class(n) for n in range(1 << 20, 1 << 30, 4093)}
    assert len(classes) <= 8 * 10 + 1
