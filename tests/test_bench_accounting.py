"""bench.py's byte accounting (no GPU): X passes of the HOSVD plan, of the sequential
reading and of column sampling, against counts written out by hand for small shapes."""
import bench


def test_hosvd_passes():
    # 512^3, R = 20, p = 10, q = 3: every mode Krylov (b = 120 < 512): 1 TTM + 3 x (1 + 4)
    assert bench.plan_passes([512] * 3, [20] * 3, 10, 3) == (16, 12)
    # video: two Krylov modes (q + 2 = 6 each), the colour mode Gram (1), the frame mode
    # Krylov (S = 40, b = 200 < 256): 1 + 6 + 6 + 1 + 6
    assert bench.plan_passes([1024, 1024, 3, 256], [40, 40, 3, 30], 10, 4) == (20, 15)
    # 16^6, R = 10, p = 5: b = 45 >= 16 everywhere: 1 + 6 Gram passes, no Krylov step
    assert bench.plan_passes([16] * 6, [10] * 6, 5, 2) == (7, 0)


def test_sequential_bytes():
    # 8 x 6 x 5, R = (2, 3, 4), p = 1, q = 1, 2-byte elements
    # step 0: Y_0 = 240 elements, S = 3, b = 6 < 8: Krylov, 1 + 2 passes + the product
    # step 1: Y_1 = 2 x 6 x 5 = 60, S = 4, b = 8 >= 6: Gram, 1 pass + the product
    # step 2: Y_2 = 2 x 3 x 5 = 30, S = 5, b = 10 >= 5: Gram, 1 pass + the product
    total, kb, ks = bench.plan_sequential([8, 6, 5], [2, 3, 4], 1, 1, 2, 2)
    assert total == (4 * 240 + 2 * 60 + 2 * 30) * 2
    assert kb == 2 * 240 * 2 and ks == 2


def test_sampled_columns_and_bytes():
    # mode 0 of 4 x 300 x 2: A = 1, C = 600 -> 5 units of 128; omega = 0.5 keeps 3 units
    assert bench.sampled_columns([4, 300, 2], 0, 0.5) == 3 * 128
    # mode 2: C = 1, A = 1200 -> 10 units; omega = 0.05 keeps ceil(0.5) = 1
    assert bench.sampled_columns([4, 300, 2], 2, 0.05) == 128
    # 64^3, R = 8, p = 4, q = 2 (all Krylov), omega = 0.25, 2-byte elements: per mode the
    # sample has ceil(0.25 U) units of 128 columns; the first core product reads X
    total, kb, ks = bench.plan_sampled([64] * 3, [8] * 3, 4, 2, 0.25, 2)
    numel = 64 ** 3
    ys = [bench.sampled_columns([64] * 3, n, 0.25) * 64 * 2 for n in range(3)]
    assert total == numel * 2 + sum(2 * y + 4 * y for y in ys)
    assert kb == sum(3 * y for y in ys) and ks == 9
