"""bench.py's byte and flop models of the Gram-Schmidt passes (host logic, no GPU).

With selective re-orthogonalisation the second pass's launches (a projection and an update)
leave at once in the columns that keep their first update, so their class counts the bytes of
the columns that ran only: a column j that runs streams (j + 2) K-vectors (projection) and
(j + 3) (update and norm), averaged over all launches of the class."""
import bench

K, T, M = 1000, 4, 30


def test_second_pass_columns_from_the_step_masks():
    # columns 0 and 2 of one stage, none of the other
    frac, avg_j = bench.second_pass_columns([0b101, 0], 3)
    assert frac == 2 / 6 and avg_j == 1.0
    # every column of every stage: the whole class ran, mean column (m - 1) / 2
    frac, avg_j = bench.second_pass_columns([(1 << M) - 1] * 4, M)
    assert frac == 1.0 and avg_j == (M - 1) / 2
    # no second pass at all
    assert bench.second_pass_columns([0, 0], M) == (0.0, 0.0)


def test_byte_model_counts_only_the_columns_that_ran():
    ab = lambda kind, gs=None: bench.algorithmic_bytes(kind, T, K, 1, 1, 3, 2, M, gs=gs)  # noqa: E731
    avg_j = (M - 1) / 2
    # first update alone: every column reads V_j and w and writes z_{j+1}
    assert ab("cgs_upd1") == (avg_j + 3) * K * T
    # two-pass form: the update-and-norm class ran on every column
    assert ab("cgs_upd_norm") == (avg_j + 3) * K * T
    # selective: 2 of 60 launches ran, on columns 1 and 3 (mean 2)
    gs = bench.second_pass_columns([0b1010, 0], M)
    assert ab("cgs_upd_norm", gs) == gs[0] * (2 + 3) * K * T
    assert ab("cgs_proj2", gs) == gs[0] * (2 + 2) * K * T
    assert ab("cgs_upd_norm", (0.0, 0.0)) == 0.0


def test_flop_model_of_the_selective_passes():
    fl = lambda kind, gs=None: bench.algorithmic_flops(kind, K, 1, 1, 3, 2, M, T=4, gs=gs)  # noqa: E731
    nc = (M + 1) / 2
    assert fl("cgs_upd1") == 2 * K * (nc + 1)          # update (j + 1 FMA) and norm per unknown
    gs = (0.1, 5.0)
    assert abs(fl("cgs_proj2", gs) - 2 * K * 0.1 * 7.0) <= 1e-9 * K  # (j + 2) FMA where it ran


def test_step_hbm_sums_the_classes_over_the_step():
    prof = {"cgs_upd1": (2, 1.0), "cgs_proj": (2, 1.0), "phi": (2, 0.5)}  # phi has no byte model
    r = bench.step_hbm(prof, T, K, 1, 1, 1000.0, 3, 2, M, 10.0)
    avg_j = (M - 1) / 2
    want = 2 * (avg_j + 3) * K * T + 2 * (avg_j + 2) * K * T
    assert abs(r["algorithmic_bytes_per_step"] - want) <= 1e-9 * want
    assert abs(r["gbs"] - round(want / 1e-2 / 1e9, 1)) <= 0.05 and r["peak"] == 1000.0
