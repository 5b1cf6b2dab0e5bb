"""The seeded synthetic inputs have the shapes, sizes and value distributions their
recipes state (the paper's instances are not available; these stand in for them):
the 200 x 400 MIP relaxation, the 50,000 x 200,000 covering LP of the benchmark,
the uneven covering sub-LPs of the batch, and the energy-system LP (checked by its
row / column / nonzero formulas, at a small size generated and at the full size by
arithmetic)."""
import numpy as np
import pytest

import lpgen


def _dense_rows(lp):
    return np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_mip_relaxation_recipe(seed):
    lp = lpgen.mip_relaxation(seed)
    assert (lp.m, lp.n) == (200, 400) and np.all(lp.sense == ord("L"))
    assert np.all(lp.is_int[:200] == 1) and np.all(lp.is_int[200:] == 0)
    assert np.all(lp.l == 0) and np.all(lp.u[:200] == 1) and np.all(lp.u[200:] == 10)
    v = lp.val
    assert np.all(v == np.round(v)) and np.all((np.abs(v) >= 1) & (np.abs(v) <= 5))
    assert 1400 <= lp.nnz <= 1800                     # Bernoulli(0.02) over 80,000 entries
    x0 = lp.meta["x0"]
    assert np.all(x0 >= lp.l) and np.all(x0 <= lp.u) and np.all(x0[:200] == np.round(x0[:200]))
    slack = lp.b - lp.dense() @ x0                    # b = A x0 + U[0, 3]
    assert np.all(slack >= 0) and np.all(slack <= 3)
    assert np.all(np.abs(lp.c) <= 1)


def test_set_cover_benchmark_recipe():
    lp = lpgen.set_cover(2025)
    assert (lp.m, lp.n, lp.nnz) == (50_000, 200_000, 1_296_541)
    assert np.all(lp.val == 1) and np.all(lp.b == 1) and np.all(lp.sense == ord("G"))
    assert np.all(lp.l == 0) and np.all(lp.u == 1) and np.all(lp.is_int == 1)
    assert np.all(lp.c == np.round(lp.c)) and lp.c.min() >= 1 and lp.c.max() <= 100
    per_col = np.bincount(lp.col, minlength=lp.n)
    assert per_col.min() >= 3 and per_col.max() <= 11  # 3-10 rows, plus a repair column
    assert np.all(np.diff(lp.row_ptr) >= 1)           # every row covered
    rows = _dense_rows(lp)
    assert len(set(zip(rows.tolist(), lp.col.tolist()))) == lp.nnz  # distinct rows per column


def test_set_cover_batch_recipe():
    lps = lpgen.set_cover_batch(4)
    for lp in lps:
        assert 2_000 <= lp.m <= 40_000 and lp.n == 4 * lp.m
        assert 0.10 <= lp.meta["fixed_fraction"] <= 0.50
        fixed = lp.l == lp.u
        assert np.all(np.isin(lp.l[fixed], (0.0, 1.0)))
        assert 0.05 <= fixed.mean() <= 0.55
        # no covering row left with every column fixed to 0
        alive = np.zeros(lp.m, dtype=bool)
        alive[_dense_rows(lp)[lp.u[lp.col] > 0]] = True
        assert alive.all()


def _energy_counts(T, R, K, L, th):
    rows = T * R + T * R * K + T * R + T * R * th
    cols = T * R * K + 3 * T * R + 2 * T * L + T * R + R * K
    nnz = T * R * (K + 3) + 4 * T * L + 2 * T * R * K + 4 * T * R + 3 * T * R * th
    return rows, cols, nnz


def test_energy_system_counts_and_coefficients():
    T, R, K, L, th = 24, 5, 3, 6, 2
    lp = lpgen.energy_system(hours=T, regions=R, lines=L, techs=K, thermal=th)
    assert (lp.m, lp.n, lp.nnz) == _energy_counts(T, R, K, L, th)
    a = np.abs(lp.val)
    assert a.min() >= 0.1 and a.max() <= 10.0
    assert np.sum(lp.is_int) == R * K and np.all(lp.u[lp.is_int == 1] == 50)
    per_col = np.bincount(lp.col, minlength=lp.n)[lp.is_int == 1]
    # a capacity column couples every hour: T availability rows, plus T ramping rows if thermal
    assert sorted(set(per_col.tolist())) == [T, 2 * T]
    # the full-size workload of the energy benchmark, by the same formulas
    assert _energy_counts(8760, 20, 6, 40, 4) == (2_102_400, 2_452_920, 7_884_000)
