"""Shared parity assertions of the GPU tests (CUDA path vs the CPU oracle).

The bar (element by element, same seeded inputs):
  * MP within `tol` of the oracle's MP (1e-9 for the FP64 kernel, 1e-3 for
    the FP32-mixed one), +inf exactly where the oracle has no neighbour;
  * PI identical wherever the oracle's best-to-second-best distance gap
    exceeds 1e-3 (several neighbours are correct inside that gap);
  * elsewhere the GPU's neighbour must be admissible and its distance (by
    the oracle's definition) within `tol` of the oracle's MP.
"""
import numpy as np

import oracle

GAP = 1e-3


def _raw_distance(x, y, m, i, j):
    """||x_i - y_j||: the non-normalised distance, straight from its definition"""
    return float(np.sqrt(np.sum((np.asarray(x[i:i + m], np.float64) -
                                 np.asarray(y[j:j + m], np.float64)) ** 2)))


def check_rows(x, m, rows, mp_gpu, pi_gpu, mp_or, pi_or, sec_or, tol, excl=None, inclusive=False,
               y=None, gap=GAP, raw=False):
    """x: series (row side); y: candidate series for an AB-join (None: self);
    raw: the non-normalised distance."""
    rows = np.asarray(rows)
    mp_g = np.asarray(mp_gpu)[rows]
    pi_g = np.asarray(pi_gpu)[rows]
    fin = np.isfinite(mp_or)
    np.testing.assert_array_equal(np.isfinite(mp_g), fin, err_msg="finite pattern differs")
    np.testing.assert_array_equal(pi_g[~fin], -1)
    if fin.any():
        err = np.abs(mp_g[fin] - mp_or[fin])
        worst = int(np.argmax(err))
        assert err.max() <= tol, (f"|dMP| {err.max():.3e} > {tol:.1e} at row "
                                  f"{rows[fin][worst]} (gpu {mp_g[fin][worst]}, oracle {mp_or[fin][worst]})")
    with np.errstate(invalid="ignore"):                 # inf - inf on rows with no neighbour
        sep = fin & ((sec_or - mp_or) > gap)
    bad = np.nonzero(pi_g[sep] != pi_or[sep])[0]
    assert bad.size == 0, (f"PI differs on {bad.size} separated rows, e.g. row {rows[sep][bad[0]]}: "
                           f"gpu {pi_g[sep][bad[0]]} oracle {pi_or[sep][bad[0]]}")
    # unseparated rows: any admissible neighbour at the optimal distance is correct
    for r in np.nonzero(fin & ~sep & (pi_g != pi_or))[0]:
        i, j = int(rows[r]), int(pi_g[r])
        if y is None:
            assert abs(i - j) >= (excl + 1 if inclusive else excl)
            d = _raw_distance(x, x, m, i, j) if raw else oracle.distance(x, m, i, j)
        else:
            d = _raw_distance(x, y, m, i, j) if raw else oracle.distance_ab(x, y, m, i, j)
        assert abs(d - mp_or[r]) <= tol, f"row {i}: neighbour {j} at {d} vs best {mp_or[r]}"
    return float(np.max(np.abs(mp_g[fin] - mp_or[fin]))) if fin.any() else 0.0
