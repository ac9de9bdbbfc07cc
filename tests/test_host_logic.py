"""Host-side logic that needs no GPU: the sweep driver's table layout."""
from paper_1311_1695_gb300 import sweep


def _rec(k, d, m, mvp, status=0):
    return dict(n_eig=k, delta=d, method=m, mvp=mvp, seconds=0.5, outer_its=7, status=status)


def test_sweep_table_layout():
    """One row per (N_eig, delta), delta 1e-3 rows first as in the paper's
    tables; JD beyond its block shows dashes; a failed run shows its status."""
    recs = [_rec(5, 1e-6, "jd", 300), _rec(5, 1e-3, "jd", 100), _rec(5, 1e-3, "dacg", 200, status=1),
            dict(n_eig=50, delta=1e-3, method="jd", skipped="block"), _rec(50, 1e-3, "irlm", 900)]
    lines = sweep.table(recs).split("\n")
    assert len(lines) == 2 + 3
    assert lines[2].startswith("| 5 | 1e-03 |") and "200 (status 1)" in lines[2]
    assert lines[3].startswith("| 50 | 1e-03 |") and "900" in lines[3]
    jd_cells = lines[3].split("|")[6:9]
    assert all(c.strip() == "—" for c in jd_cells)
    assert lines[4].startswith("| 5 | 1e-06 |") and "300" in lines[4]
