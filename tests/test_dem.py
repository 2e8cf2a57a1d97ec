"""The library's text DEM reader (bsd_dem_*) against a hand-worked fixture and
against the independent reader in oracle/dem.py.  Host code only: no GPU."""
import json
import os

import numpy as np
import pytest

from oracle import dem as O
from paper_2512_07057_gb300 import binding as B
from paper_2512_07057_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _columns(row_ptr, col_idx, rows, N):
    cols = [[] for _ in range(N)]
    for i in range(rows):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            cols[col_idx[e]].append(i)
    return cols


def _dense(d, key_rp, key_ci, rows):
    X = np.zeros((rows, d["N"]), np.uint8)
    for i in range(rows):
        X[i, d[key_ci][d[key_rp][i]:d[key_rp][i + 1]]] = 1
    return X


def test_golden_fixture():
    text = open(os.path.join(GOLD, "dem_small.dem")).read()
    g = json.load(open(os.path.join(GOLD, "dem_small.json")))
    d = B.bsd_dem_read(text)
    assert (d["M"], d["N"], d["K"]) == (g["M"], g["N"], g["K"])
    assert _columns(d["H_row_ptr"], d["H_col_idx"], d["M"], d["N"]) == g["H_columns"]
    assert _columns(d["A_row_ptr"], d["A_col_idx"], d["K"], d["N"]) == g["A_columns"]
    assert list(d["priors"]) == g["priors"]
    dm = B.bsd_dem_read(text, merge=True)
    np.testing.assert_allclose(dm["priors"], g["merged_priors"], rtol=1e-15)
    # every row's column indices ascend (bsd_create's requirement)
    for i in range(d["M"]):
        seg = d["H_col_idx"][d["H_row_ptr"][i]:d["H_row_ptr"][i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_round_trip_of_the_phenomenological_dem():
    prob = W.bb_phenomenological(12, 6, 12, 2e-3, 3e-3)
    text = W.problem_to_dem(prob)
    d = B.bsd_dem_read(text)
    assert (d["M"], d["N"], d["K"]) == (prob.M, prob.N, prob.K)
    assert np.array_equal(d["H_row_ptr"], prob.H_row_ptr) and np.array_equal(d["H_col_idx"], prob.H_col_idx)
    assert np.array_equal(d["A_row_ptr"], prob.A_row_ptr) and np.array_equal(d["A_col_idx"], prob.A_col_idx)
    assert np.array_equal(d["priors"], prob.priors)


def _random_dem(rng, depth=0):
    """Random text with nested repeats, shifts, tags, comments and '^'."""
    out = []
    for _ in range(int(rng.integers(1, 6))):
        r = rng.random()
        if r < 0.55:
            tg = ["D%d" % rng.integers(0, 12) for _ in range(rng.integers(0, 5))]
            tg += ["L%d" % rng.integers(0, 3) for _ in range(rng.integers(0, 2))]
            if len(tg) > 1 and rng.random() < 0.3:
                tg.insert(int(rng.integers(1, len(tg))), "^")
            tag = "[t%d]" % rng.integers(0, 9) if rng.random() < 0.2 else ""
            out.append(f"error{tag}({rng.uniform(1e-4, 0.3):.17g}) " + " ".join(tg))
        elif r < 0.7:
            out.append(f"shift_detectors({rng.integers(0, 3)}, 1) {rng.integers(0, 7)}")
        elif r < 0.8:
            out.append(f"detector({rng.uniform():.3f}) D{rng.integers(0, 20)}  # a comment")
        elif r < 0.85:
            out.append(f"logical_observable L{rng.integers(0, 5)}")
        elif depth < 2:
            out.append(f"repeat {rng.integers(0, 4)} {{")
            out += ["    " + s for s in _random_dem(rng, depth + 1)]
            out.append("}")
    return out


@pytest.mark.parametrize("seed", range(25))
def test_random_texts_agree_with_the_oracle_reader(seed):
    rng = np.random.default_rng(seed)
    text = "\n".join(_random_dem(rng) + ["error(0.01) D0"]) + "\n"
    for merge in (False, True):
        d = B.bsd_dem_read(text, merge=merge)
        r = O.read_dem(text, merge=merge)
        assert (d["M"], d["N"], d["K"]) == (r["M"], r["N"], r["K"])
        assert np.array_equal(_dense(d, "H_row_ptr", "H_col_idx", d["M"]), r["H"])
        assert np.array_equal(_dense(d, "A_row_ptr", "A_col_idx", d["K"]), r["A"])
        np.testing.assert_allclose(d["priors"], r["priors"], rtol=1e-15)


@pytest.mark.parametrize("text,code,line", [
    ("error(0.1) D0\nflip(0.2) D1\n", B.BSD_ERR_UNSUPPORTED, 2),       # unknown instruction
    ("error(0.1) D0\nerror(1.5) D1\n", B.BSD_ERR_INVALID_ARG, 2),      # probability outside [0, 1]
    ("error(0.1) D0 X3\n", B.BSD_ERR_INVALID_ARG, 1),                  # unknown target
    ("repeat 2 {\nerror(0.1) D0\n", B.BSD_ERR_INVALID_ARG, 3),         # block not closed
    ("error(0.1) D0\n}\n", B.BSD_ERR_INVALID_ARG, 2),                  # stray brace
    ("error(0.1 D0\n", B.BSD_ERR_INVALID_ARG, 1),                      # unclosed arguments
])
def test_errors_name_the_line(text, code, line):
    with pytest.raises(B.BsdError) as ei:
        B.bsd_dem_read(text)
    assert ei.value.code == code
    assert f"line {line}" in str(ei.value)
