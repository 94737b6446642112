"""The bench line's comparison with the oracle (bench.oracle_agreement), on the CPU.

The "GPU side" here is made by the oracle itself on a small canyon (4 RX), so the report must show
full agreement; then single planted differences (a length, a validity bit, a solved bit, a gradient
entry) must each show up in the field that reports them.
"""

import numpy as np
import pytest

import bench
from paper_2510_16172_gb300 import scenes


@pytest.fixture(scope="module")
def case(oracle_lib):
    oracle = oracle_lib
    sc = scenes.urban_canyon(0, rx_grid=2)
    n_paths = 32 ** 3 * 4
    g = np.sort(np.random.default_rng(7).choice(n_paths, 3000, replace=False))
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 3, 3, g)
    ref = oracle.solve(sc, ids, order, ti, ri)
    w = (ref["status"] & (oracle.VALID | oracle.SOLVED)) == (oracle.VALID | oracle.SOLVED)
    at = oracle.solve(sc, ids, order, ti, ri, solver=oracle.BFGS, max_iters=0, T_start=ref["T"],
                      dL=w.astype(np.float64))
    grads = oracle.reduce_gradients(sc, ids, order, ti, ri, at["dtheta"] * w[:, None])
    S = {"g": g, "T": ref["T"].copy(), "L": ref["L"].copy(), "status": ref["status"].astype(np.int64),
         "w": w, "grads": [x.copy() for x in grads]}
    return oracle, sc, S


def report(sc, S):
    return bench.oracle_agreement(sc, S, lambda g: bench.oracle_decode_canyon(sc, g))


def copy(S):
    return {k: (v.copy() if isinstance(v, np.ndarray) else [x.copy() for x in v]) for k, v in S.items()}


def test_identical_results_agree(case):
    _, sc, S = case
    r = report(sc, S)
    assert r["solved_both"] > 1000 and r["solved_gpu_only"] == 0 and r["solved_oracle_only"] == 0
    assert r["max_dX_m"] == 0.0 and r["max_rel_dL"] == 0.0
    assert r["mask_mismatches"] == 0
    assert r["gradient_paths"] == int(S["w"].sum()) > 100
    assert max(r["gradient_rel_err"].values()) < 1e-12


def test_planted_differences_are_reported(case):
    oracle, sc, S = case
    solved = np.flatnonzero((S["status"] & oracle.SOLVED) > 0)
    k = solved[len(solved) // 2]

    P = copy(S)
    P["L"][k] *= 1.0 + 1e-4
    assert report(sc, P)["max_rel_dL"] == pytest.approx(1e-4, rel=1e-6)

    P = copy(S)
    P["status"][k] ^= oracle.VALID
    assert report(sc, P)["mask_mismatches"] == 1

    P = copy(S)
    P["status"][k] &= ~oracle.SOLVED
    r = report(sc, P)
    assert r["solved_oracle_only"] == 1 and r["solved_both"] == len(solved) - 1

    P = copy(S)
    P["T"][k, 0, 0] += 1e-3  # the point moves by 1e-3 x |a1| of its object
    assert report(sc, P)["max_dX_m"] > 1e-3

    P = copy(S)
    v = P["grads"][2]
    i = np.unravel_index(np.abs(v).argmax(), v.shape)
    v[i] *= 1.01
    assert report(sc, P)["gradient_rel_err"]["vertices"] == pytest.approx(0.01, rel=1e-6)
