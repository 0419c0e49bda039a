"""The learned initial guess end to end on a small grid: solver-generated
data, training with the GPU kernels, and solves started from the guess.

The guess is kept only when its FP64 defect beats that of u = 0, so the
converged result is the V-cycle's own: started from the guess or from zero,
the solutions agree to the parity bar, and a rejected guess costs no cycle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_learned_guess_trains_and_keeps_the_solution():
    from paper_1111_0983_gb300 import learn
    n = 129
    X, U, M, bad = learn.make_dataset(list(range(48)), chunk=48, log=lambda s: None, n=n)
    assert X.shape[0] + bad == 48 and X.shape[0] >= 40
    params, hist = learn.train(X, U, M, 200, batch=4, lr=2e-3, lap_weight=0.0, log=lambda s: None)
    assert np.mean(hist[-20:]) < 0.5 * np.mean(hist[:5]), (hist[:5], hist[-20:])
    rows = learn.evaluate(params, [learn.TEST_BASE + i for i in range(4)], rtol=1e-11, n=n)
    for r in rows:
        assert r["converged"]
        assert r["solution_rel_diff"] < 1e-10, r
        if not r["guess_kept"]:
            assert r["cycles_guess"] == r["cycles_zero"], r


def test_stored_network_on_held_out_513_problems():
    """The committed network (trained on the GPU kernels on 2048 solver-generated
    513^2 star problems) on the first three held-out seeds: its guess is closer
    to the solution than u = 0 on two of them (relative L2 errors 0.14 and
    0.73 where u = 0 has 1; the third, 1.96, is worse), every solve converges
    to the V-cycle's own solution, and a guess the defect test rejects costs
    no cycle.  What it does not gain -- cycles at 1e-10 -- is reported by the
    benchmark (guesses_kept, first-cycle defects)."""
    from paper_1111_0983_gb300 import learn
    rows = learn.evaluate(learn.load_weights(), [learn.TEST_BASE + i for i in range(3)])
    errs = sorted(r["guess_rel_err_l2"] for r in rows)
    assert errs[0] < 0.5 and errs[1] < 1.0, rows
    for r in rows:
        assert r["converged"], r
        assert r["solution_rel_diff"] < 1e-10, r
        if not r["guess_kept"]:
            assert r["cycles_guess"] == r["cycles_zero"], r
