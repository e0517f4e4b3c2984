"""What a warm start can gain at best, on the oracle (CPU): preconditioned CG to a relative
residual of 3e-12 needs about as many iterations per decade of error reduction, so a start
vector whose error is a fraction eps of the answer in every mode saves about
log10(1/eps) / log10(1/3e-12) of the cold iterations -- a tenth per decade on these tiles.
A start 90% right everywhere saves ~10%; saving 15% needs ~3% error in every mode, far below
what local point and height statistics predict (the learned start's held-out prediction
leaves most of the weights' variance unexplained). The GPU test of the learned start
(tests/test_gpu_warmstart.py) states its measured iteration ratio against this bound."""
import numpy as np
import pytest

import datagen as dg
import oracle as O


@pytest.mark.parametrize("seed", [900001, 900002])
def test_iterations_saved_per_decade_of_start_accuracy(seed):
    pb = dg.tile(seed, N=8000)                         # 8,000 points, 800 Halton centres
    A = O.design_matrix(pb.points, pb.centres, pb.R)
    B, b = O.normal_system(A, pb.h)
    c = O.solve_normal(B, b, method="lu")
    _, i0, _ = O.pcg(B, b, tol=3e-12)
    ratios = []
    for eps in (0.1, 0.01, 1e-3):
        _, i1, rel = O.pcg(B, b, tol=3e-12, x0=(1.0 - eps) * c)
        assert rel <= 3e-12
        ratios.append(i1 / i0)
    # measured 0.889-0.903, 0.786-0.801, 0.693-0.702 on seeds 900001-900003
    assert 0.85 <= ratios[0] <= 0.95, ratios
    assert 0.74 <= ratios[1] <= 0.84, ratios
    assert 0.64 <= ratios[2] <= 0.74, ratios
    # about the same saving per decade
    steps = np.diff([1.0] + ratios)
    assert np.all(np.abs(steps + 0.1) <= 0.04), steps
