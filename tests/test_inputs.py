"""The synthetic workloads: every dt literal lies just below half the oracle's
von Neumann limit for its model's largest velocity, and the generated models
stay within that velocity; the c5 survey's windows lie inside its grid."""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs


@pytest.mark.parametrize("key", sorted(inputs.DT))
def test_dt_literals_below_half_cfl(oracle, key):
    name, so = key
    limit = oracle.cfl_dt(so, (inputs.H,) * 3, inputs.V_MAX[name])
    assert 0.45 * limit < inputs.DT[key] < 0.5 * limit


def test_models_within_v_max_and_contiguous():
    cases = [("c1", inputs.c1(nt=2)), ("c2", inputs.c2(nt=2, n=(48, 40, 64))),
             ("c3", inputs.c3(nt=2, n=(40, 36, 32))), ("c4", inputs.c4(nt=2, n=(64, 64, 64))),
             ("c4", inputs.c4(nt=2, n=(64, 64, 64), true_model=False)),
             ("c5", inputs.c5(nshots=2, nt=2)), ("c5", inputs.c5(nshots=2, nt=2, true_model=False))]
    for name, p in cases:
        assert float(np.sqrt(1.0 / p.m.min())) <= inputs.V_MAX[name] * (1 + 1e-6), name
        for a in (p.m, p.damp):
            assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"], name


def test_c5_windows_inside_grid():
    s = inputs.c5(nshots=64, nt=2)
    assert len(s.shots) == 64
    for sh in s.shots:
        for a in range(3):
            assert sh["origin"][a] >= 0 and sh["origin"][a] + sh["n"][a] <= s.n[a]
        assert 128 <= sh["n"][0] <= 320 and 128 <= sh["n"][1] <= 320 and 128 <= sh["n"][2] <= 256
        ext = [(sh["n"][a] - 1) * inputs.H for a in range(3)]
        for pts in (sh["src_xyz"], sh["rec_xyz"]):
            assert np.all(pts >= 0) and np.all(pts <= np.array(ext, np.float32) + 1e-6)
