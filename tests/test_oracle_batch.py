"""Pins for the oracle's batched survey (forward_batched, gradient_batched).

A shot covering the whole grid reduces to the single-shot forward and
gradient; a shot's traces do not see the model outside its window; the
survey gradient is zero outside every window; and it matches central finite
differences of the survey misfit J(m) = sum_s 1/2 |d_s(m) - d_obs,s|^2 over
the global model, which fixes the window offsets of both the extraction and
the scatter (a shifted window fails it).
"""
import numpy as np


def _survey(seed=3):
    rng = np.random.default_rng(seed)
    n = (18, 16, 14)
    h = (0.01, 0.011, 0.009)
    m = 0.25 + 0.2 * rng.random(n)
    damp = 2.0 * rng.random(n)
    shots = [
        dict(origin=(0, 0, 0), n=(12, 11, 10), src=[[0.05, 0.06, 0.04]],
             rec=[[0.02 + 0.01 * i, 0.07, 0.05] for i in range(5)]),
        dict(origin=(5, 4, 3), n=(13, 12, 11), src=[[0.07, 0.05, 0.03]],
             rec=[[0.03 + 0.01 * i, 0.04, 0.06] for i in range(6)]),
        dict(origin=(6, 5, 4), n=(10, 10, 10), src=[[0.04, 0.04, 0.04], [0.06, 0.05, 0.02]],
             rec=[[0.05, 0.02 + 0.01 * i, 0.03] for i in range(4)]),
    ]
    return rng, n, h, m, damp, shots


def _ricker(nt, dt, f=40.0, t0=0.025):
    t = np.arange(nt) * dt
    a = (np.pi * f * (t - t0)) ** 2
    return (1 - 2 * a) * np.exp(-a)


def test_whole_grid_shot_is_the_single_shot_path(oracle):
    rng, n, h, m, damp, _ = _survey()
    nt, dt, so = 20, 1e-3, 4
    src = [[0.08, 0.07, 0.06]]
    rec = [[0.03 * i + 0.01, 0.05, 0.04] for i in range(4)]
    q = rng.standard_normal((nt, 1))
    res = rng.standard_normal((nt, 4))
    shot = dict(origin=(0, 0, 0), n=n, src=src, rec=rec)
    d1 = oracle.forward_batched(m, damp, h, dt, nt, so, [shot], [q])[0]
    d0, _, _ = oracle.forward(m, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
    assert np.array_equal(d1, d0)
    g1 = oracle.gradient_batched(m, damp, h, dt, nt, so, [shot], [q], [res])
    g0 = oracle.gradient(m, damp, h, dt, nt, so, src, q, rec, res)
    assert np.array_equal(g1, g0)


def test_shot_sees_only_its_window(oracle):
    rng, n, h, m, damp, shots = _survey()
    nt, dt, so = 20, 1e-3, 4
    q = [rng.standard_normal((nt, len(s["src"]))) for s in shots]
    d = oracle.forward_batched(m, damp, h, dt, nt, so, shots, q)
    m2 = m.copy()
    m2[13:, :, :] *= 1.5  # outside shot 0's window (x < 12) only
    d2 = oracle.forward_batched(m2, damp, h, dt, nt, so, shots, q)
    assert np.array_equal(d[0], d2[0])
    assert not np.array_equal(d[1], d2[1])


def test_gradient_zero_outside_windows(oracle):
    rng, n, h, m, damp, shots = _survey()
    nt, dt, so = 20, 1e-3, 4
    q = [rng.standard_normal((nt, len(s["src"]))) for s in shots]
    res = [rng.standard_normal((nt, len(s["rec"]))) for s in shots]
    g = oracle.gradient_batched(m, damp, h, dt, nt, so, shots, q, res)
    covered = np.zeros(n, bool)
    for s in shots:
        o, k = s["origin"], s["n"]
        covered[o[0]:o[0] + k[0], o[1]:o[1] + k[1], o[2]:o[2] + k[2]] = True
    assert np.all(g[~covered] == 0.0)
    assert np.abs(g[covered]).max() > 0


def test_survey_gradient_finite_differences(oracle):
    rng, n, h, m, damp, shots = _survey(5)
    nt, dt, so = 50, 1e-3, 4
    w = _ricker(nt, dt)
    q = [np.tile(w[:, None], (1, len(s["src"]))) for s in shots]
    m_true = m.copy()
    m_true[7:11, 6:10, 5:9] *= 1.1
    d_obs = oracle.forward_batched(m_true, damp, h, dt, nt, so, shots, q)

    def misfit(mm):
        d = oracle.forward_batched(mm, damp, h, dt, nt, so, shots, q)
        return 0.5 * sum(float(np.sum((a - b) ** 2)) for a, b in zip(d, d_obs)), d

    j0, d0 = misfit(m)
    res = [a - b for a, b in zip(d0, d_obs)]
    g = oracle.gradient_batched(m, damp, h, dt, nt, so, shots, q, res)
    for k in range(2):
        dm = rng.standard_normal(n)
        dm *= 0.01 * np.abs(m).max() / np.abs(dm).max()
        want = float(np.sum(g * dm))
        eps = 5e-3
        jp, _ = misfit(m + eps * dm)
        jm, _ = misfit(m - eps * dm)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - want) <= 1e-5 * abs(want)
