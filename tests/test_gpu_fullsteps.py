"""Parity after the full step counts of the propagation workloads.

The 512^3 so-8 model family (two layers with +-2 % noise, 40-point damping
layer, Ricker 15 Hz near the top, a line of receivers) runs its full 1000
steps, and the smooth random 1.5-4.5 km/s model family runs its full 500
steps at so 16 and so 8, on grids the FP64 oracle finishes in seconds.  The
FP32 GPU field must stay within rel-L2 1e-5 of the oracle after every 100
steps up to nt (FP32 phase drift grows with the number of steps, so a check
after a few steps says little about nt), and the traces within 1e-5 of their
maximum.  The time-tiled sweeps (both kernel families) must equal the untiled
sweep bit for bit after nt steps.

The error curve is printed (pytest -rP shows it).
"""
import os

import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
SEG = 100


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _gpu(wavelib, dev, p, nt, tune):
    import torch
    grid = wavelib.Grid(p.n, p.h, p.dt, nt, p.space_order)
    nrec = len(p.rec_xyz)
    d, ul, _, ws = wavelib.fwd(grid, _t(p.m, dev), _t(p.damp, dev), p.src_xyz, _t(p.src_q[:nt], dev),
                               p.rec_xyz if nrec else None, tuning=tune, want_u_last=True)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    torch.cuda.synchronize()
    return (d.cpu().numpy() if nrec else None), ul.cpu().numpy()


def _curve(wavelib, cuda, oracle, p, tiled):
    """rel-L2 of u^n against the oracle for n = SEG, 2 SEG, ..., nt; the
    oracle runs the steps once, in segments that carry (u^n, u^{n-1})."""
    oracle.set_threads(os.cpu_count() or 1)
    f64 = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    h = [float(np.float32(v)) for v in p.h]
    dt = float(np.float32(p.dt))
    nrec = len(p.rec_xyz)
    u0 = um1 = None
    d_ref = []
    errs = []
    untiled = wavelib.Tuning(time_tile=1, kernel=wavelib.WAVE_KERNEL_SHARED)
    for n1 in range(SEG, p.nt + 1, SEG):
        d, ul, _ = oracle.forward(f64(p.m), f64(p.damp), h, dt, SEG, p.space_order, f64(p.src_xyz),
                                  f64(p.src_q[n1 - SEG:n1]), f64(p.rec_xyz) if nrec else None,
                                  u0=u0, um1=um1)
        u0, um1 = ul[0], ul[1]
        if nrec:
            d_ref.append(d)
        dg, ug = _gpu(wavelib, cuda, p, n1, untiled)
        err = float(np.linalg.norm(f64(ug[0]) - u0) / np.linalg.norm(u0))
        errs.append((n1, err))
        if n1 == p.nt:
            final = (dg, ug)
    print("%s so %d %s: rel-L2 of u^n against the FP64 oracle: %s"
          % (p.name, p.space_order, "x".join(map(str, p.n)),
             ", ".join("n=%d %.2e" % e for e in errs)))
    for n1, err in errs:
        assert err <= TOL, (n1, err)
    dg, ug = final
    if nrec:
        dref = np.concatenate(d_ref)
        assert np.abs(dg - dref).max() <= TOL * np.abs(dref).max()
    for tune in tiled:
        dt_, ut = _gpu(wavelib, cuda, p, p.nt, tune)
        assert np.array_equal(ut, ug), tune
        if nrec:
            assert np.array_equal(dt_, dg), tune
    return errs


def test_c2_family_full_1000_steps(wavelib, cuda, oracle):
    # the 512^3 model family on 160^3: two layers with noise, the 40-point
    # damping layer, the source at (n/2, n/2, 2) and receivers along x
    p = inputs.c2(nt=1000, n=(160, 160, 160))
    tiled = [wavelib.Tuning(time_tile=2, kernel=wavelib.WAVE_KERNEL_STAGED),
             wavelib.Tuning(time_tile=1, kernel=wavelib.WAVE_KERNEL_STAGED),
             wavelib.Tuning(time_tile=2, kernel=wavelib.WAVE_KERNEL_SHARED)]
    _curve(wavelib, cuda, oracle, p, tiled)


@pytest.mark.parametrize("so", [16, 8])
def test_smooth_model_full_500_steps(wavelib, cuda, oracle, so):
    # the 768 x 768 x 512 smooth random model family on 128 x 128 x 96
    p = inputs.c3(space_order=so, nt=500, n=(128, 128, 96))
    tiled = [wavelib.Tuning(time_tile=1, kernel=wavelib.WAVE_KERNEL_STAGED)]
    depths = {v["time_tile"] for v in wavelib.list_variants(so)
              if v["kernel"] == wavelib.WAVE_KERNEL_STAGED}
    if 2 in depths:
        tiled.append(wavelib.Tuning(time_tile=2, kernel=wavelib.WAVE_KERNEL_STAGED))
    _curve(wavelib, cuda, oracle, p, tiled)
