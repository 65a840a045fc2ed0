"""GPU parity of wave_grad_revolve (binomial checkpointing).

The schedule changes only which forward steps are recomputed and from which
stored state; every reversed step runs the same recompute and adjoint sweeps
as wave_grad.  So the gradient must equal wave_grad's (uniform checkpoints
from wave_fwd) bit for bit, for any slot count, any checkpoint interval and
any forward plan (tiled forward advances included), and match the FP64
oracle gradient within rel-L2 1e-5.
"""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _f64(a):
    return np.asarray(a, dtype=np.float64)


@pytest.mark.parametrize("so,nt,k,slots,T", [(8, 23, 5, 0, 1), (8, 23, 5, 3, 1), (8, 23, 23, 22, 1),
                                             (4, 31, 7, 4, 2), (12, 19, 4, 2, 0)])
def test_revolve_equals_uniform_checkpoints(wavelib, cuda, oracle, so, nt, k, slots, T):
    import torch
    n = (30, 28, 26)
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=30 + so, nsrc=2, nrec=7)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    res = np.random.default_rng(so).standard_normal((nt, len(rec))).astype(np.float32)
    tm, td, tq, tr = _t(m, cuda), _t(damp, cuda), _t(q, cuda), _t(res, cuda)
    tune = wavelib.Tuning(time_tile=T, kernel=wavelib.WAVE_KERNEL_STAGED if T == 2 else 0)
    g, ws = wavelib.grad_revolve(grid, tm, td, src, tq, rec, tr, slots, tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    _, _, ck, _ = wavelib.fwd(grid, tm, td, src, tq, None, tuning=wavelib.Tuning(time_tile=1), ckpt_every=k)
    want, _ = wavelib.grad(grid, tm, td, src, tq, rec, tr, ck, k, tuning=wavelib.Tuning(time_tile=1))
    torch.cuda.synchronize()
    assert torch.equal(g, want)
    h = [float(np.float32(v)) for v in grid.h]
    gref = oracle.gradient(_f64(m), _f64(damp), h, float(np.float32(dt)), nt, so, _f64(src), _f64(q),
                           _f64(rec), _f64(res))
    err = float(np.linalg.norm(_f64(g.cpu().numpy()) - gref) / np.linalg.norm(gref))
    assert err <= TOL, err


def test_revolve_workspace_checks(wavelib, cuda):
    """Too many slots or too small a workspace is refused before any work."""
    import torch
    n, so, nt = (20, 18, 22), 4, 9
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=2, nsrc=1, nrec=2)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    args = (grid, _t(m, cuda), _t(damp, cuda), src, _t(q, cuda), rec, _t(np.zeros((nt, 2)), cuda))
    with pytest.raises(wavelib.WaveError):
        wavelib.grad_revolve(*args, nt + 1)
    small = torch.empty(wavelib.workspace_bytes(grid, wavelib.WAVE_OP_REVOLVE, 1, 2, 2) - 256,
                        dtype=torch.uint8, device=cuda)
    with pytest.raises((wavelib.WaveError, ValueError)):
        wavelib.grad_revolve(*args, 2, workspace=small)
