"""wave_fwd_noalloc: forward modelling on the library's static workspace.

Collected last, so that it runs both after every other test and alone in a
fresh process.  Through the C ABI it must give what wave_fwd gives on the
same inputs and tuning (rel-L2 <= 1e-5, the tolerance of the forward parity
tests), on two calls in a row that share the static array; and it must refuse
a grid whose workspace exceeds WAVE_NOALLOC_MAX_BYTES before queueing work.
"""
import ctypes

import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

TOL = 1e-5


def _relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_rejects_oversized_grid(wavelib):
    # host-side check: nothing is enqueued and no device is touched
    grid = wavelib.Grid((256, 256, 256), (inputs.H,) * 3, 1e-4, 10, 8)
    need = wavelib.workspace_bytes(grid, wavelib.WAVE_OP_FWD, 0, 0)
    assert need > wavelib.WAVE_NOALLOC_MAX_BYTES
    g = grid.c()
    rc = wavelib._lib().wave_fwd_noalloc(ctypes.byref(g), None, None, None, None, None, None,
                                         None, None, None, None)
    assert rc == wavelib.WAVE_ENOSPACE


@pytest.mark.gpu
def test_noalloc_matches_wave_fwd_on_two_calls(wavelib, cuda):
    import torch
    so, nt = 8, 24
    cases = []
    for seed, n, T in ((11, (48, 40, 52), 1), (12, (37, 50, 45), 2)):
        m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=seed, nsrc=2, nrec=6)
        dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
        grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
        assert wavelib.workspace_bytes(grid, wavelib.WAVE_OP_FWD, len(src), len(rec)) \
            <= wavelib.WAVE_NOALLOC_MAX_BYTES
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(cuda)  # noqa: E731
        cases.append(dict(grid=grid, m=t(m), damp=t(damp), src=src, q=t(q), rec=rec,
                          tune=wavelib.Tuning(time_tile=T),
                          rec_out=torch.empty((nt, len(rec)), dtype=torch.float32, device=cuda),
                          u_out=torch.empty((2,) + n, dtype=torch.float32, device=cuda)))
    # the two no-alloc calls in a row, on buffers that exist before them
    for c in cases:
        st = wavelib.fwd_noalloc(c["grid"], c["m"], c["damp"], c["src"], c["q"], c["rec"],
                                 c["rec_out"], c["u_out"], tuning=c["tune"])
        assert st == wavelib.WAVE_OK
    got = [(c["rec_out"].cpu().numpy(), c["u_out"].cpu().numpy()) for c in cases]
    for c, (d_na, u_na) in zip(cases, got):
        d, ul, _, ws = wavelib.fwd(c["grid"], c["m"], c["damp"], c["src"], c["q"], c["rec"],
                                   tuning=c["tune"], want_u_last=True)
        assert wavelib.status(ws) == wavelib.WAVE_OK
        d, ul = d.cpu().numpy(), ul.cpu().numpy()
        assert np.abs(d).max() > 0 and np.abs(ul).max() > 0
        assert _relerr(u_na, ul) <= TOL
        assert _relerr(d_na, d) <= TOL
    torch.cuda.synchronize()
