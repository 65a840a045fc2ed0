"""wave_fwd_noalloc: forward modelling on the library's static workspace.

Collected last, so that it runs both after every other test and alone in a
fresh process.  Through the C ABI it must give what wave_fwd gives on the
same inputs and plan: the same kernels run in the same order, so the traces
and the last two wavefield levels must be equal bit for bit (a tolerance could
hide state left in the shared array by an earlier call).  This is checked on
two calls in a row that share the static array, with an explicit tiling, with
the autotuner choosing the plan on the shared array (tuning NULL), and with
the asynchronous return (status NULL).  A grid whose workspace exceeds
WAVE_NOALLOC_MAX_BYTES must be refused before any work is queued.
"""
import ctypes

import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs


def test_noalloc_rejects_oversized_grid(wavelib):
    # host-side check: nothing is enqueued and no device is touched
    grid = wavelib.Grid((256, 256, 256), (inputs.H,) * 3, 1e-4, 10, 8)
    need = wavelib.workspace_bytes(grid, wavelib.WAVE_OP_FWD, 0, 0)
    assert need > wavelib.WAVE_NOALLOC_MAX_BYTES
    g = grid.c()
    rc = wavelib._lib().wave_fwd_noalloc(ctypes.byref(g), None, None, None, None, None, None,
                                         None, None, None, None)
    assert rc == wavelib.WAVE_ENOSPACE


def _case(wavelib, cuda, seed, n, tune, so=8, nt=24):
    import torch
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=seed, nsrc=2, nrec=6)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    assert wavelib.workspace_bytes(grid, wavelib.WAVE_OP_FWD, len(src), len(rec), tuning=tune) \
        <= wavelib.WAVE_NOALLOC_MAX_BYTES
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(cuda)  # noqa: E731
    return dict(grid=grid, m=t(m), damp=t(damp), src=src, q=t(q), rec=rec, tune=tune,
                rec_out=torch.full((nt, len(rec)), np.nan, dtype=torch.float32, device=cuda),
                u_out=torch.full((2,) + n, np.nan, dtype=torch.float32, device=cuda))


def _check_against_fwd(wavelib, cases):
    got = [(c["rec_out"].cpu().numpy(), c["u_out"].cpu().numpy()) for c in cases]
    for c, (d_na, u_na) in zip(cases, got):
        d, ul, _, ws = wavelib.fwd(c["grid"], c["m"], c["damp"], c["src"], c["q"], c["rec"],
                                   tuning=c["tune"], want_u_last=True)
        assert wavelib.status(ws) == wavelib.WAVE_OK
        d, ul = d.cpu().numpy(), ul.cpu().numpy()
        assert np.abs(d).max() > 0 and np.abs(ul).max() > 0
        assert np.array_equal(u_na, ul), "last levels differ from wave_fwd"
        assert np.array_equal(d_na, d), "traces differ from wave_fwd"


@pytest.mark.gpu
def test_noalloc_matches_wave_fwd_on_two_calls(wavelib, cuda):
    cases = [_case(wavelib, cuda, 11, (48, 40, 52), wavelib.Tuning(time_tile=1)),
             _case(wavelib, cuda, 12, (37, 50, 45), wavelib.Tuning(time_tile=2))]
    # the two no-alloc calls in a row, on buffers that exist before them
    for c in cases:
        st = wavelib.fwd_noalloc(c["grid"], c["m"], c["damp"], c["src"], c["q"], c["rec"],
                                 c["rec_out"], c["u_out"], tuning=c["tune"])
        assert st == wavelib.WAVE_OK
    _check_against_fwd(wavelib, cases)


@pytest.mark.gpu
def test_noalloc_autotuned_and_asynchronous(wavelib, cuda, monkeypatch):
    import torch
    monkeypatch.delenv("WAVE_TUNE_CACHE", raising=False)
    # tuning NULL: the first call for this shape runs the autotuner on the
    # shared array; wave_fwd with tuning NULL then reuses the cached plan
    c0 = _case(wavelib, cuda, 13, (44, 36, 40), None)
    st = wavelib.fwd_noalloc(c0["grid"], c0["m"], c0["damp"], c0["src"], c0["q"], c0["rec"],
                             c0["rec_out"], c0["u_out"], tuning=None)
    assert st == wavelib.WAVE_OK
    # status NULL: the call returns once queued; the caller orders the read
    c1 = _case(wavelib, cuda, 14, (40, 46, 38), wavelib.Tuning(time_tile=2))
    for _ in range(2):  # two calls in a row on the shared array, no wait between
        assert wavelib.fwd_noalloc(c1["grid"], c1["m"], c1["damp"], c1["src"], c1["q"], c1["rec"],
                                   c1["rec_out"], c1["u_out"], tuning=c1["tune"],
                                   wait=False) is None
    torch.cuda.synchronize()
    _check_against_fwd(wavelib, [c0, c1])
