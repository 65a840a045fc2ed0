"""GPU parity of the batched survey (wave_fwd_batched, wave_grad_batched).

* every shot's traces equal wave_fwd on its window, bit for bit, untiled
  (shots in lockstep, one launch per step) and time-tiled (one stream per
  shot), with more shots than concurrent slots;
* the survey gradient equals the per-shot wave_grad gradients added into a
  zero global array in shot order, bit for bit, for either engine and any
  concurrency;
* both match the FP64 oracle of the survey: traces within 1e-5 of max |d|,
  gradient rel-L2 <= 1e-5;
* a window outside the global grid is refused before any work is queued.
"""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _survey(wavelib, so, nt, seed=21):
    rng = np.random.default_rng(seed)
    n = (40, 36, 38)
    m, damp, _, _, _ = inputs.random_problem(n, so, nt, seed=seed)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    wins = [((0, 0, 0), (24, 22, 26)), ((10, 8, 6), (30, 28, 30)), ((16, 12, 0), (22, 24, 20)),
            ((3, 14, 9), (21, 20, 29)), ((0, 0, 0), n)]
    shots, q, qn = [], [], []
    for i, (o, k) in enumerate(wins):
        ext = np.array([(k[a] - 1) * inputs.H for a in range(3)])
        ns, nr = 1 + i % 2, 3 + i
        src = (0.1 + 0.8 * rng.random((ns, 3))) * ext
        rec = (0.05 + 0.9 * rng.random((nr, 3))) * ext
        shots.append(wavelib.Shot(origin=o, n=k, src_xyz=src.astype(np.float32),
                                  rec_xyz=rec.astype(np.float32)))
        qq = rng.standard_normal((nt, ns)).astype(np.float32)
        qn.append(qq)
    h = [float(np.float32(v)) for v in grid.h]
    return grid, h, float(np.float32(dt)), m, damp, shots, qn


def _oshots(shots):
    return [dict(origin=s.origin, n=s.n, src=np.asarray(s.src_xyz, np.float64),
                 rec=np.asarray(s.rec_xyz, np.float64)) for s in shots]


def _win(s):
    return tuple(slice(s.origin[a], s.origin[a] + s.n[a]) for a in range(3))


@pytest.mark.parametrize("so,T", [(8, 1), (4, 2)])
def test_fwd_batched_equals_single_shots_and_oracle(wavelib, cuda, oracle, so, T):
    import torch
    nt = 24
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt)
    tm, td = _t(m, cuda), _t(damp, cuda)
    tune = wavelib.Tuning(time_tile=T)
    recs, ws = wavelib.fwd_batched(grid, shots, tm, td, [_t(x, cuda) for x in q], concurrency=2,
                                   tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    dref = oracle.forward_batched(np.float64(m), np.float64(damp), h, dt, nt, so, _oshots(shots),
                                  [np.float64(x) for x in q])
    for s, r, qq, dr in zip(shots, recs, q, dref):
        w = _win(s)
        gw = wavelib.Grid(s.n, grid.h, grid.dt, nt, so)
        d1, _, _, ws1 = wavelib.fwd(gw, tm[w].contiguous(), td[w].contiguous(), s.src_xyz,
                                    _t(qq, cuda), s.rec_xyz, tuning=tune)
        assert wavelib.status(ws1) == wavelib.WAVE_OK
        torch.cuda.synchronize()
        assert np.array_equal(r.cpu().numpy(), d1.cpu().numpy())
        assert np.abs(r.cpu().numpy() - dr).max() <= TOL * np.abs(dr).max()


@pytest.mark.parametrize("conc,tile", [(2, None), (3, None), (2, (12, 2))])
def test_grad_batched_equals_shot_order_sum_and_oracle(wavelib, cuda, oracle, conc, tile):
    """tile None: the default untiled shape, run in lockstep; (tile_y, vec):
    another untiled shape, which has no batched kernel and runs per shot."""
    import torch
    so, nt, k = 8, 30, 7
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=5)
    rng = np.random.default_rng(9)
    res = [rng.standard_normal((nt, len(s.rec_xyz))).astype(np.float32) for s in shots]
    tm, td = _t(m, cuda), _t(damp, cuda)
    tune = (wavelib.Tuning(time_tile=1) if tile is None
            else wavelib.Tuning(time_tile=1, tile_y=tile[0], vec=tile[1]))
    g, ws = wavelib.grad_batched(grid, shots, tm, td, [_t(x, cuda) for x in q],
                                 [_t(x, cuda) for x in res], k, concurrency=conc, tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    # the same sum by hand: per-shot forward with checkpoints + wave_grad
    want = torch.zeros(grid.n, dtype=torch.float32, device=cuda)
    for s, qq, rr in zip(shots, q, res):
        w = _win(s)
        gw = wavelib.Grid(s.n, grid.h, grid.dt, nt, so)
        mw, dw = tm[w].contiguous(), td[w].contiguous()
        _, _, ck, _ = wavelib.fwd(gw, mw, dw, s.src_xyz, _t(qq, cuda), None,
                                  tuning=wavelib.Tuning(time_tile=1), ckpt_every=k)
        gi, wsg = wavelib.grad(gw, mw, dw, s.src_xyz, _t(qq, cuda), s.rec_xyz, _t(rr, cuda), ck, k,
                               tuning=wavelib.Tuning(time_tile=1))
        assert wavelib.status(wsg) == wavelib.WAVE_OK
        want[w] += gi
    torch.cuda.synchronize()
    assert torch.equal(g, want)
    gref = oracle.gradient_batched(np.float64(m), np.float64(damp), h, dt, nt, so, _oshots(shots),
                                   [np.float64(x) for x in q], [np.float64(x) for x in res])
    err = float(np.linalg.norm(g.cpu().numpy().astype(np.float64) - gref) / np.linalg.norm(gref))
    assert err <= TOL, err


@pytest.mark.parametrize("so", [2, 4, 6, 8, 10, 12, 14, 16])
def test_lockstep_fwd_equals_per_shot_every_order(wavelib, cuda, so):
    """The batched kernel of every space order: each shot's traces equal
    wave_fwd on its window, bit for bit, with the shots of a group of
    different window sizes in one launch."""
    import torch
    nt = 9
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=so)
    tm, td = _t(m, cuda), _t(damp, cuda)
    recs, ws = wavelib.fwd_batched(grid, shots, tm, td, [_t(x, cuda) for x in q], concurrency=4)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    for s, r, qq in zip(shots, recs, q):
        w = _win(s)
        gw = wavelib.Grid(s.n, grid.h, grid.dt, nt, so)
        d1, _, _, _ = wavelib.fwd(gw, tm[w].contiguous(), td[w].contiguous(), s.src_xyz,
                                  _t(qq, cuda), s.rec_xyz, tuning=wavelib.Tuning(time_tile=1))
        torch.cuda.synchronize()
        assert np.array_equal(r.cpu().numpy(), d1.cpu().numpy())


def test_lockstep_reused_workspace_and_side_stream(wavelib, cuda):
    """Two different surveys through one workspace, the second on a side
    stream: the per-shot tables and TMA descriptors the first call left at the
    same addresses must not leak into the second, whose traces equal a call
    on a fresh workspace."""
    import torch
    so, nt = 8, 11
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=3)
    tm, td = _t(m, cuda), _t(damp, cuda)
    qa = [_t(x, cuda) for x in q]
    # the second survey: the same windows in reverse order, other traces
    shots_b, qb = shots[::-1], [2.0 * x for x in qa[::-1]]
    nbytes = max(wavelib.batch_workspace_bytes(grid, shots, 0, 2),
                 wavelib.batch_workspace_bytes(grid, shots_b, 0, 2))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=cuda)
    fresh, _ = wavelib.fwd_batched(grid, shots_b, tm, td, qb, concurrency=2)
    torch.cuda.synchronize()
    wavelib.fwd_batched(grid, shots, tm, td, qa, concurrency=2, workspace=ws)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        again, _ = wavelib.fwd_batched(grid, shots_b, tm, td, qb, concurrency=2, workspace=ws,
                                       stream=side)
    side.synchronize()
    assert wavelib.status(ws) == wavelib.WAVE_OK
    for x, y in zip(again, fresh):
        assert torch.equal(x, y)


def test_lockstep_from_two_host_threads(wavelib, cuda):
    """Two host threads run batched surveys at the same time, each on its own
    stream and workspace (the library's graph capture is shared): both equal
    the same calls made one after the other."""
    import threading
    import torch
    so, nt = 8, 9
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=11)
    tm, td = _t(m, cuda), _t(damp, cuda)
    qa = [_t(x, cuda) for x in q]
    qb = [3.0 * x for x in qa]
    want_a, _ = wavelib.fwd_batched(grid, shots, tm, td, qa, concurrency=2)
    want_b, _ = wavelib.fwd_batched(grid, shots, tm, td, qb, concurrency=3)
    torch.cuda.synchronize()
    got, errors = {}, []

    def run(name, qq, conc):
        try:
            st = torch.cuda.Stream()
            st.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(st):
                for _ in range(3):
                    r, ws = wavelib.fwd_batched(grid, shots, tm, td, qq, concurrency=conc, stream=st)
            st.synchronize()
            assert wavelib.status(ws) == wavelib.WAVE_OK
            got[name] = r
        except Exception as e:  # reported on the main thread
            errors.append(e)

    th = [threading.Thread(target=run, args=("a", qa, 2)), threading.Thread(target=run, args=("b", qb, 3))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for x, y in zip(got["a"], want_a):
        assert torch.equal(x, y)
    for x, y in zip(got["b"], want_b):
        assert torch.equal(x, y)


def test_batch_refuses_window_outside_grid(wavelib, cuda):
    import torch
    grid = wavelib.Grid((20, 20, 20), (inputs.H,) * 3, 1e-4, 4, 4)
    bad = [wavelib.Shot(origin=(10, 0, 0), n=(12, 10, 10))]
    assert wavelib.batch_workspace_bytes(grid, bad, 0, 1) == 0
    tm = torch.ones(grid.n, device=cuda)
    with pytest.raises(wavelib.WaveError):
        wavelib.fwd_batched(grid, bad, tm, tm, [torch.zeros((4, 0), device=cuda)], concurrency=1,
                            workspace=torch.empty(1 << 20, dtype=torch.uint8, device=cuda))


def _per_shot_fwd(wavelib, cuda, grid, shots, tm, td, q, nt, so):
    import torch
    out = []
    for s, qq in zip(shots, q):
        w = _win(s)
        gw = wavelib.Grid(s.n, grid.h, grid.dt, nt, so)
        d1, _, _, _ = wavelib.fwd(gw, tm[w].contiguous(), td[w].contiguous(), s.src_xyz,
                                  _t(qq, cuda), s.rec_xyz, tuning=wavelib.Tuning(time_tile=1))
        out.append(d1)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("so,T", [(2, 1), (2, 2), (4, 1), (4, 2)])
def test_lockstep_staged_fwd_equals_per_shot(wavelib, cuda, so, T):
    """The batched stage-specialised kernel (depth 1 and 2) runs the shots of
    a group in lockstep: each shot's traces equal wave_fwd on its window, bit
    for bit, and the group's forward kernel is the one the tuning names."""
    import torch
    nt = 24
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=40 + so + T)
    tm, td = _t(m, cuda), _t(damp, cuda)
    tune = wavelib.Tuning(time_tile=T, kernel=wavelib.WAVE_KERNEL_STAGED)
    recs, ws = wavelib.fwd_batched(grid, shots, tm, td, [_t(x, cuda) for x in q], concurrency=3,
                                   tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    want = _per_shot_fwd(wavelib, cuda, grid, shots, tm, td, q, nt, so)
    for r, d1 in zip(recs, want):
        assert torch.equal(r, d1)


@pytest.mark.parametrize("so,T", [(4, 1), (4, 2), (8, 1), (8, 2)])
def test_lockstep_staged_grad_equals_shot_order_sum(wavelib, cuda, so, T):
    """Gradient groups whose forward phases (with checkpoints every k steps,
    k a multiple of T) and recompute / imaging-condition phases run on
    batched stage-specialised kernels (at so 8 and T = 2 the gradient phases
    have a shape of their own, 32x32, beside the forward's 64x24): the survey
    gradient equals the per-shot wave_grad gradients added in shot order, bit
    for bit."""
    import torch
    nt, k = 30, 6
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=17)
    rng = np.random.default_rng(4)
    res = [rng.standard_normal((nt, len(s.rec_xyz))).astype(np.float32) for s in shots]
    tm, td = _t(m, cuda), _t(damp, cuda)
    tune = wavelib.Tuning(time_tile=T, kernel=wavelib.WAVE_KERNEL_STAGED)
    g, ws = wavelib.grad_batched(grid, shots, tm, td, [_t(x, cuda) for x in q],
                                 [_t(x, cuda) for x in res], k, concurrency=2, tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    p = wavelib.describe_batch_plan(grid, shots, k, 2, tune)
    assert (p["time_tile"], p["kernel"]) == (T, wavelib.WAVE_KERNEL_STAGED)
    assert (p["grad_kernel"], p["grad_time_tile"]) == (wavelib.WAVE_KERNEL_STAGED, T)
    want = torch.zeros(grid.n, dtype=torch.float32, device=cuda)
    for s, qq, rr in zip(shots, q, res):
        w = _win(s)
        gw = wavelib.Grid(s.n, grid.h, grid.dt, nt, so)
        mw, dw = tm[w].contiguous(), td[w].contiguous()
        _, _, ck, _ = wavelib.fwd(gw, mw, dw, s.src_xyz, _t(qq, cuda), None,
                                  tuning=wavelib.Tuning(time_tile=1), ckpt_every=k)
        gi, wsg = wavelib.grad(gw, mw, dw, s.src_xyz, _t(qq, cuda), s.rec_xyz, _t(rr, cuda), ck, k,
                               tuning=wavelib.Tuning(time_tile=1))
        assert wavelib.status(wsg) == wavelib.WAVE_OK
        want[w] += gi
    torch.cuda.synchronize()
    assert torch.equal(g, want)


@pytest.mark.parametrize("so,nt,k", [(4, 24, 0), (2, 23, 0), (4, 30, 6), (4, 30, 5)])
def test_lockstep_autotuned_forward_kernel(wavelib, cuda, so, nt, k):
    """time_tile 0: the group times its forward kernel (the batched kernel of
    sweep.cuh or a batched stage-specialised one whose depth divides nt and
    the checkpoint interval) and gives the per-shot results bit for bit,
    whichever it picks; the second call takes the cached choice."""
    import torch
    grid, h, dt, m, damp, shots, q = _survey(wavelib, so, nt, seed=60 + nt)
    tm, td = _t(m, cuda), _t(damp, cuda)
    qd = [_t(x, cuda) for x in q]
    if k == 0:
        want = _per_shot_fwd(wavelib, cuda, grid, shots, tm, td, q, nt, so)
        for _ in range(2):
            recs, ws = wavelib.fwd_batched(grid, shots, tm, td, qd, concurrency=4)
            assert wavelib.status(ws) == wavelib.WAVE_OK
            for r, d1 in zip(recs, want):
                assert torch.equal(r, d1)
        p = wavelib.describe_batch_plan(grid, shots, 0, 4)
        assert p["lockstep"] and p["time_tile"] >= 1 and nt % p["time_tile"] == 0
        return
    rng = np.random.default_rng(8)
    res = [_t(rng.standard_normal((nt, len(s.rec_xyz))), cuda) for s in shots]
    ref, _ = wavelib.grad_batched(grid, shots, tm, td, qd, res, k, concurrency=3,
                                  tuning=wavelib.Tuning(time_tile=1))
    for _ in range(2):
        g, ws = wavelib.grad_batched(grid, shots, tm, td, qd, res, k, concurrency=3)
        assert wavelib.status(ws) == wavelib.WAVE_OK
        torch.cuda.synchronize()
        assert torch.equal(g, ref)
    p = wavelib.describe_batch_plan(grid, shots, k, 3)
    assert p["lockstep"] and p["time_tile"] >= 1 and k % p["time_tile"] == 0
