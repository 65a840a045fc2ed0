"""GPU parity of the forward sweep (untiled and time-tiled) through the C ABI.

* every compiled (space order, T) variant against the FP64 oracle: rel-L2 of
  the final wavefield <= 1e-5 (the tolerance the target sets for FP32 after nt
  steps) and receiver traces within 1e-5 of max |d|;
* tiled == untiled bitwise (the paper's verification rule, Sec. 4.3 and
  Sec. 5.4.3), also across launch splits and x-chunks;
* edge cases: ragged shapes, z not a multiple of 4, minimum grid, nt = 1,
  no sparse points, shared source points, points on the upper faces;
* the 64^3 so-4 workload in full, and the 512^3 so-8 workload in the launch
  configuration the benchmark uses, compared with the oracle on a crop that
  holds the whole domain of dependence.
"""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _run(wavelib, dev, grid, m, damp, src, q, rec, T, tile_x=0, tile_y=0, kernel=0, rows=0):
    import torch
    d, ul, _, ws = wavelib.fwd(grid, _t(m, dev), _t(damp, dev), src, _t(q, dev) if len(src) else None,
                               rec, tuning=wavelib.Tuning(time_tile=T, tile_x=tile_x, tile_y=tile_y,
                                                          kernel=kernel, rows=rows),
                               want_u_last=True)
    assert wavelib.status(ws) == 0
    torch.cuda.synchronize()
    return d.cpu().numpy(), ul.cpu().numpy()


def _oracle(oracle, grid, m, damp, src, q, rec):
    f64 = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    h = [float(np.float32(v)) for v in grid.h]
    return oracle.forward(f64(m), f64(damp), h, float(np.float32(grid.dt)), grid.nt,
                          grid.space_order, f64(src) if len(src) else None,
                          f64(q) if len(src) else None, f64(rec) if len(rec) else None)


def _relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _variants():
    # (space order, T) pairs compiled into the library
    return [(2, 1), (2, 2), (2, 3), (2, 4), (4, 1), (4, 2), (4, 3), (4, 4), (6, 1), (6, 2),
            (8, 1), (8, 2), (10, 1), (12, 1), (14, 1), (16, 1)]


@pytest.mark.parametrize("so,T", _variants())
def test_forward_vs_oracle_and_untiled(wavelib, cuda, oracle, so, T):
    n = (45, 70, 83)  # ragged in every axis, nz not a multiple of 4
    nt = 31
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=so * 10 + T, nsrc=3, nrec=7)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    d, ul = _run(wavelib, cuda, grid, m, damp, src, q, rec, T)
    dref, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
    assert np.all(np.isfinite(ul)) and np.any(ul)
    assert _relerr(ul[0], uref[0]) <= TOL
    assert _relerr(ul[1], uref[1]) <= TOL
    assert np.abs(d - dref).max() <= TOL * np.abs(dref).max()
    if T > 1:
        d1, ul1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1)
        assert np.array_equal(ul, ul1)
        assert np.array_equal(d, d1)


@pytest.mark.parametrize("so,T,nt,tile_x", [(4, 4, 23, 0), (4, 3, 10, 17), (8, 2, 9, 9),
                                             (2, 4, 1, 0), (4, 2, 2, 40)])
def test_tiled_bitwise_across_splits(wavelib, cuda, so, T, nt, tile_x):
    # nt not a multiple of T (remainder launches use smaller T), odd x-chunks
    n = (61, 37, 50)
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=99, nsrc=2, nrec=4)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    d1, u1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1)
    dT, uT = _run(wavelib, cuda, grid, m, damp, src, q, rec, T, tile_x=tile_x)
    assert np.array_equal(u1, uT) and np.array_equal(d1, dT)
    assert np.any(u1)


@pytest.mark.parametrize("so", [4, 8, 16])
def test_edge_cases(wavelib, cuda, oracle, so):
    # minimum grid (n = so + 1), no receivers, shared source points, sources
    # and receivers on the upper faces
    n = (so + 1, so + 2, so + 3)
    nt = 12
    rng = np.random.default_rng(so)
    m = (1.0 / rng.uniform(1.5, 2.5, size=n) ** 2).astype(np.float32)
    damp = rng.random(n).astype(np.float32)
    ext = [(k - 1) * inputs.H for k in n]
    src = np.array([[ext[0], ext[1], ext[2]], [0.5 * ext[0], 0.3 * ext[1], 0.7 * ext[2]],
                    [0.5 * ext[0], 0.3 * ext[1], 0.7 * ext[2]]], dtype=np.float32)
    q = rng.standard_normal((nt, 3)).astype(np.float32)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 2.5)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    empty = np.zeros((0, 3), np.float32)
    for T in (1, 2):
        try:
            d, ul = _run(wavelib, cuda, grid, m, damp, src, q, empty, T)
        except wavelib.WaveError as e:
            assert e.code == wavelib.WAVE_EUNSUPPORTED and T > 1
            continue
        _, uref, _ = _oracle(oracle, grid, m, damp, src, q, empty)
        assert d.shape == (nt, 0)
        assert _relerr(ul[0], uref[0]) <= TOL
    # no sources at all: the field stays exactly zero
    _, ul = _run(wavelib, cuda, grid, m, damp, empty, np.zeros((nt, 0), np.float32), empty, 1)
    assert not np.any(ul)


def test_c1_workload_vs_oracle(wavelib, cuda, oracle):
    p = inputs.c1()
    grid = wavelib.Grid(p.n, p.h, p.dt, p.nt, p.space_order)
    dref, uref, _ = _oracle(oracle, grid, p.m, p.damp, p.src_xyz, p.src_q, p.rec_xyz)
    for T in (1, 2, 4):
        d, ul = _run(wavelib, cuda, grid, p.m, p.damp, p.src_xyz, p.src_q, p.rec_xyz, T)
        assert _relerr(ul[0], uref[0]) <= TOL
        # the direct wave has not reached these receivers yet (see the input
        # notes): traces are compared against the wavefield's scale
        assert np.abs(d - dref).max() <= TOL * np.abs(uref[0]).max()


def test_linearity_bitwise(wavelib, cuda):
    n = (40, 41, 42)
    nt = 20
    m, damp, src, q, rec = inputs.random_problem(n, 8, nt, seed=5)
    dt = 0.4 * wavelib.cfl_dt(8, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, 8)
    d1, u1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 2)
    d2, u2 = _run(wavelib, cuda, grid, m, damp, src, 2 * q, rec, 2)
    # Scaling by 2 commutes with every rounding except in the subnormal range,
    # where the rounding step is absolute (2^-149): bitwise there, one ulp below.
    # Values that passed through the subnormal range at any step carry that
    # absolute rounding, so compare bitwise only well above it.
    big = np.abs(2 * u1) >= 1e-30
    assert np.array_equal(u2[big], 2 * u1[big])
    assert np.abs(u2 - 2 * u1).max() <= 1e-36
    db = np.abs(2 * d1) >= 1e-30
    assert np.array_equal(d2[db], 2 * d1[db])


def test_status_flags(wavelib, cuda):
    import torch
    n = (20, 20, 20)
    m = np.full(n, 1 / 4.0, np.float32)
    damp = np.zeros(n, np.float32)
    grid = wavelib.Grid(n, (inputs.H,) * 3, 10 * wavelib.cfl_dt(4, (inputs.H,) * 3, 2.0), 3, 4)
    _, _, _, ws = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), tuning=wavelib.Tuning(time_tile=1))
    assert wavelib.status(ws) == wavelib.WAVE_EUNSTABLE
    m[3, 4, 5] = -1.0
    grid.dt = 0.4 * wavelib.cfl_dt(4, (inputs.H,) * 3, 2.0)
    _, _, _, ws = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), tuning=wavelib.Tuning(time_tile=1))
    assert wavelib.status(ws) == wavelib.WAVE_EINVAL
    torch.cuda.synchronize()


def test_c2_full_grid_crop_vs_oracle(wavelib, cuda, oracle):
    # 512^3 so 8 (two layers + noise, 40-point damping) in the benchmark's
    # launch configuration.  After nt steps the field is supported within
    # r * nt cells of the source (the stencil reaches r cells per step), so a
    # crop holding that region reproduces it exactly in exact arithmetic.
    import torch
    nt = 24
    p = inputs.c2(nt=nt)
    r = p.space_order // 2
    grid = wavelib.Grid(p.n, p.h, p.dt, nt, p.space_order)
    tm, td, tq = _t(p.m, cuda), _t(p.damp, cuda), _t(p.src_q, cuda)
    out = {}
    for T in (1, 2):
        d, ul, _, ws = wavelib.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz,
                                   tuning=wavelib.Tuning(time_tile=T), want_u_last=True)
        assert wavelib.status(ws) == 0
        out[T] = (d.cpu().numpy(), ul.cpu().numpy())
        del d, ul, ws
        torch.cuda.empty_cache()
    assert np.array_equal(out[1][1], out[2][1]) and np.array_equal(out[1][0], out[2][0])
    s = (np.asarray(p.src_xyz[0]) / inputs.H).round().astype(int)
    half = r * nt + 2
    lo = [max(0, s[a] - half) for a in range(3)]
    hi = [min(p.n[a], s[a] + half + 2) for a in range(3)]
    sl = tuple(slice(lo[a], hi[a]) for a in range(3))
    keep = [i for i in range(len(p.rec_xyz))
            if all(lo[a] * inputs.H <= p.rec_xyz[i, a] <= (hi[a] - 2) * inputs.H for a in range(3))]
    # shift the points in float64 so that x/h keeps its fraction exactly (an
    # FP32 shift moves near-node fractions by ~1e-6 of a cell)
    shift = np.array([lo[a] * float(np.float32(inputs.H)) for a in range(3)], np.float64)
    cgrid = wavelib.Grid(tuple(hi[a] - lo[a] for a in range(3)), p.h, p.dt, nt, p.space_order)
    dref, uref, _ = _oracle(oracle, cgrid, p.m[sl], p.damp[sl],
                            p.src_xyz.astype(np.float64) - shift, p.src_q,
                            p.rec_xyz[keep].astype(np.float64) - shift)
    u = out[1][1][0]
    assert np.abs(u).sum() == pytest.approx(np.abs(u[sl]).sum(), rel=1e-12)  # support inside the crop
    assert _relerr(u[sl], uref[0]) <= TOL
    d = out[1][0][:, keep]
    assert np.abs(d - dref).max() <= TOL * np.abs(dref).max()


@pytest.mark.parametrize("so", [2, 4, 6, 8, 10, 12, 14, 16])
def test_every_compiled_variant(wavelib, cuda, oracle, so):
    # every (T, tile, vec, prefetch) variant compiled for this order: bitwise
    # equal to the untiled default, and at parity with the oracle
    n = (37, 45, 51)
    nt = 13
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=so + 1000, nsrc=2, nrec=5)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    d1, u1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1)
    _, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
    assert _relerr(u1[0], uref[0]) <= TOL
    variants = wavelib.list_variants(so)
    assert len(variants) >= 1
    for v in variants:
        import torch
        dv, uv, _, ws = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), src, _t(q, cuda), rec,
                                    tuning=wavelib.Tuning(time_tile=v["time_tile"], tile_y=v["tile_y"],
                                                          vec=v["vec"], tile_z=v["tile_z"],
                                                          kernel=v["kernel"], rows=v["rows"]),
                                    want_u_last=True)
        assert wavelib.status(ws) == 0
        torch.cuda.synchronize()
        assert np.array_equal(uv.cpu().numpy(), u1), v
        assert np.array_equal(dv.cpu().numpy(), d1), v


def test_bounded_wait_timeout_reports_status(wavelib, cuda, oracle):
    # The test hook withholds every TMA load of the sweep, so each consumer's
    # bounded mbarrier wait runs out (~2 s); the call must report
    # WAVE_ETIMEOUT through wave_status and leave the context usable.
    import torch
    n, so, nt = (20, 18, 24), 4, 1
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=77)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    tune = wavelib.Tuning(time_tile=1, flags=wavelib.WAVE_TEST_WITHHOLD)
    _, _, _, ws = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), src, _t(q, cuda), rec, tuning=tune)
    assert wavelib.status(ws) == wavelib.WAVE_ETIMEOUT
    # the context still works: a normal call right after is correct
    d, ul = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1)
    _, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
    assert _relerr(ul[0], uref[0]) <= TOL
    torch.cuda.synchronize()


def test_chunk_sizes_in_any_order(wavelib, cuda, oracle):
    # A large x-chunk, then a shape whose default-chunk search queries many
    # smaller chunks, then a mid-size chunk: every launch of the same kernel
    # must get the dynamic shared memory it asks for.
    so, nt = 8, 6
    for n, tile_x in (((96, 20, 24), 96), ((300, 18, 20), 0), ((80, 20, 24), 40)):
        m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=3)
        dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
        grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
        d, ul = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1, tile_x=tile_x)
        _, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
        assert _relerr(ul[0], uref[0]) <= TOL


@pytest.mark.parametrize("so,T,kernel", [(2, 1, 0), (2, 2, 0), (2, 4, 0), (8, 1, 0), (16, 1, 0),
                                         (4, 2, 2), (8, 2, 2), (8, 1, 2)])
def test_dense_receiver_carpet(wavelib, cuda, oracle, so, T, kernel):
    """A carpet of receivers: a 21 x 23 grid of off-grid points at one depth
    plus a few more scattered points, so that one block holds hundreds of
    record entries across its planes (more than it has threads), several
    per plane and grid point.  Traces against the oracle, and against the
    untiled sweep bit for bit."""
    n = (36, 40, 44)
    nt = 14
    m, damp, src, q, _ = inputs.random_problem(n, so, nt, seed=7 + so + T, nsrc=2, nrec=1)
    gx, gy = np.meshgrid(np.linspace(1.3, n[0] - 2.6, 21), np.linspace(0.7, n[1] - 3.2, 23), indexing="ij")
    carpet = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 3.4)], axis=1)
    extra = np.random.default_rng(3).random((40, 3)) * (np.array(n) - 1)
    rec = (np.concatenate([carpet, extra]) * inputs.H).astype(np.float32)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    d, ul = _run(wavelib, cuda, grid, m, damp, src, q, rec, T, tile_x=12, kernel=kernel)
    dref, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
    assert np.abs(d - dref).max() <= TOL * np.abs(dref).max()
    assert _relerr(ul[0], uref[0]) <= TOL
    if T > 1 or kernel:
        d1, ul1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1, kernel=wavelib.WAVE_KERNEL_SHARED)
        assert np.array_equal(d, d1) and np.array_equal(ul, ul1)


@pytest.mark.parametrize("so", [4, 8, 14, 16])
def test_staged_kernel_splits_bitwise(wavelib, cuda, oracle, so):
    """The stage-specialised sweep (each time step of a tile on its own
    warps) at T = 1 and 2 and both rows-per-thread shapes, with x-chunks from
    5 planes (shorter than the stencil reach 2RT) to the whole grid and an
    odd step count (the last step of T = 2 falls back to T = 1): bitwise
    equal to the untiled sweep of the other kernel family, which is at parity
    with the oracle.  Sources sit on chunk and tile boundaries."""
    n = (41, 53, 61)
    nt = 11
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=90 + so, nsrc=3, nrec=9)
    src[0] = np.array([10.0, 16.0, 28.0], np.float32) * inputs.H  # on x/y/z tile edges
    src[1] = np.array([20.5, 15.5, 27.5], np.float32) * inputs.H
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    d1, u1 = _run(wavelib, cuda, grid, m, damp, src, q, rec, 1, kernel=wavelib.WAVE_KERNEL_SHARED)
    dref, uref, _ = _oracle(oracle, grid, m, damp, src, q, rec)
    assert _relerr(u1[0], uref[0]) <= TOL
    assert np.abs(d1 - dref).max() <= TOL * np.abs(dref).max()
    shapes = [(v["time_tile"], v["rows"], v["tile_y"], v["tile_z"]) for v in wavelib.list_variants(so)
              if v["kernel"] == wavelib.WAVE_KERNEL_STAGED]
    assert shapes
    for T, rows, ty, tz in shapes:
        for tile_x in (5, 10, 23, n[0]):
            import torch
            d, ul, _, ws = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), src, _t(q, cuda), rec,
                                       tuning=wavelib.Tuning(time_tile=T, tile_x=tile_x, tile_y=ty, tile_z=tz,
                                                             kernel=wavelib.WAVE_KERNEL_STAGED, rows=rows),
                                       want_u_last=True)
            assert wavelib.status(ws) == 0
            torch.cuda.synchronize()
            assert np.array_equal(ul.cpu().numpy(), u1), (T, rows, ty, tz, tile_x)
            assert np.array_equal(d.cpu().numpy(), d1), (T, rows, ty, tz, tile_x)
