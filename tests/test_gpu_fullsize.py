"""Parity at the full sizes of the 768 x 768 x 512 sweep (c3) and the FWI
gradient (c4).

* c3, space orders 4/8/12/16: the deepest compiled time tile is bitwise equal
  to the untiled sweep on the whole grid, and the untiled field matches the
  FP64 oracle (rel-L2 <= 1e-5) on a crop that holds the whole domain of
  dependence of the source after nt steps (r * nt cells per side).
* c4, 256^3, 2000 steps, checkpoints every 50: the gradient of
  J = 1/2 |d(m) - d_obs|^2 through the autograd Function matches central
  finite differences of J along 8 seeded random directions.
"""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


@pytest.fixture(scope="module")
def c3_model():
    p = inputs.c3(space_order=4, nt=2)
    return p.m, p.damp


@pytest.mark.parametrize("so,nt", [(4, 30), (8, 20), (12, 14), (16, 12)])
def test_c3_full_grid(wavelib, cuda, oracle, c3_model, so, nt):
    import torch
    m, damp = c3_model
    n = m.shape
    h = (inputs.H,) * 3
    dt = inputs.DT[("c3", so)]
    src = np.array([[n[0] // 2 * inputs.H, n[1] // 2 * inputs.H, 2 * inputs.H]], np.float32)
    q = inputs.ricker(15.0, dt, nt)[:, None]
    grid = wavelib.Grid(n, h, dt, nt, so)
    tm, td, tq = _t(m, cuda), _t(damp, cuda), _t(q, cuda)
    deepest = max(v["time_tile"] for v in wavelib.list_variants(so))
    out = {}
    for T in sorted({1, deepest}):
        _, ul, _, ws = wavelib.fwd(grid, tm, td, src, tq, None, tuning=wavelib.Tuning(time_tile=T),
                                   want_u_last=True)
        assert wavelib.status(ws) == 0
        out[T] = ul[0].cpu().numpy()
        del ul, ws
        torch.cuda.empty_cache()
    assert np.array_equal(out[1], out[deepest])
    r = so // 2
    s = (src[0] / inputs.H).round().astype(int)
    half = r * nt + 2
    lo = [max(0, s[a] - half) for a in range(3)]
    hi = [min(n[a], s[a] + half + 2) for a in range(3)]
    sl = tuple(slice(lo[a], hi[a]) for a in range(3))
    shift = np.array([lo[a] * float(np.float32(inputs.H)) for a in range(3)], np.float64)
    hh = [float(np.float32(v)) for v in h]
    _, uref, _ = oracle.forward(np.float64(m[sl]), np.float64(damp[sl]), hh, float(np.float32(dt)), nt,
                                so, src_xyz=src.astype(np.float64) - shift, src_q=np.float64(q))
    u = out[1]
    assert np.abs(u).sum() == pytest.approx(np.abs(u[sl]).sum(), rel=1e-12)  # support inside the crop
    err = float(np.linalg.norm(np.float64(u[sl]) - uref[0]) / np.linalg.norm(uref[0]))
    assert err <= TOL, err


def test_c4_gradient_finite_differences(wavelib, cuda):
    import torch
    from paper_1806_08299_gb300.autograd import modeling
    pt = inputs.c4(nt=2000, true_model=True)
    p0 = inputs.c4(nt=2000, true_model=False)
    grid = wavelib.Grid(p0.n, p0.h, p0.dt, p0.nt, p0.space_order)
    td, tq = _t(p0.damp, cuda), _t(p0.src_q, cuda)
    k = 50
    d_obs, _, _, _ = wavelib.fwd(grid, _t(pt.m, cuda), td, pt.src_xyz, tq, pt.rec_xyz)
    d_obs = d_obs.double()

    def misfit(mm):
        d, _, _, ws = wavelib.fwd(grid, mm, td, p0.src_xyz, tq, p0.rec_xyz)
        assert wavelib.status(ws) == 0
        return 0.5 * float(((d.double() - d_obs) ** 2).sum())

    m0 = _t(p0.m, cuda).requires_grad_(True)
    d = modeling(m0, grid, td, p0.src_xyz, tq, p0.rec_xyz, ckpt_every=k)
    loss = 0.5 * ((d.double() - d_obs) ** 2).sum()
    loss.backward()
    g = m0.grad.double()
    assert torch.isfinite(g).all()
    j0 = float(loss)
    assert j0 > 0
    rng = np.random.default_rng(4)
    n = p0.n
    report = []
    idx = [np.arange(v) for v in n]
    x, y, z = np.meshgrid(*idx, indexing="ij", sparse=True)
    for i in range(8):
        # a random smooth bump of compact support (radius 2w) around the
        # anomaly, away from the source and receivers near the surface
        c = [n[0] // 2 + rng.integers(-30, 31), n[1] // 2 + rng.integers(-30, 31),
             n[2] // 2 + rng.integers(-30, 31)]
        w = rng.uniform(8.0, 20.0)
        r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * w)
        dm = (rng.choice([-1.0, 1.0]) * np.where(r < 1.0, np.cos(0.5 * np.pi * r) ** 2, 0.0)).astype(np.float32)
        eps = 5e-3 * float(p0.m.max())
        tdm = _t(dm, cuda)
        with torch.no_grad():
            mp = (m0 + eps * tdm).contiguous()
            mm = (m0 - eps * tdm).contiguous()
            jp = misfit(mp)
            jm = misfit(mm)
            # the perturbation FP32 actually applied: m0 = 0.25 sits on a binade
            # edge, where m + e and m - e round with different spacings
            applied = (mp.double() - mm.double()) / 2
        fd = (jp - jm) / (2 * eps)
        want = float((g * applied).sum()) / eps
        # Each FP32 misfit carries relative error up to ~2e-5 (the forward's
        # 1e-5 parity bound on the traces), so the difference quotient is
        # uncertain by up to 2e-5 J / eps on top of 1 % for truncation.
        floor = 2e-5 * max(j0, jp, jm) / eps
        # which bound decides this direction, and the relative error reached
        report.append((i, fd, want, abs(fd - want) / abs(want), floor / abs(want)))
        print("c4 FD direction %d: fd %.6e  adjoint %.6e  rel.err %.2e  floor/|adjoint| %.2e" % report[-1])
        assert abs(fd - want) <= 1e-2 * abs(want) + floor, (i, fd, want, floor)
