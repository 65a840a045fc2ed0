"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module only builds inputs: velocity models, absorbing-layer damping
profiles, source wavelets and acquisition geometry.  It contains none of the
wave solver's arithmetic.  The paper measures its acoustic operator on a
512^3 grid with deterministically generated input (Sec. 5.8.1-5.8.2); it
publishes no dataset, so every workload here is synthetic:

  c1  64^3, h = 10 m, so 4, constant 1.5 km/s, no damping, 100 steps,
      Ricker 10 Hz at the centre, 32 receivers on a line at depth 2h.
  c2  512^3, so 8, two layers 1.5/2.5 km/s (interface at half depth) with
      +-2% uniform noise, 40-point damping layer, 1000 steps, Ricker 15 Hz,
      512 receivers.
  c3  768 x 768 x 512, so 4/8/12/16, smooth random velocity 1.5-4.5 km/s
      (smoothed seeded noise), 40-point damping layer, 500 steps, one source.
  c4  FWI gradient, 256^3, so 8, 2.0 km/s with a 30-point sphere of
      2.2 km/s (true) or without it (initial), 2000 steps, 256 receivers.
  c5  survey of 64 shots, each a window of one 512 x 512 x 256 model (four
      layers 1.5 -> 3.0 km/s and a Gaussian anomaly), window sizes
      nx, ny ~ U{128..320}, nz ~ U{128..256} at seeded offsets, one Ricker
      10 Hz source and 128 receivers per shot, 1500 steps, so 8.

dt is fixed per workload as a literal just below half the von Neumann limit
of the scheme for the model's largest velocity (the tests check these
literals against the oracle's limit).
"""
import math
from dataclasses import dataclass, field

import numpy as np

H = 0.01  # km (10 m)
DAMP_WIDTH = 40

# dt (s) just below 0.5 x the stability limit for (space order, v_max)
DT = {
    ("c1", 4): 1.666e-3,   # v_max 1.5
    ("c2", 8): 0.887e-3,   # v_max 2.5 * 1.02
    ("c3", 4): 0.555e-3,   # v_max 4.5
    ("c3", 8): 0.503e-3,
    ("c3", 12): 0.482e-3,
    ("c3", 16): 0.470e-3,
    ("c4", 8): 1.029e-3,   # v_max 2.2
    ("c5", 8): 0.752e-3,   # v_max 3.01 (layer 3.0 plus the anomaly tail)
}
V_MAX = {"c1": 1.5, "c2": 2.5 * 1.02, "c3": 4.5, "c4": 2.2, "c5": 3.01}


@dataclass
class Problem:
    name: str
    n: tuple
    h: tuple
    dt: float
    nt: int
    space_order: int
    m: np.ndarray                # float32 [nx][ny][nz], s^2/km^2
    damp: np.ndarray             # float32 [nx][ny][nz], 1/s
    src_xyz: np.ndarray          # float32 [nsrc][3], km
    src_q: np.ndarray            # float32 [nt][nsrc]
    rec_xyz: np.ndarray          # float32 [nrec][3], km
    extra: dict = field(default_factory=dict)

    @property
    def points(self):
        return int(np.prod(self.n))


def ricker(f0, dt, nt, t0=None):
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0,
    t = n dt, t0 = 1/f0 by default; computed in float64, returned as float32."""
    t0 = 1.0 / f0 if t0 is None else t0
    tau = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * tau) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def damping_profile(n, h, v_max, width=DAMP_WIDTH):
    """Separable absorbing layer: damp = p_x + p_y + p_z with
    p(d) = d0 (d/width)^2 for a point d cells into the layer (0 inside) and
    d0 = 3 v_max ln(1000) / (2 width h)."""
    out = np.zeros(n, dtype=np.float64)
    for a in range(3):
        idx = np.arange(n[a], dtype=np.float64)
        d = np.maximum(np.maximum(width - idx, idx - (n[a] - 1 - width)), 0.0)
        d0 = 3.0 * v_max * math.log(1000.0) / (2.0 * width * h[a])
        p = d0 * (d / width) ** 2
        shape = [1, 1, 1]
        shape[a] = n[a]
        out = out + p.reshape(shape)
    return out.astype(np.float32)


def _line_x(nrec, n, h, y, z):
    x = np.linspace(0.0, (n[0] - 1) * h[0], nrec)
    return np.stack([x, np.full(nrec, y * h[1]), np.full(nrec, z * h[2])], axis=1).astype(np.float32)


def c1(nt=100):
    n = (64, 64, 64)
    h = (H, H, H)
    dt = DT[("c1", 4)]
    m = np.full(n, 1.0 / 1.5 ** 2, dtype=np.float32)
    damp = np.zeros(n, dtype=np.float32)
    src = np.array([[32 * H, 32 * H, 32 * H]], dtype=np.float32)
    q = ricker(10.0, dt, nt)[:, None]
    rec = _line_x(32, n, h, 32, 2)
    return Problem("c1", n, h, dt, nt, 4, m, damp, src, q, rec)


def c2(nt=1000, n=(512, 512, 512), seed=2):
    """Two-layer model with uniform noise; source and receivers near the top."""
    h = (H, H, H)
    dt = DT[("c2", 8)]
    rng = np.random.default_rng(seed)
    v = np.where(np.arange(n[2]) < n[2] // 2, 1.5, 2.5).astype(np.float32)[None, None, :]
    v = v * (1.0 + rng.uniform(-0.02, 0.02, size=n).astype(np.float32))
    m = (1.0 / (v * v)).astype(np.float32)
    damp = damping_profile(n, h, V_MAX["c2"])
    src = np.array([[n[0] // 2 * H, n[1] // 2 * H, 2 * H]], dtype=np.float32)
    q = ricker(15.0, dt, nt)[:, None]
    rec = np.stack([np.arange(n[0]) * H, np.full(n[0], n[1] // 2 * H), np.full(n[0], 2 * H)],
                   axis=1).astype(np.float32)
    return Problem("c2", tuple(n), h, dt, nt, 8, m, damp, src, q, rec)


def smooth_velocity(n, seed, vmin=1.5, vmax=4.5, coarse=8):
    """Smooth random velocity: seeded N(0,1) noise on a grid `coarse` times
    coarser, a 3-point binomial smoothing, trilinear upsampling, and a
    min-max rescale to [vmin, vmax]."""
    rng = np.random.default_rng(seed)
    cn = [max(2, (k + coarse - 1) // coarse + 1) for k in n]
    g = rng.standard_normal(cn)
    for a in range(3):
        g = 0.25 * np.roll(g, 1, a) + 0.5 * g + 0.25 * np.roll(g, -1, a)
    out = g
    for a in range(3):
        pos = np.arange(n[a]) / coarse
        i0 = np.minimum(np.floor(pos).astype(int), cn[a] - 2)
        f = (pos - i0).reshape([-1 if b == a else 1 for b in range(3)])
        out = (np.take(out, i0, axis=a) * (1 - f) + np.take(out, i0 + 1, axis=a) * f)
    lo, hi = out.min(), out.max()
    return (vmin + (vmax - vmin) * (out - lo) / (hi - lo)).astype(np.float32)


def c3(space_order=8, nt=500, n=(768, 768, 512), seed=3):
    h = (H, H, H)
    dt = DT[("c3", space_order)]
    v = smooth_velocity(n, seed)
    m = (1.0 / (v * v)).astype(np.float32)
    damp = damping_profile(n, h, V_MAX["c3"])
    src = np.array([[n[0] // 2 * H, n[1] // 2 * H, 2 * H]], dtype=np.float32)
    q = ricker(15.0, dt, nt)[:, None]
    rec = np.zeros((0, 3), dtype=np.float32)
    return Problem("c3", tuple(n), h, dt, nt, space_order, m, damp, src, q, rec)


def c4(nt=2000, n=(256, 256, 256), true_model=True):
    h = (H, H, H)
    dt = DT[("c4", 8)]
    idx = [np.arange(k) for k in n]
    x, y, z = np.meshgrid(*idx, indexing="ij", sparse=True)
    c = [k // 2 for k in n]
    inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= 30 ** 2
    v = np.full(n, 2.0, dtype=np.float32)
    if true_model:
        v = np.where(inside, np.float32(2.2), v)
    m = (1.0 / (v * v)).astype(np.float32)
    damp = damping_profile(n, h, V_MAX["c4"])
    src = np.array([[n[0] // 2 * H, n[1] // 2 * H, 2 * H]], dtype=np.float32)
    q = ricker(10.0, dt, nt)[:, None]
    rec = np.stack([np.arange(n[0]) * H, np.full(n[0], n[1] // 2 * H), np.full(n[0], 2 * H)],
                   axis=1).astype(np.float32)
    return Problem("c4", tuple(n), h, dt, nt, 8, m, damp, src, q, rec,
                   extra={"anomaly_mask": inside})


def random_problem(n, space_order, nt, seed, nsrc=2, nrec=5, damp_scale=3.0, h=(H, H, H),
                   v_range=(1.5, 3.0)):
    """Small heterogeneous problem for parity tests: random smooth-ish model,
    random damping, random off-node sources and receivers, random traces."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(*v_range, size=n).astype(np.float32)
    m = (1.0 / (v * v)).astype(np.float32)
    damp = (damp_scale * rng.random(n)).astype(np.float32)
    ext = np.array([(n[a] - 1) * h[a] for a in range(3)])
    src = (rng.random((nsrc, 3)) * ext).astype(np.float32)
    rec = (rng.random((nrec, 3)) * ext).astype(np.float32)
    q = rng.standard_normal((nt, nsrc)).astype(np.float32)
    return m, damp, src, q, rec


@dataclass
class Survey:
    name: str
    n: tuple                     # global grid
    h: tuple
    dt: float
    nt: int
    space_order: int
    m: np.ndarray                # float32 global [nx][ny][nz]
    damp: np.ndarray             # float32 global
    shots: list                  # dicts: origin, n, src_xyz, rec_xyz (window-relative, km)
    src_q: list                  # float32 [nt][nsrc_s] per shot

    @property
    def updates_per_sweep(self):
        """Grid-point updates of one sweep over every shot's window."""
        return int(sum(int(np.prod(s["n"])) for s in self.shots)) * self.nt


def c5(nshots=64, nt=1500, n=(512, 512, 256), seed=5, true_model=True):
    """Windowed-shot survey.  The global model has four layers in depth
    (1.5, 2.0, 2.5, 3.0 km/s) and, for the true model, a Gaussian anomaly of
    +0.2 km/s (radius parameter 24 cells) at mid depth; a 40-point damping
    layer lines the global boundary.  Shot s: window extent nx, ny ~
    U{128..320}, nz ~ U{128..256} (clipped to the grid) at a uniform offset
    that keeps it inside, one Ricker 10 Hz source at the window's top centre
    (depth 2h) and 128 receivers on a line along x at the window's centre y,
    depth 2h."""
    h = (H, H, H)
    dt = DT[("c5", 8)]
    rng = np.random.default_rng(seed)
    z = np.arange(n[2])
    v1 = np.choose(np.minimum(4 * z // n[2], 3), [1.5, 2.0, 2.5, 3.0]).astype(np.float32)
    v = np.ascontiguousarray(np.broadcast_to(v1[None, None, :], n), dtype=np.float32)
    if true_model:
        idx = [np.arange(k) for k in n]
        x, y, zz = np.meshgrid(*idx, indexing="ij", sparse=True)
        r2 = (x - n[0] // 2) ** 2 + (y - n[1] // 2) ** 2 + (zz - n[2] // 2) ** 2
        v = v + (0.2 * np.exp(-r2 / (2.0 * 24.0 ** 2))).astype(np.float32)
    m = (1.0 / (v * v)).astype(np.float32)
    damp = damping_profile(n, h, V_MAX["c5"])
    shots, qs = [], []
    w = ricker(10.0, dt, nt)[:, None]
    for _ in range(nshots):
        k = [min(int(rng.integers(128, 321)), n[0]), min(int(rng.integers(128, 321)), n[1]),
             min(int(rng.integers(128, 257)), n[2])]
        o = [int(rng.integers(0, n[a] - k[a] + 1)) for a in range(3)]
        src = np.array([[(k[0] // 2) * H, (k[1] // 2) * H, 2 * H]], dtype=np.float32)
        rec = np.stack([np.linspace(0.0, (k[0] - 1) * H, 128), np.full(128, (k[1] // 2) * H),
                        np.full(128, 2 * H)], axis=1).astype(np.float32)
        shots.append({"origin": tuple(o), "n": tuple(k), "src_xyz": src, "rec_xyz": rec})
        qs.append(w.copy())
    return Survey("c5", tuple(n), h, dt, nt, 8, m, damp, shots, qs)
