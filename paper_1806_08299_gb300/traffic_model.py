"""Traffic model of the sweep kernels (host-side arithmetic, no GPU).

The tile-face estimate of Sec. 5.3 counts, for a tile, the bytes that cross
its faces per update.  On the GPU the faces are two: HBM <-> L2 and L2 <->
shared memory.

* DRAM: a launch of depth T reads u^n, u^{n-1}, B, C once and writes
  levels n+T and n+T-1 (one level for T = 1, written in place), when the
  overlapping halos of neighbouring blocks and the x-halo planes of
  neighbouring chunks are served by L2.  That gives 20 B per point-update
  untiled and 24/T for depth T.  The gradient modes add their extra arrays.
* L2 -> SM: the TMA boxes a block loads per x-plane, divided by the points
  it outputs per plane and per step.  Halo rows and columns are counted
  every time, so this is the figure that grows as tiles shrink.

`dram_bytes_per_update` is the algorithmic figure that the benchmark's
roofline uses; `l2_bytes_per_update` is the on-chip load the shape implies.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Shape:
    """A compiled sweep shape: radius R, depth T, z-points per thread V,
    output tile BZ x BY, gradient-mode extra boxes XB, kernel family
    (1: every stage of a tile on the same warps, sweep.cuh; 2: one group of
    warps per stage, tsweep.cuh)."""
    R: int
    T: int
    V: int
    BZ: int
    BY: int
    XB: int = 0
    kernel: int = 1

    @property
    def RT(self):
        return self.R * self.T

    @property
    def A0(self):
        return (self.RT + 3) // 4 * 4           # z halo, 16-byte aligned

    @property
    def W0(self):
        return self.BZ + 2 * self.A0              # K-box width

    @property
    def H0(self):
        return self.BY + 2 * self.RT              # layout rows

    @property
    def RP(self):
        return (self.R + 3) // 4 * 4

    @property
    def PW(self):
        return self.W0 + 2 * self.RP              # centre-box width

    @property
    def HK(self):
        return self.H0 - 2 * self.R               # K-box rows

    @property
    def split(self):
        return self.T == 1 and self.R >= 3        # no ring U: centre and x-queue boxes per slot

    # the stage-specialised sweep: stage 1 covers the tile widened by the
    # halo stage 2 reads, (T-1)R rows and (T-1)RP columns per side
    @property
    def W1(self):
        return self.BZ + 2 * (self.T - 1) * self.RP

    @property
    def H1(self):
        return self.BY + 2 * (self.T - 1) * self.R

    def stage_points_per_update(self):
        """Point updates computed per output point-update: stage 1 repeats
        the halo that stage 2 reads."""
        if self.kernel == 2:
            return (self.W1 * self.H1 + (self.T - 1) * self.BZ * self.BY) / (self.T * self.BZ * self.BY)
        return 1.0


def dram_bytes_per_update(T, mode="wave"):
    """Algorithmic DRAM bytes per point-update of one sweep of depth T.

    mode: 'wave' (forward / adjoint), 'recompute' (also reads E and writes
    the second difference D), 'imaging' (also reads D and reads and writes
    the gradient accumulator G).  The gradient modes run untiled (T = 1)."""
    if T < 1:
        raise ValueError("T >= 1")
    base = 20.0 if T == 1 else 24.0 / T
    extra = {"wave": 0.0, "recompute": 8.0, "imaging": 12.0}[mode]
    if extra and T != 1:
        raise ValueError("gradient modes are untiled")
    return base + extra


def l2_bytes_per_update(s):
    """Bytes a block loads from L2 through TMA per output point-update."""
    if s.kernel == 2:
        # per plane: the centre box of stage 1 (its region with the stencil
        # halo), level n, n-1, B and C over its region, and for T = 2 level
        # n, B and C over the tile for stage 2
        cbox = 4 * (s.W1 + 2 * s.RP) * (s.H1 + 2 * s.R)
        per_plane = cbox + 4 * 4 * s.W1 * s.H1 + (3 * 4 * s.BZ * s.BY if s.T == 2 else 0)
        return per_plane / (s.BZ * s.BY * s.T)
    ubox = 4 * s.PW * s.H0                       # haloed level-n plane
    kbox = 4 * s.W0 * s.HK                       # u^{n-1}, B, C (and XB extras) per plane
    per_plane = ubox + (3 + s.XB) * kbox + (kbox if s.split else 0)
    return per_plane / (s.BZ * s.BY * s.T)


def roof_gpts(bytes_per_update, gbs):
    """GPts/s at a bandwidth of gbs GB/s."""
    return gbs / bytes_per_update
