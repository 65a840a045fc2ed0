"""The host-side traffic model (paper_1806_08299_gb300/traffic_model.py):
closed forms of its DRAM figures and of the TMA box bytes of a shape."""
import pytest

from paper_1806_08299_gb300 import traffic_model as tm


def test_dram_bytes_closed_forms():
    assert tm.dram_bytes_per_update(1) == 20.0
    assert tm.dram_bytes_per_update(2) == 12.0
    assert tm.dram_bytes_per_update(4) == 6.0
    assert tm.dram_bytes_per_update(1, "recompute") == 28.0
    assert tm.dram_bytes_per_update(1, "imaging") == 32.0
    with pytest.raises(ValueError):
        tm.dram_bytes_per_update(2, "imaging")
    assert tm.roof_gpts(20.0, 6696.2) == pytest.approx(334.81)


def test_l2_bytes_of_the_default_so8_shape():
    # 64x8 tile, R = 4: centre box 80 x 16, K boxes 72 x 8, no ring U (split)
    s = tm.Shape(R=4, T=1, V=4, BZ=64, BY=8)
    assert (s.PW, s.H0, s.W0, s.HK, s.split) == (80, 16, 72, 8, True)
    per_plane = 4 * 80 * 16 + 4 * (4 * 72 * 8)
    assert tm.l2_bytes_per_update(s) == per_plane / (64 * 8)


def test_l2_bytes_fall_with_tile_size_and_depth_shares_the_load():
    small = tm.l2_bytes_per_update(tm.Shape(R=2, T=2, V=4, BZ=56, BY=12))
    wide = tm.l2_bytes_per_update(tm.Shape(R=2, T=2, V=4, BZ=120, BY=14))
    assert wide < small
    # a ring-U shape (R <= 2) loads its centre box once per plane, no separate feed box
    s = tm.Shape(R=2, T=1, V=8, BZ=64, BY=16)
    assert not s.split
    assert tm.l2_bytes_per_update(s) == (4 * s.PW * s.H0 + 3 * 4 * s.W0 * s.HK) / (64 * 16)


def test_staged_shape_boxes_and_redundancy():
    # depth-2 staged 64 x 24 tile at so 8: stage 1 covers 72 x 32 (RP = 4 columns,
    # R = 4 rows per side), its centre box 80 x 40; stage 2 loads three 64 x 24 boxes
    s = tm.Shape(R=4, T=2, V=4, BZ=64, BY=24, kernel=2)
    assert (s.W1, s.H1) == (72, 32)
    per_plane = 4 * 80 * 40 + 4 * 4 * 72 * 32 + 3 * 4 * 64 * 24
    assert tm.l2_bytes_per_update(s) == per_plane / (64 * 24 * 2)
    assert s.stage_points_per_update() == (72 * 32 + 64 * 24) / (2 * 64 * 24)
    # the untiled staged sweep computes each point once and loads its own tile
    u = tm.Shape(R=4, T=1, V=4, BZ=64, BY=16, kernel=2)
    assert (u.W1, u.H1, u.stage_points_per_update()) == (64, 16, 1.0)
    assert tm.l2_bytes_per_update(u) == (4 * 72 * 24 + 4 * 4 * 64 * 16) / (64 * 16)
