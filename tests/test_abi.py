"""CPU-side checks of the C ABI: the library loads, exports every function
include/wave.h declares, and its host-only functions (coefficients, stability
limit, workspace sizing, argument checks) behave; no kernel is launched."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(wave_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(wavelib):
    names = _declared()
    assert len(names) >= 10
    lib = ctypes.CDLL(wavelib.library_path())
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(wavelib.EXPORTED) == names


def test_coefficients_match_oracle(wavelib, oracle):
    for so in range(2, 17, 2):
        want = [float(v) for v in oracle.fd2_central_weights(so)]
        got = wavelib.fd_coefficients(so)
        assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_cfl_matches_oracle(wavelib, oracle):
    h32 = [float(np.float32(v)) for v in (0.01, 0.012, 0.02)]
    for so in (2, 4, 8, 12, 16):
        assert wavelib.cfl_dt(so, h32, 2.5) == pytest.approx(oracle.cfl_dt(so, h32, 2.5), rel=1e-6)


def test_workspace_and_ckpt_sizes(wavelib):
    g = wavelib.Grid((33, 34, 35), (0.01,) * 3, 1e-3, 40, 8)
    npad = 33 * 34 * 40  # z padded to a multiple of 8
    fwd = wavelib.workspace_bytes(g, wavelib.WAVE_OP_FWD, 2, 5)
    assert fwd >= 6 * 4 * npad + 40 * 8 * 5 * 4
    assert fwd % 256 == 0
    grad = wavelib.workspace_bytes(g, wavelib.WAVE_OP_GRAD, 2, 5, ckpt_every=7)
    assert grad >= (3 + 4 + 4 + 1 + 7) * 4 * npad
    assert wavelib.ckpt_bytes(g, 7) == 6 * 2 * 4 * npad
    assert wavelib.workspace_bytes(g, wavelib.WAVE_OP_GRAD, 2, 5, ckpt_every=0) == 0
    bad = wavelib.Grid((33, 34, 35), (0.01,) * 3, 1e-3, 40, 7)
    assert wavelib.workspace_bytes(bad, wavelib.WAVE_OP_FWD, 0, 0) == 0


@pytest.mark.parametrize("field,value", [("space_order", 3), ("space_order", 18), ("nt", 0),
                                         ("dt", -1.0), ("n", (4, 40, 40))])
def test_invalid_grid_rejected_without_gpu(wavelib, field, value):
    lib = wavelib._lib()
    g = wavelib.Grid((40, 40, 40), (0.01,) * 3, 1e-3, 10, 8)
    setattr(g, field, value)
    cg = g.c()
    dummy = ctypes.c_void_p(256)
    rc = lib.wave_fwd(ctypes.byref(cg), dummy, dummy, None, None, None, None, None, None, 0,
                      None, dummy, 1 << 30, None)
    assert rc == wavelib.WAVE_EINVAL


def test_strerror(wavelib):
    lib = wavelib._lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(lib.wave_strerror(code), bytes)


def test_binding_structs_match_header_layout(wavelib, tmp_path):
    """The ctypes structs of the binding have the header's field names, sizes
    and offsets: a small C program compiled against include/wave.h prints
    them (gcc, host only)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"wave_grid": wavelib._Grid, "wave_points": wavelib._Points,
               "wave_tuning": wavelib._Tuning, "wave_shot": wavelib._Shot}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wave.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, fname)]) == getattr(cls, fname).offset, (cname, fname)
        # and the header declares no field the binding lacks
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname),
                         open(os.path.join(INCLUDE, "wave.h")).read(), flags=re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        declared = re.findall(r"\b([a-z_][a-z0-9_]*)\s*(?:\[\d+\])?\s*;", body)
        assert declared == [f for f, _ in cls._fields_], (cname, declared)


def test_tile_z_and_plan_cache_file_without_gpu(wavelib, tmp_path, monkeypatch):
    """tile_z picks among compiled shapes that differ only in z-width, and the
    plan cache file keeps it (a line without it takes the first such shape);
    plan queries need no GPU."""
    g = wavelib.Grid((200, 180, 512), (0.01,) * 3, 1e-4, 10, 4)
    first = wavelib.describe_plan(g, wavelib.Tuning(time_tile=2, tile_y=12, vec=4))
    wide = wavelib.describe_plan(g, wavelib.Tuning(time_tile=2, tile_y=12, vec=4, tile_z=128, tile_x=77))
    assert (first["tile_z"], wide["tile_z"], wide["tile_x"]) == (56, 128, 77)
    with pytest.raises(wavelib.WaveError):
        wavelib.describe_plan(g, wavelib.Tuning(time_tile=2, tile_y=12, vec=4, tile_z=72))
    cache = tmp_path / "plans.txt"
    # nx ny nz so T_requested -> T tile_y vec chunk [tile_z]
    cache.write_text("201 181 513 4 0 2 12 4 96 128\n"
                     "202 182 514 4 0 2 12 4 64\n"
                     "this line is ignored\n")
    monkeypatch.setenv("WAVE_TUNE_CACHE", str(cache))
    a = wavelib.describe_plan(wavelib.Grid((201, 181, 513), (0.01,) * 3, 1e-4, 10, 4),
                              wavelib.Tuning(time_tile=0))
    b = wavelib.describe_plan(wavelib.Grid((202, 182, 514), (0.01,) * 3, 1e-4, 10, 4),
                              wavelib.Tuning(time_tile=0))
    assert (a["time_tile"], a["tile_y"], a["tile_x"], a["tile_z"]) == (2, 12, 96, 128)
    assert (b["time_tile"], b["tile_y"], b["tile_x"], b["tile_z"]) == (2, 12, 64, 56)


def test_plan_bound_closed_forms_without_gpu(wavelib):
    """wave_plan_bound with explicit bandwidths: the larger of the DRAM and LSU
    terms, worked out by hand for two plans of the 512^3 so-8 grid."""
    g = wavelib.Grid((512, 512, 512), (0.01,) * 3, 1e-4, 10, 8)
    N = 512 ** 3
    hbm, lsu = 8000.0, 40000.0  # GB/s
    # staged untiled 64x16 tile, 2 rows of 4 z-points per thread, x-chunk 64:
    # every point once; per thread and plane it moves 2 x 16 B of queue feed,
    # 2 rows x 2 z-halos of 4 floats, 8 y-neighbour rows of 16 B, 3 x 2 x 16 B
    # of n-1, B, C and 2 x 16 B of output: 352 B for 8 points
    t1 = wavelib.Tuning(time_tile=1, tile_y=16, tile_z=64, kernel=2, rows=2, tile_x=64)
    dram = 20.0 * N / (hbm * 1e9) * 1e3
    lsu_ms = N * 44.0 / (lsu * 1e9) * 1e3
    assert wavelib.plan_bound(g, t1, hbm, lsu, -1) == pytest.approx(max(dram, lsu_ms), rel=1e-12)
    assert dram > lsu_ms  # DRAM binds the untiled sweep
    # staged depth 2, 64x24 tile, x-chunk 103: stage 1 covers 72 x 32 over each
    # chunk's planes plus 4 on either side (552 planes), stage 2 the tile over
    # 512 planes; 8 x 22 tiles (the last row of tiles overhangs 512); stage 2
    # stores two levels (64 B per thread and plane instead of 32)
    t2 = wavelib.Tuning(time_tile=2, tile_y=24, tile_z=64, kernel=2, rows=2, tile_x=103)
    lsu_b = 8 * 22 * (552 * 32 * 72 * 44.0 + 512 * 24 * 64 * 48.0)
    want = max(24.0 * N / (hbm * 1e9), lsu_b / (lsu * 1e9)) * 1e3 / 2
    assert wavelib.plan_bound(g, t2, hbm, lsu, -1) == pytest.approx(want, rel=1e-12)
    # fields inside L2 drop the DRAM term; a wider recomputed halo raises the bound
    small = wavelib.Grid((64, 64, 64), (0.01,) * 3, 1e-4, 10, 8)
    t1s = wavelib.Tuning(time_tile=1, tile_y=16, tile_z=64, kernel=2, rows=2, tile_x=64)
    assert wavelib.plan_bound(small, t1s, hbm, lsu, 128e6) == pytest.approx(
        64 ** 3 * 44.0 / (lsu * 1e9) * 1e3, rel=1e-12)
    g16 = wavelib.Grid((512, 512, 512), (0.01,) * 3, 1e-4, 10, 16)
    deep = wavelib.plan_bound(g16, wavelib.Tuning(time_tile=2, tile_y=8, tile_z=32, kernel=2, rows=2,
                                                  tile_x=64), hbm, lsu, -1)
    flat = wavelib.plan_bound(g16, wavelib.Tuning(time_tile=1, tile_y=24, tile_z=64, kernel=2, rows=2,
                                                  tile_x=64), hbm, lsu, -1)
    assert deep > flat


def test_batch_plan_of_named_tunings_without_gpu(wavelib):
    """Which kernel a batched call's groups run, for tunings that name it (no
    timing needed): the batched stage-specialised shape of the named depth
    when it divides nt and the checkpoint interval, the shared-warp batched
    kernel for the default untiled shape, shot by shot otherwise."""
    g = wavelib.Grid((48, 40, 44), (0.01,) * 3, 1e-3, 24, 4)
    shots = [wavelib.Shot(origin=(0, 0, 0), n=(30, 30, 30), src_xyz=[[0.1, 0.1, 0.1]],
                          rec_xyz=[[0.2, 0.2, 0.2]]),
             wavelib.Shot(origin=(10, 5, 8), n=(32, 30, 34), src_xyz=[[0.1, 0.1, 0.1]],
                          rec_xyz=[[0.2, 0.1, 0.2]])]
    staged = wavelib.WAVE_KERNEL_STAGED
    p = wavelib.describe_batch_plan(g, shots, 0, 2, wavelib.Tuning(time_tile=2, kernel=staged))
    assert p["lockstep"] and (p["time_tile"], p["kernel"]) == (2, staged)
    p = wavelib.describe_batch_plan(g, shots, 6, 2, wavelib.Tuning(time_tile=2, kernel=staged))
    assert (p["time_tile"], p["kernel"]) == (2, staged)
    # depth 2 does not divide a checkpoint interval of 5: shot by shot
    assert wavelib.describe_batch_plan(g, shots, 5, 2, wavelib.Tuning(time_tile=2, kernel=staged)) is None
    p = wavelib.describe_batch_plan(g, shots, 0, 2, wavelib.Tuning(time_tile=1))
    assert (p["time_tile"], p["kernel"]) == (1, wavelib.WAVE_KERNEL_SHARED)
    # a shared-warp depth-2 tile has no batched kernel
    assert wavelib.describe_batch_plan(g, shots, 0, 2, wavelib.Tuning(time_tile=2)) is None
    odd = wavelib.Grid((48, 40, 44), (0.01,) * 3, 1e-3, 23, 4)
    assert wavelib.describe_batch_plan(odd, shots, 0, 2, wavelib.Tuning(time_tile=2, kernel=staged)) is None


def test_grad_plan_query_before_any_gradient_call(wavelib):
    # host-side query: no gradient call with these arguments has run in this
    # process, so there is no timed choice to report; bad arguments are refused
    g = wavelib.Grid((40, 36, 44), (0.01,) * 3, 1e-3, 30, 8)
    with pytest.raises(wavelib.WaveError) as e:
        wavelib.describe_grad_plan(g, 1, 3, 10, tuning=wavelib.Tuning(time_tile=1))
    assert e.value.code == wavelib.WAVE_EUNSUPPORTED
    with pytest.raises(wavelib.WaveError) as e:
        wavelib.describe_grad_plan(g, 1, 3, 0)
    assert e.value.code == wavelib.WAVE_EINVAL
