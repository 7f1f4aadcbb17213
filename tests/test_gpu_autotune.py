"""Launch-shape autotuning: the thermal kernel choices give the same results
bit for bit, and so do EM runs of one tile height (tiles share no reduction;
the halo is recomputed identically); tile heights that send a node through
the two-node path in one case and the one-node path in the other agree to
FP32 rounding (the code generator contracts some packed multiply-adds into
FMAs that the one-node path rounds in two steps). Timing leaves the context's
state untouched, and a second context of the same grid shape takes the
cached choice."""
import numpy as np
import pytest

import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, hetero_problem, random_fields, rel_l2, seed_both

pytestmark = pytest.mark.gpu

FIELDS = [api.COSIM_F_EX, api.COSIM_F_EY, api.COSIM_F_EZ, api.COSIM_F_HX, api.COSIM_F_HY, api.COSIM_F_HZ]


def _run(p, shape, steps=40, thermal=6):
    ctx = context(p, FP32)
    ctx.autotune(fixed=shape)
    assert (ctx.query(api.COSIM_Q_EM_TILE_Y), ctx.query(api.COSIM_Q_TH_BLOCK_Y)) == shape
    if p.sources:
        ctx.set_sources(p.source_tables(ctx.dt, steps))
    else:
        E, H = random_fields(p, seed=3)
        for a in range(3):
            ctx.write(api.COSIM_F_EX + a, E[a])
            ctx.write(api.COSIM_F_HX + a, H[a])
    ctx.em_steps(steps)
    ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
    ctx.thermal_steps(thermal)
    out = [ctx.read(f, np.float32) for f in FIELDS + [api.COSIM_F_Q, api.COSIM_F_T]]
    ctx.close()
    return out


@pytest.mark.parametrize("which", ["tiny", "hetero", "wide"])
def test_launch_shapes_agree(which):
    """("wide": interior tile pairs exist, and the 8- and 4-row tilings put
    different nodes in pair tiles and in border tiles)"""
    if which == "tiny":
        p = W.tiny_package()
    elif which == "hetero":
        p = hetero_problem(45, 37, 9, seed=61, em_bc=(2, 2, 2, 1, 0, 2), cpml=4)
    else:
        p = hetero_problem(140, 33, 7, seed=63, em_bc=(2, 2, 2, 1, 0, 2), cpml=4)
    runs = {shape: _run(p, shape) for shape in [(8, 0), (8, 4), (8, 8), (8, 16), (4, 0), (4, 4), (4, 8), (4, 16)]}
    for ty in (8, 4):
        ref = runs[(ty, 0)]
        for by in (4, 8, 16):
            for f, (a, b) in enumerate(zip(ref, runs[(ty, by)])):
                assert np.array_equal(a, b), ((ty, by), f)
    for f, (a, b) in enumerate(zip(runs[(8, 0)], runs[(4, 0)])):
        if which == "wide":
            assert rel_l2(b, a) < 1e-5, f
        else:  # no node reaches the two-node path: identical
            assert np.array_equal(a, b), f


def test_autotune_leaves_state_and_caches_the_choice():
    p = hetero_problem(61, 29, 11, seed=62, em_bc=(2, 2, 2, 2, 0, 2), cpml=4)
    ctx = context(p, FP32)
    E, H = random_fields(p, seed=4)
    for a in range(3):
        ctx.write(api.COSIM_F_EX + a, E[a])
        ctx.write(api.COSIM_F_HX + a, H[a])
    ctx.em_steps(5)
    before = [ctx.read(f) for f in FIELDS + [api.COSIM_F_T, api.COSIM_F_Q]]
    ty, by = ctx.autotune(force=True)
    assert ty in (4, 8) and by in (0, 4, 8, 16)
    after = [ctx.read(f) for f in FIELDS + [api.COSIM_F_T, api.COSIM_F_Q]]
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    assert ctx.query(api.COSIM_Q_STEP) == 5
    other = context(p, FP32)
    assert other.autotune() == (ty, by)  # cached for the shape
    other.close()
    ctx.em_steps(5)  # steps continue with the tuned shape
    ctx.close()
    c64 = context(p, FP64)
    ty64, _ = c64.autotune(force=True)
    assert ty64 == 8  # FP64 keeps the 8-row tile
    c64.close()
