"""Out-of-memory handling on the host side (the library's failure paths, no GPU
fault involved): pic_inject_alloc_failure makes one of the library's device
allocations fail as an exhausted device would, and the call that made it must
return PIC_ERR_OOM and leave the grid usable -- or, at creation, leave nothing
behind."""
import numpy as np
import pytest

from paper_1101_0809_gb300 import workloads as W
from pichelpers import make_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


@pytest.fixture(autouse=True)
def disarm(P):
    yield
    P.pic_inject_alloc_failure(-1)


def test_failed_pool_allocation_keeps_the_previous_particles(P):
    wl = W.c0_small2d(steps=4)
    grid = make_grid(P, wl, P.PIC_FP32)
    before = grid.particles(0)
    sp = wl.species[0]
    x2 = sp.x[:, :100].copy()
    P.pic_inject_alloc_failure(0)        # the first allocation of the load: the new pool
    with pytest.raises(P.PicError) as e:
        grid.load(1, 1.0, 1836.0, sp.weight, x2, np.zeros_like(x2))
    assert e.value.code == P.PIC_ERR_OOM
    after = grid.particles(0)
    for b, a in zip(before, after):
        if isinstance(b, list):
            for u, v in zip(b, a):
                np.testing.assert_array_equal(u, v)
        else:
            np.testing.assert_array_equal(b, a)
    assert P.pic_num_particles(grid.h, 1) == 0
    P.pic_step(grid.h, 3)
    d = P.pic_diagnostics(grid.h)
    assert d["n_particles"] == sp.n and d["error_word"] == 0
    grid.load(1, 1.0, 1836.0, sp.weight, x2, np.zeros_like(x2))    # disarmed: the load now works
    assert P.pic_num_particles(grid.h, 1) == 100
    grid.close()


@pytest.mark.parametrize("after", [3, 15, 17, 22, 60])
def test_failure_after_the_pool_leaves_a_usable_grid(P, after):
    """A failure among the sort and work-list buffers that follow the pool
    leaves the grid with its fields and no particles; it steps, reports, loads
    again and steps on."""
    wl = W.c0_small2d(steps=4)
    grid = make_grid(P, wl, P.PIC_FP32)
    P.pic_step(grid.h, 2)
    sp = wl.species[0]
    P.pic_inject_alloc_failure(after)
    try:
        grid.load(0, sp.q, sp.m, sp.weight, sp.x[:, :4000], sp.w[:, :4000])
        failed = False
    except P.PicError as e:
        assert e.code == P.PIC_ERR_OOM
        failed = True
    P.pic_inject_alloc_failure(-1)
    n0 = P.pic_num_particles(grid.h, 0)
    assert n0 in (0, 4000, sp.n)
    if failed:
        assert n0 in (0, sp.n)
    P.pic_step(grid.h, 12)               # crosses a sort interval
    d = P.pic_diagnostics(grid.h)
    assert d["n_particles"] == n0 and d["error_word"] == 0
    grid.load(0, sp.q, sp.m, sp.weight, sp.x, sp.w)
    P.pic_step(grid.h, 2)
    assert P.pic_diagnostics(grid.h)["n_particles"] == sp.n
    grid.close()


def test_failure_at_creation_returns_oom_and_leaves_nothing(P):
    wl = W.c0_small2d()
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=wl.tile, rho_bg=wl.rho_bg)
    for after in (0, 1, 3, 5):          # E, B, J and the run tables come first
        P.pic_inject_alloc_failure(after)
        with pytest.raises(P.PicError) as e:
            P.Grid(desc)
        assert e.value.code == P.PIC_ERR_OOM
    P.pic_inject_alloc_failure(-1)
    grid = make_grid(P, wl, P.PIC_FP32)
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    grid.close()
