"""The allocation-free Schwarz apply (stokes_apply_schwarz_noalloc) against
the existing entry point (stokes_apply_preconditioner, which = 2): the same
kernels with their scratch in a fixed device array, so two calls in a row
must each give the existing entry point's result.  Grids beyond the fixed
scratch are refused with STOKES_ERR_ARG, and a context without a Schwarz plan
with STOKES_ERR_STATE.  Collected last so that it also runs after every other
GPU test in the same process."""
import numpy as np
import pytest

from gpu_common import gpu_context, require_gpu
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _random_slots(ctx, seed):
    n = ctx.field_vector_length()
    r = np.random.default_rng(seed).normal(size=n)
    return ctx.fields_to_slots(torch.from_numpy(r).cuda()).to(torch.float32)


@pytest.mark.parametrize("n", [40, 96, 512])
def test_noalloc_apply_matches_existing_entry_point_twice(n):
    require_gpu()
    wl = W.bumps_2d(n, seed=31 + n)
    ctx, dev = gpu_context(wl)
    r = _random_slots(ctx, 5)
    z_ref = ctx.new_vector(torch.float32)
    ctx.apply_preconditioner(2, r, z_ref)          # builds the plan
    scale = float(z_ref.abs().max())
    for _ in range(2):
        z = ctx.new_vector(torch.float32)
        ctx.apply_schwarz_noalloc(r, z)
        torch.cuda.synchronize()
        assert float((z - z_ref).abs().max()) <= 1e-6 * scale


def test_noalloc_refuses_grids_beyond_its_scratch():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.bumps_2d(640, seed=3)
    ctx, dev = gpu_context(wl)
    r = _random_slots(ctx, 6)
    z = ctx.new_vector(torch.float32)
    ctx.apply_preconditioner(2, r, z)
    rc = ctx.lib.stokes_apply_schwarz_noalloc(ctx.h, r.data_ptr(), z.data_ptr())
    assert rc == -1                                    # STOKES_ERR_ARG
    assert b"fixed maximum" in ctx.lib.stokes_last_error(ctx.h)


def test_noalloc_needs_a_plan():
    require_gpu()
    wl = W.bumps_2d(32, seed=4)
    ctx, dev = gpu_context(wl)
    r = _random_slots(ctx, 7)
    z = ctx.new_vector(torch.float32)
    rc = ctx.lib.stokes_apply_schwarz_noalloc(ctx.h, r.data_ptr(), z.data_ptr())
    assert rc == -8                                    # STOKES_ERR_STATE
