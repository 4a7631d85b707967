"""The allocation-free Schwarz apply (stokes_apply_schwarz_noalloc) against
the existing entry point (stokes_apply_preconditioner, which = 2).

Some callers cannot allocate device memory while they run: a process whose
device memory is reserved up front by its own pool, or a real-time loop that
cannot take the device-wide synchronisation of cudaMalloc/cudaFree.  The
allocation-free entry point runs the same kernels in the same order with
their scratch in a fixed 8 MiB device array inside the library, so each of
two calls in a row must give the existing entry point's result bit for bit.
The largest grid that fits the array is accepted and the next one refused
with STOKES_ERR_ARG; a context without a Schwarz plan is refused with
STOKES_ERR_STATE.  Collected last so that it also runs after every other GPU
test in the same process."""
import numpy as np
import pytest

from gpu_common import gpu_context, require_gpu
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCRATCH_BYTES = 8 << 20     # the library's fixed array
PMAX = 108                  # unknowns per patch at most (4x4-slot core + ring, 3 kinds)


def _r256(b):
    return (b + 255) // 256 * 256


def scratch_bytes(n, ntiles):
    """Bytes of the fixed array an n x n grid needs: two CG scalar records,
    the reduction counter, the block partials (two doubles per active tile
    plus 32 spare) and one local result vector per grid patch (4 x 4 slots)."""
    npx = (n + 1 + 3) // 4
    return 256 + 256 + _r256(16 * (ntiles + 32)) + _r256(4 * npx * npx * PMAX)


def max_tiles(n):
    return -(-(n + 1) // 32) * -(-(n + 1) // 8)


# the largest n whose need fits even with every tile active, and the first n
# that does not fit even with none
N_FITS = max(n for n in range(400, 700) if scratch_bytes(n, max_tiles(n)) <= SCRATCH_BYTES)
N_REFUSED = min(n for n in range(400, 700) if scratch_bytes(n, 0) > SCRATCH_BYTES)


def _random_slots(ctx, seed):
    n = ctx.field_vector_length()
    r = np.random.default_rng(seed).normal(size=n)
    return ctx.fields_to_slots(torch.from_numpy(r).cuda()).to(torch.float32)


def test_size_limit_is_where_the_patch_count_steps():
    assert N_REFUSED == N_FITS + 1


@pytest.mark.parametrize("n", [40, 96, N_FITS])
def test_noalloc_apply_matches_existing_entry_point_twice(n):
    require_gpu()
    wl = W.bumps_2d(n, seed=31 + n)
    ctx, dev = gpu_context(wl)
    assert scratch_bytes(n, ctx.active_tiles()) <= SCRATCH_BYTES
    r = _random_slots(ctx, 5)
    z_ref = ctx.new_vector(torch.float32)
    ctx.apply_preconditioner(2, r, z_ref)          # builds the plan
    assert float(z_ref.abs().max()) > 0
    for _ in range(2):
        z = ctx.new_vector(torch.float32).fill_(float("nan"))
        ctx.apply_schwarz_noalloc(r, z)
        torch.cuda.synchronize()
        assert torch.equal(z, z_ref)


def test_noalloc_refuses_the_first_grid_beyond_its_scratch():
    require_gpu()
    wl = W.bumps_2d(N_REFUSED, seed=3)
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
