"""Helpers shared by the GPU parity tests (oracle side and CUDA side are
built from the same seeded workload; nothing here computes the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import system as S_  # noqa: E402


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_system(wl, **kw):
    return S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()), **kw)


def gpu_context(wl):
    from paper_1010_2832_gb300 import stokes
    return stokes.context_for(wl)


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def gpu_apply_fields(ctx, x_fields, precision):
    """A x through the C ABI for an unknown vector in field (oracle) order."""
    from paper_1010_2832_gb300 import stokes
    xs = ctx.fields_to_slots(to_gpu(x_fields))
    if precision == stokes.FP64:
        ys = ctx.new_vector()
        ctx.apply(xs, ys, precision)
    else:
        x32 = xs.to(torch.float32)
        y32 = ctx.new_vector(torch.float32)
        ctx.apply(x32, y32, precision)
        ys = y32.to(torch.float64)
    return ctx.slots_to_fields(ys).cpu().numpy()


def face_flags(S):
    """Oracle face status in the library's flag bits."""
    from oracle import operators as O
    wall = O.boundary_face_mask(tuple(S.inp.n))
    return (S.live * 1 + S.bad * 2 + S.invalid_face * 4 + wall * 8).astype(np.uint8)


def abs_matvec(A, x):
    """|A| |x|: the scale against which a rounded A x is compared."""
    Aa = abs(A)
    return Aa @ np.abs(x)


def golden_velocity_samples(name):
    """(face indices, oracle velocities, scale) stored by
    tests/golden/make_oracle_velocity_samples.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"oracle_velocity_{name}.txt")
    idx, val, scale = [], [], None
    for line in open(path):
        if line.startswith("# scale"):
            scale = float(line.split(":")[1])
        elif line.strip() and not line.startswith("#"):
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    return np.array(idx), np.array(val), scale
