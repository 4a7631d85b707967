"""Thin Python binding of libstokes (include/stokes.h) over ctypes.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are torch CUDA tensors (float64 unless stated), whose
data pointers are handed to the C entry points; the context's stream is the
torch stream current at creation.  There is no CPU fallback: importing
without the built library raises.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstokes.so")

FP64, FP32, BF16 = 0, 1, 2
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NOT_CONVERGED", -4: "ERR_BREAKDOWN",
          -5: "ERR_TIMEOUT", -7: "ERR_NONFINITE", -8: "ERR_STATE"}


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double), ("dt", C.c_double), ("origin", C.c_double * 3)]


class Layout(C.Structure):
    _fields_ = [("nfields", C.c_int), ("field_stride", C.c_int64), ("base", C.c_int64),
                ("pitch", C.c_int), ("rows", C.c_int), ("planes", C.c_int), ("total", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("mode", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("inner_tol", C.c_double),
                ("max_outer", C.c_int), ("check_every", C.c_int), ("precond", C.c_int), ("use_graph", C.c_int),
                ("wait_test", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("outer", C.c_int), ("rel_residual", C.c_double),
                ("ms_rhs", C.c_double), ("ms_solve", C.c_double), ("ms_recover", C.c_double),
                ("precision_used", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = ("stokes_create", "stokes_destroy", "stokes_last_error", "stokes_build_weights", "stokes_vector_layout",
            "stokes_apply", "stokes_rhs", "stokes_recover", "stokes_default_options", "stokes_solve_step",
            "stokes_solve_system", "stokes_export", "stokes_export_size", "stokes_slots_to_fields",
            "stokes_fields_to_slots", "stokes_last_apply_ms", "stokes_bench_cg_kernels", "stokes_active_tiles",
            "stokes_batch_create", "stokes_batch_solve", "stokes_batch_destroy", "stokes_batch_tuning",
            "stokes_solve_batched", "stokes_net_create", "stokes_net_destroy", "stokes_net_param_count",
            "stokes_net_layer", "stokes_net_set_params", "stokes_net_get_params", "stokes_net_forward",
            "stokes_net_gradient", "stokes_net_train_step", "stokes_set_learned_preconditioner",
            "stokes_learned_grid", "stokes_learned_features", "stokes_learned_targets",
            "stokes_learned_jacobi_steps", "stokes_apply_preconditioner", "stokes_schwarz_setup_ms",
            "stokes_apply_schwarz_noalloc", "stokes_bench_schwarz_kernels", "stokes_traction_u_star",
            "stokes_advect", "stokes_set_min_face_liquid")


class BatchIO(C.Structure):
    _fields_ = [("u_star", C.c_void_p * 3), ("u_out", C.c_void_p * 3), ("tau_out", C.c_void_p * 5),
                ("p_out", C.c_void_p)]

_lib = None


def load_library(path=LIB_PATH):
    """Load libstokes.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libstokes.so not found at {path}: run paper_1010_2832_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    PP = C.POINTER(C.c_void_p)
    sig = {
        "stokes_create": (I, [C.POINTER(P), C.POINTER(Grid), P]),
        "stokes_destroy": (I, [P]),
        "stokes_last_error": (C.c_char_p, [P]),
        "stokes_build_weights": (I, [P, P, P, PP, PP, PP]),
        "stokes_vector_layout": (I, [P, C.POINTER(Layout)]),
        "stokes_apply": (I, [P, P, P, I]),
        "stokes_rhs": (I, [P, PP, P]),
        "stokes_recover": (I, [P, PP, P, PP]),
        "stokes_default_options": (None, [C.POINTER(Options)]),
        "stokes_solve_step": (I, [P, PP, PP, PP, P, C.POINTER(Options), C.POINTER(Stats)]),
        "stokes_solve_system": (I, [P, P, P, C.POINTER(Options), C.POINTER(Stats)]),
        "stokes_export": (I, [P, I, P]),
        "stokes_export_size": (I64, [P, I]),
        "stokes_slots_to_fields": (I, [P, P, P]),
        "stokes_fields_to_slots": (I, [P, P, P]),
        "stokes_last_apply_ms": (D, [P]),
        "stokes_bench_cg_kernels": (I, [P, I, I, C.POINTER(D), C.POINTER(D)]),
        "stokes_active_tiles": (I, [P]),
        "stokes_batch_create": (I, [C.POINTER(P), I, C.POINTER(P), C.POINTER(Options), C.c_char_p]),
        "stokes_batch_solve": (I, [P, C.POINTER(BatchIO), C.POINTER(Stats), C.POINTER(D)]),
        "stokes_batch_destroy": (I, [P]),
        "stokes_batch_tuning": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(D), C.POINTER(I)]),
        "stokes_solve_batched": (I, [I, C.POINTER(P), C.POINTER(BatchIO), C.POINTER(Options), C.POINTER(Stats)]),
        "stokes_net_create": (I, [C.POINTER(P), I, I, I, I64]),
        "stokes_net_destroy": (I, [P]),
        "stokes_net_param_count": (I64, [P]),
        "stokes_net_layer": (I, [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I64), C.POINTER(I64)]),
        "stokes_net_set_params": (I, [P, P]),
        "stokes_net_get_params": (I, [P, P]),
        "stokes_net_forward": (I, [P, I, I, I, I, P, P]),
        "stokes_net_gradient": (I, [P, I, I, I, I, P, P, C.POINTER(D), P]),
        "stokes_net_train_step": (I, [P, I, I, I, I, P, P, C.c_float, C.POINTER(D)]),
        "stokes_set_learned_preconditioner": (I, [P, P]),
        "stokes_learned_grid": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
        "stokes_learned_features": (I, [P, P, P, C.POINTER(D)]),
        "stokes_learned_targets": (I, [P, P, D, P]),
        "stokes_learned_jacobi_steps": (C.c_long, [P]),
        "stokes_apply_preconditioner": (I, [P, I, P, P]),
        "stokes_schwarz_setup_ms": (D, [P]),
        "stokes_apply_schwarz_noalloc": (I, [P, P, P]),
        "stokes_bench_schwarz_kernels": (I, [P, I, C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
        "stokes_traction_u_star": (I, [P, PP, P, PP, PP]),
        "stokes_advect": (I, [P, PP, P, C.POINTER(D), I, P, P, PP, P]),
        "stokes_set_min_face_liquid": (I, [P, D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptrs(tensors):
    arr = (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
    return C.cast(arr, C.POINTER(C.c_void_p)), arr


def _dev(t, dtype=torch.float64):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor of dtype %s" % dtype)
    return t


class StokesError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_options(**kw):
    lib = load_library()
    o = Options()
    lib.stokes_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class StokesContext:
    """One grid on the current CUDA device (see include/stokes.h)."""

    def __init__(self, dim, n, h, dt, origin=(0.0, 0.0, 0.0), stream=None):
        self.lib = load_library()
        g = Grid()
        g.dim = dim
        g.nx, g.ny = n[0], n[1]
        g.nz = n[2] if dim == 3 else 0
        g.h, g.dt = h, dt
        for d in range(3):
            g.origin[d] = origin[d] if d < len(origin) else 0.0
        self.dim, self.n = dim, tuple(n)
        # None: the library makes its own stream, ordered with torch's
        # (legacy) default stream; a torch.cuda.Stream is used as given
        self.stream = stream
        h_ = C.c_void_p()
        sp = None if stream is None else C.c_void_p(stream.cuda_stream)
        st = self.lib.stokes_create(C.byref(h_), C.byref(g), sp)
        if st != 0:
            raise StokesError(st, self.lib.stokes_last_error(None).decode())
        self.h = h_
        lay = Layout()
        self.lib.stokes_vector_layout(self.h, C.byref(lay))
        self.layout = lay
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.stokes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise StokesError(st, self.lib.stokes_last_error(self.h).decode())
        return st

    # ---- weights ---------------------------------------------------------
    def build_weights(self, phi_liquid, phi_solid, rho, mu, u_bc):
        rp, ra = _ptrs([_dev(t) for t in rho])
        mp, ma = _ptrs([_dev(t) for t in mu])
        up, ua = _ptrs([_dev(t) for t in u_bc])
        self._check(self.lib.stokes_build_weights(self.h, _dev(phi_liquid).data_ptr(), _dev(phi_solid).data_ptr(),
                                                  rp, mp, up))

    # ---- vectors -----------------------------------------------------------
    def set_min_face_liquid(self, eps):
        """Floor of the live faces' mass fraction from the next weight build
        (stokes_set_min_face_liquid); 0 is the paper's system."""
        self._check(self.lib.stokes_set_min_face_liquid(self.h, float(eps)))

    def new_vector(self, dtype=torch.float64):
        return torch.zeros(self.layout.total, dtype=dtype, device="cuda")

    def apply(self, x, y, precision=FP64):
        dt = torch.float64 if precision == FP64 else torch.float32
        self._check(self.lib.stokes_apply(self.h, _dev(x, dt).data_ptr(), _dev(y, dt).data_ptr(), precision))

    def last_apply_ms(self):
        return self.lib.stokes_last_apply_ms(self.h)

    def rhs(self, u_star, b):
        up, ua = _ptrs([_dev(t) for t in u_star])
        self._check(self.lib.stokes_rhs(self.h, up, _dev(b).data_ptr()))

    def recover(self, u_star, x, u_out):
        up, ua = _ptrs([_dev(t) for t in u_star])
        op, oa = _ptrs([_dev(t) for t in u_out])
        self._check(self.lib.stokes_recover(self.h, up, _dev(x).data_ptr(), op))

    def solve_system(self, b, x, options=None):
        o = options or default_options()
        st = Stats()
        rc = self.lib.stokes_solve_system(self.h, _dev(b).data_ptr(), _dev(x).data_ptr(), C.byref(o), C.byref(st))
        if rc not in (0, -3):
            self._check(rc)
        return st

    def traction_u_star(self, tau_bc, p_bc, u_star, u_star_out):
        """u* carrying a prescribed surface pressure / deviatoric stress
        (stokes_traction_u_star); lists of FP64 device tensors."""
        tp, ta = _ptrs([_dev(t) for t in tau_bc])
        up, ua = _ptrs([_dev(t) for t in u_star])
        op, oa = _ptrs([_dev(t) for t in u_star_out])
        self._check(self.lib.stokes_traction_u_star(self.h, tp, _dev(p_bc).data_ptr(), up, op))

    def advect(self, u_in, u_out, gravity, ext_passes=0, phi_in=None, phi_out=None, valid=None, phi_union=None):
        """Transport stage around the Stokes step (stokes_advect): u_out <- u*,
        phi_out <- advected level set; FP64 device tensors, valid a uint8
        device tensor (u then v faces) or None for the context's weights."""
        up, ua = _ptrs([_dev(t) for t in u_in])
        op, oa = _ptrs([_dev(t) for t in u_out])
        g = (C.c_double * 2)(*[float(x) for x in gravity])
        ptr = lambda t: None if t is None else t.data_ptr()
        if valid is not None and (valid.dtype != torch.uint8 or not valid.is_cuda):
            raise TypeError("valid must be a uint8 device tensor")
        self._check(self.lib.stokes_advect(self.h, up, ptr(None if phi_in is None else _dev(phi_in)),
                                           g, int(ext_passes), ptr(valid),
                                           ptr(None if phi_union is None else _dev(phi_union)), op,
                                           ptr(None if phi_out is None else _dev(phi_out))))

    def solve_step(self, u_star, u_out, tau_out, p_out, options=None):
        o = options or default_options()
        st = Stats()
        up, ua = _ptrs([_dev(t) for t in u_star])
        op, oa = _ptrs([_dev(t) for t in u_out])
        tp, ta = _ptrs([_dev(t) for t in tau_out])
        rc = self.lib.stokes_solve_step(self.h, up, op, tp, _dev(p_out).data_ptr(), C.byref(o), C.byref(st))
        if rc not in (0, -3):
            self._check(rc)
        return st

    def export(self, what):
        n = self.lib.stokes_export_size(self.h, what)
        buf = torch.zeros(n, dtype=torch.uint8, device="cuda")
        self._check(self.lib.stokes_export(self.h, what, buf.data_ptr()))
        return buf.view(torch.float64) if what in (0, 1) else buf

    def slots_to_fields(self, slots):
        n = self.field_vector_length()
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        self._check(self.lib.stokes_slots_to_fields(self.h, _dev(slots).data_ptr(), out.data_ptr()))
        return out

    def fields_to_slots(self, fields):
        out = self.new_vector()
        self._check(self.lib.stokes_fields_to_slots(self.h, _dev(fields).data_ptr(), out.data_ptr()))
        return out

    def bench_cg_kernels(self, precision=FP32, launches=50):
        """Mean device ms of the CG-mode apply and of the update kernel."""
        a, u = C.c_double(), C.c_double()
        self._check(self.lib.stokes_bench_cg_kernels(self.h, precision, launches, C.byref(a), C.byref(u)))
        return a.value, u.value

    def bench_schwarz_kernels(self, launches=50):
        """Mean device ms of the Schwarz local solves and of the gather, and the
        local solves' algorithmic bytes per launch."""
        a, g, b = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.stokes_bench_schwarz_kernels(self.h, launches, C.byref(a), C.byref(g), C.byref(b)))
        return a.value, g.value, b.value

    def active_tiles(self):
        return self.lib.stokes_active_tiles(self.h)

    def apply_preconditioner(self, which, r32, z32):
        self._check(self.lib.stokes_apply_preconditioner(self.h, which, _dev(r32, torch.float32).data_ptr(),
                                                         _dev(z32, torch.float32).data_ptr()))

    def apply_schwarz_noalloc(self, r32, z32):
        """Allocation-free Schwarz apply (same result as apply_preconditioner(2));
        the plan must exist.  For callers that cannot allocate device memory."""
        self._check(self.lib.stokes_apply_schwarz_noalloc(self.h, _dev(r32, torch.float32).data_ptr(),
                                                          _dev(z32, torch.float32).data_ptr()))

    def schwarz_setup_ms(self):
        return self.lib.stokes_schwarz_setup_ms(self.h)

    def field_vector_length(self):
        nx, ny = self.n[0], self.n[1]
        if self.dim == 2:
            return 2 * nx * ny + (nx + 1) * (ny + 1)
        nz = self.n[2]
        return (3 * nx * ny * nz + nz * (ny + 1) * (nx + 1) + (nz + 1) * ny * (nx + 1)
                + (nz + 1) * (ny + 1) * nx)


class Batch:
    """Many 2D contexts solved together in one persistent launch (see
    stokes_batch_create in include/stokes.h)."""

    def __init__(self, contexts, options=None, tune_cache=None):
        self.lib = load_library()
        self.contexts = list(contexts)
        n = len(self.contexts)
        arr = (C.c_void_p * n)(*[c.h.value for c in self.contexts])
        self.opt = options or default_options()
        h = C.c_void_p()
        st = self.lib.stokes_batch_create(C.byref(h), n, arr, C.byref(self.opt),
                                          tune_cache.encode() if tune_cache else None)
        if st != 0:
            raise StokesError(st, "stokes_batch_create failed")
        self.h = h

    def tuning(self):
        ty, cps, us, g = C.c_int(), C.c_int(), C.c_double(), C.c_int()
        self.lib.stokes_batch_tuning(self.h, C.byref(ty), C.byref(cps), C.byref(us), C.byref(g))
        return dict(tile_rows=ty.value, ctas_per_sm=cps.value, us_per_iter=us.value, graph=bool(g.value))

    def solve(self, u_star, u_out, tau_out, p_out):
        """Lists (one entry per instance) of tensors in field layout."""
        n = len(self.contexts)
        io = (BatchIO * n)()
        for i in range(n):
            for d in range(2):
                io[i].u_star[d] = _dev(u_star[i][d]).data_ptr()
                io[i].u_out[d] = _dev(u_out[i][d]).data_ptr()
                io[i].tau_out[d] = _dev(tau_out[i][d]).data_ptr()
            io[i].p_out = _dev(p_out[i]).data_ptr()
        stats = (Stats * n)()
        ms = C.c_double()
        rc = self.lib.stokes_batch_solve(self.h, io, stats, C.byref(ms))
        if rc not in (0, -3):
            raise StokesError(rc, "stokes_batch_solve failed")
        return [s.as_dict() for s in stats], ms.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.stokes_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The learned preconditioner's network (stokes_net_* in include/stokes.h)."""

    def __init__(self, dim, cin, cout, max_voxels):
        import numpy as np  # noqa: F401
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.stokes_net_create(C.byref(h), dim, cin, cout, int(max_voxels))
        if st != 0:
            raise StokesError(st, "stokes_net_create failed")
        self.h, self.dim, self.cin, self.cout = h, dim, cin, cout
        self.n = self.lib.stokes_net_param_count(self.h)

    def layers(self):
        out = []
        for i in range(11):
            ci, co, ks, wo, bo = C.c_int(), C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
            self.lib.stokes_net_layer(self.h, i, C.byref(ci), C.byref(co), C.byref(ks), C.byref(wo), C.byref(bo))
            out.append((ci.value, co.value, ks.value, wo.value, bo.value))
        return out

    def set_params(self, theta32):
        import numpy as np
        a = np.ascontiguousarray(theta32, dtype=np.float32)
        assert a.size == self.n
        self.lib.stokes_net_set_params(self.h, a.ctypes.data)

    def get_params(self):
        import numpy as np
        a = np.zeros(self.n, dtype=np.float32)
        self.lib.stokes_net_get_params(self.h, a.ctypes.data)
        return a

    def from_oracle_layout(self, theta):
        """Oracle order (per conv: W[cout][cin][k..], b) -> this library's
        layout (per conv: W[tap][cin][cout], b, 4-float aligned)."""
        import numpy as np
        out = np.zeros(self.n, dtype=np.float32)
        o = 0
        for ci, co, ks, wo, bo in self.layers():
            kd = (ks,) * self.dim
            nw = co * ci * int(np.prod(kd))
            W = np.asarray(theta[o:o + nw]).reshape((co, ci) + kd)
            o += nw
            perm = tuple(range(2, 2 + self.dim)) + (1, 0)
            out[wo:wo + nw] = W.transpose(perm).reshape(-1)
            out[bo:bo + co] = theta[o:o + co]
            o += co
        return out

    def to_oracle_layout(self, p):
        import numpy as np
        parts = []
        for ci, co, ks, wo, bo in self.layers():
            kd = (ks,) * self.dim
            nw = co * ci * int(np.prod(kd))
            W = np.asarray(p[wo:wo + nw], dtype=np.float64).reshape(kd + (ci, co))
            inv = (self.dim + 1, self.dim) + tuple(range(self.dim))
            parts.append(W.transpose(inv).reshape(-1))
            parts.append(np.asarray(p[bo:bo + co], dtype=np.float64))
        return np.concatenate(parts)

    def forward(self, x, shape):
        B, D, H, W = shape
        y = torch.zeros(B * D * H * W * self.cout, dtype=torch.float32, device="cuda")
        st = self.lib.stokes_net_forward(self.h, B, D, H, W, _dev(x, torch.float32).data_ptr(), y.data_ptr())
        if st != 0:
            raise StokesError(st, "stokes_net_forward failed")
        return y

    def gradient(self, x, y, shape):
        import numpy as np
        B, D, H, W = shape
        g = np.zeros(self.n, dtype=np.float32)
        loss = C.c_double()
        st = self.lib.stokes_net_gradient(self.h, B, D, H, W, _dev(x, torch.float32).data_ptr(),
                                          _dev(y, torch.float32).data_ptr(), C.byref(loss), g.ctypes.data)
        if st != 0:
            raise StokesError(st, "stokes_net_gradient failed")
        return loss.value, g

    def train_step(self, x, y, shape, lr):
        B, D, H, W = shape
        loss = C.c_double()
        st = self.lib.stokes_net_train_step(self.h, B, D, H, W, _dev(x, torch.float32).data_ptr(),
                                            _dev(y, torch.float32).data_ptr(), C.c_float(lr), C.byref(loss))
        if st != 0:
            raise StokesError(st, "stokes_net_train_step failed")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.stokes_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def learned_grid(ctx):
    v = [C.c_int() for _ in range(5)]
    ctx.lib.stokes_learned_grid(ctx.h, *[C.byref(a) for a in v])
    return tuple(a.value for a in v)   # D, H, W, cin, cout


def attach_network(ctx, net):
    ctx._check(ctx.lib.stokes_set_learned_preconditioner(ctx.h, net.h if net is not None else None))
    ctx._net = net


def learned_jacobi_steps(ctx):
    """Jacobi fallback steps taken by the last learned-preconditioner solve."""
    return int(ctx.lib.stokes_learned_jacobi_steps(ctx.h))


def learned_features(ctx, r):
    D, H, W, cin, cout = learned_grid(ctx)
    x = torch.zeros(D * H * W * cin, dtype=torch.float32, device="cuda")
    rms = C.c_double()
    ctx._check(ctx.lib.stokes_learned_features(ctx.h, _dev(r).data_ptr(), x.data_ptr(), C.byref(rms)))
    return x, rms.value


def learned_targets(ctx, e, rms):
    D, H, W, cin, cout = learned_grid(ctx)
    y = torch.zeros(D * H * W * cout, dtype=torch.float32, device="cuda")
    ctx._check(ctx.lib.stokes_learned_targets(ctx.h, _dev(e).data_ptr(), C.c_double(rms), y.data_ptr()))
    return y


def upload_workload(wl):
    """Copy a ``workloads.Workload`` to CUDA tensors: dict of lists."""
    t = lambda a: torch.from_numpy(a).to("cuda").contiguous()
    return dict(phi_liquid=t(wl.phi_liquid), phi_solid=t(wl.phi_solid), rho=[t(a) for a in wl.rho],
                mu=[t(a) for a in wl.mu], u_bc=[t(a) for a in wl.u_bc], u_star=[t(a) for a in wl.u_star])


def context_for(wl, stream=None, min_face_liquid=0.0):
    """Create a context for a workload and build its weights on the device
    (with the given floor of the live faces' mass fraction)."""
    ctx = StokesContext(wl.dim, wl.n, wl.h, wl.dt, wl.origin, stream=stream)
    if min_face_liquid:
        ctx.set_min_face_liquid(min_face_liquid)
    d = upload_workload(wl)
    ctx.build_weights(d["phi_liquid"], d["phi_solid"], d["rho"], d["mu"], d["u_bc"])
    return ctx, d
