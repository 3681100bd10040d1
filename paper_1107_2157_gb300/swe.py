"""ctypes binding of the C ABI in include/swe.h (argument marshalling only).

Every ``swe_*`` function here calls the function of the same name in
libswe.so; no step of the method runs in Python.  ``Grid`` is a small
convenience wrapper that owns a context handle and marshals numpy arrays
(host) or torch tensors (host or device) into pointer/stride arguments.

Loading fails loudly if libswe.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswe.so")

SWE_OK, SWE_EINVAL, SWE_ENOMEM, SWE_ECUDA, SWE_ETIMEOUT, SWE_ECHECK, SWE_EUNSUPPORTED = range(7)
SWE_F32, SWE_F64 = 0, 1
SWE_KERNEL_AUTO, SWE_KERNEL_NAIVE, SWE_KERNEL_TILED, SWE_KERNEL_TEMPORAL = range(4)
SWE_FLAG_NONPOSITIVE, SWE_FLAG_MASS, SWE_FLAG_TIMEOUT, SWE_FLAG_FALLBACK = 1, 2, 4, 8
(SWE_BQ_VARIANT, SWE_BQ_CTAS_PER_SM, SWE_BQ_BLOCKS, SWE_BQ_TILES, SWE_BQ_TILE_X, SWE_BQ_TILE_Y,
 SWE_BQ_STAGES, SWE_BQ_DEPTH, SWE_BQ_GRAPH, SWE_BQ_LAUNCHES, SWE_BQ_TUNED, SWE_BQ_CELLS,
 SWE_BQ_VARIANT_COUNT, SWE_BQ_KIND) = range(14)
(SWE_Q_KERNEL, SWE_Q_DEPTH, SWE_Q_PITCH, SWE_Q_LAUNCHES, SWE_Q_TILE_X, SWE_Q_TILE_Y,
 SWE_Q_STATE_PTR, SWE_Q_STEPS_PER_LAUNCH, SWE_Q_SHAPE) = range(9)
SWE_PQ_PARTS, SWE_PQ_HALO_CELLS, SWE_PQ_LAUNCHES, SWE_PQ_ERROR = range(4)
SWE_RQ_LAUNCHES, SWE_RQ_TILE_X, SWE_RQ_TILE_Y, SWE_RQ_SMEM, SWE_RQ_ERROR = range(5)


class SweError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, strerror(status), status))


class swe_options(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("kernel", ctypes.c_int), ("depth", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


_lib: Optional[ctypes.CDLL] = None
_vp = ctypes.c_void_p
_i, _d, _ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong

# name -> (restype, argtypes)
_SIGS = {
    "swe_options_init": (None, [ctypes.POINTER(swe_options)]),
    "swe_create": (_i, [_i, _i, _d, _d, _d, _d, ctypes.POINTER(_vp)]),
    "swe_create_ex": (_i, [_i, _i, _d, _d, _d, _d, ctypes.POINTER(swe_options), ctypes.POINTER(_vp)]),
    "swe_destroy": (None, [_vp]),
    "swe_set_dt": (_i, [_vp, _d]),
    "swe_set_state": (_i, [_vp, _vp, _vp, _vp, _ll, _i, _vp]),
    "swe_get_state": (_i, [_vp, _vp, _vp, _vp, _ll, _i, _vp]),
    "swe_step": (_i, [_vp, _i, _vp]),
    "swe_mass": (_i, [_vp, ctypes.POINTER(_d), _vp]),
    "swe_cfl_dt": (_i, [_vp, _d, ctypes.POINTER(_d), _vp]),
    "swe_run": (_i, [_vp, _i, _d, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_vp), _vp]),
    "swe_check": (_i, [_vp, _vp]),
    "swe_query": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "swe_strerror": (ctypes.c_char_p, [_i]),
    "swe_mass_noalloc": (_i, [_i, _vp, _i, _i, _ll, _d, _d, _vp, _vp]),
    "swe_batch_create": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _d, ctypes.POINTER(_vp)]),
    "swe_batch_destroy": (None, [_vp]),
    "swe_batch_set_state": (_i, [_vp, _i, _vp, _vp, _vp, _ll, _i, _vp]),
    "swe_batch_get_state": (_i, [_vp, _i, _vp, _vp, _vp, _ll, _i, _vp]),
    "swe_batch_set_dt": (_i, [_vp, _vp, _vp]),
    "swe_batch_step": (_i, [_vp, _i, _vp]),
    "swe_batch_status": (_i, [_vp, _vp, _vp]),
    "swe_batch_mass": (_i, [_vp, _vp, _vp]),
    "swe_batch_cfl_dt": (_i, [_vp, _d, _vp, _vp]),
    "swe_batch_tune": (_i, [_vp, ctypes.c_char_p, _vp]),
    "swe_batch_configure": (_i, [_vp, _i, _i]),
    "swe_batch_query": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "swe_selftest_wait": (_i, [_i, _d, _vp]),
    "swe_probe_rate": (_i, [_i, ctypes.POINTER(_d)]),
    "swe_batch_state_ptr": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "swe_batch_copy_states": (_i, [_vp, _vp, _vp]),
    "swe_net_param_count": (ctypes.c_size_t, []),
    "swe_net_create": (_i, [_i, _i, _i, ctypes.POINTER(_vp)]),
    "swe_net_destroy": (None, [_vp]),
    "swe_net_set_params": (_i, [_vp, _vp]),
    "swe_net_get_params": (_i, [_vp, _vp]),
    "swe_net_set_norm": (_i, [_vp, _vp]),
    "swe_net_prep_input": (_i, [_vp, _i, _vp, _vp, _ll, _ll, _ll, _vp]),
    "swe_net_infer": (_i, [_vp, _i, _vp, _vp]),
    "swe_net_apply": (_i, [_vp, _i, _vp, _ll, _ll, _ll, _i, _vp]),
    "swe_net_correct": (_i, [_vp, _i, _vp, _ll, _ll, _ll, _i, _vp]),
    "swe_net_make_target": (_i, [_vp, _i, _vp, _vp, _ll, _ll, _ll, ctypes.c_float, _vp, _vp]),
    "swe_net_train_step": (_i, [_vp, _i, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, _i,
                                ctypes.POINTER(_d), _vp, _vp, _vp]),
    "swe_net_check": (_i, [_vp, _vp]),
    "swe_batch_learned_step": (_i, [_vp, _vp, _i, _i, _vp]),
    "swe_net_set_loss_weighting": (_i, [_vp, ctypes.c_float, ctypes.c_float]),
    "swe_resample": (_i, [_vp, _ll, _ll, _ll, _i, _i, _vp, _ll, _ll, _ll, _i, _i, _i, _vp]),
    "swe_part_create": (_i, [_i, _i, _i, _i, _d, _d, _d, _d, ctypes.POINTER(_vp)]),
    "swe_part_destroy": (None, [_vp]),
    "swe_part_set_state": (_i, [_vp, _vp, _vp, _vp, _ll, _vp]),
    "swe_part_get_state": (_i, [_vp, _vp, _vp, _vp, _ll, _vp]),
    "swe_part_step": (_i, [_vp, _i, _vp]),
    "swe_part_query": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "swe_part_create_rank": (_i, [_i, _i, _i, _d, _d, _d, _d, ctypes.POINTER(_vp)]),
    "swe_part_edges": (_i, [_vp, _vp, _vp]),
    "swe_part_set_ghosts": (_i, [_vp, _vp, _i, _vp]),
    "swe_region_create": (_i, [_i, _i, _i, _ll, _i, ctypes.POINTER(_vp)]),
    "swe_region_destroy": (None, [_vp]),
    "swe_region_step": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _d, _d, _d, _vp]),
    "swe_region_walls": (_i, [_vp, ctypes.POINTER(_vp), _i, _vp]),
    "swe_region_step_bed": (_i, [_vp, ctypes.POINTER(_vp), _vp, ctypes.POINTER(_vp), _d, _d, _d, _d, _vp]),
    "swe_region_boundary": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i), _vp]),
    "swe_region_run_bc": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _i, ctypes.POINTER(_i), _d, _d, _d,
                               _d, _vp, ctypes.POINTER(_i)]),
    "swe_region_run": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _d, _d, _d, _d, _vp,
                            ctypes.POINTER(_i)]),
    "swe_region_query": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "swe_region_shapes": (_i, [_i, _i, ctypes.POINTER(_i), _i, ctypes.POINTER(_i)]),
    "swe_selftest_gelu": (_i, [_vp, _vp, _i, _i, _vp]),
    "swe_selftest_div": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "swe_downsample": (_i, [_i, _vp, _ll, _ll, _ll, _vp, _ll, _ll, _ll, _i, _i, _i, _vp]),
}


def lib() -> ctypes.CDLL:
    """Load libswe.so (built by paper_1107_2157_gb300.build / build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libswe.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def strerror(status: int) -> str:
    try:
        return lib().swe_strerror(int(status)).decode()
    except Exception:  # pragma: no cover
        return "status %d" % status


def check(status: int, where: str) -> None:
    if status != SWE_OK:
        raise SweError(status, where)


# --- the C ABI under its own names --------------------------------------------------

def swe_options_init() -> swe_options:
    o = swe_options()
    lib().swe_options_init(ctypes.byref(o))
    return o


def swe_create(nx, ny, dx, dy, dt, g) -> int:
    h = _vp()
    check(lib().swe_create(nx, ny, dx, dy, dt, g, ctypes.byref(h)), "swe_create")
    return h.value


def swe_create_ex(nx, ny, dx, dy, dt, g, opt: swe_options) -> int:
    h = _vp()
    check(lib().swe_create_ex(nx, ny, dx, dy, dt, g, ctypes.byref(opt), ctypes.byref(h)), "swe_create_ex")
    return h.value


def swe_destroy(ctx) -> None:
    lib().swe_destroy(ctx)


def swe_set_dt(ctx, dt) -> None:
    check(lib().swe_set_dt(ctx, dt), "swe_set_dt")


def swe_set_state(ctx, h, hu, hv, ld, on_device, stream=None) -> None:
    check(lib().swe_set_state(ctx, h, hu, hv, ld, on_device, stream), "swe_set_state")


def swe_get_state(ctx, h, hu, hv, ld, on_device, stream=None) -> None:
    check(lib().swe_get_state(ctx, h, hu, hv, ld, on_device, stream), "swe_get_state")


def swe_step(ctx, n_steps, stream=None) -> None:
    check(lib().swe_step(ctx, int(n_steps), stream), "swe_step")


def swe_mass(ctx, stream=None) -> float:
    m = _d()
    check(lib().swe_mass(ctx, ctypes.byref(m), stream), "swe_mass")
    return m.value


def swe_cfl_dt(ctx, cfl, stream=None) -> float:
    d = _d()
    check(lib().swe_cfl_dt(ctx, cfl, ctypes.byref(d), stream), "swe_cfl_dt")
    return d.value


def swe_run(ctx, n_steps, cfl, events=None, stream=None):
    """CFL dt, n_steps steps and the mass in one call (see include/swe.h);
    ``events``: optional four torch.cuda.Event (or None) recorded before the
    job, around the step launches and after the results' copy.  Returns
    (dt, mass)."""
    d, m = _d(), _d()
    ev = None
    if events is not None:
        # torch creates a CUDA event at its first record; swe_run records it
        # again at its place on ``stream``
        for e in events:
            if e is not None:
                e.record()
        ev = (_vp * 4)(*[None if e is None else e.cuda_event for e in events])
    check(lib().swe_run(ctx, int(n_steps), cfl, ctypes.byref(d), ctypes.byref(m), ev, stream), "swe_run")
    return d.value, m.value


def swe_check(ctx, stream=None) -> int:
    return int(lib().swe_check(ctx, stream))


def swe_query(ctx, key) -> int:
    v = _ll()
    check(lib().swe_query(ctx, int(key), ctypes.byref(v)), "swe_query")
    return v.value


def swe_mass_noalloc(dtype, h, nx, ny, ld, dx, dy, mass_dev, stream=None) -> None:
    """FP64 mass of a caller-owned device plane into ``mass_dev`` (device
    pointer to one double); allocates nothing (see include/swe.h)."""
    check(lib().swe_mass_noalloc(int(dtype), h, int(nx), int(ny), int(ld), dx, dy, mass_dev, stream),
          "swe_mass_noalloc")


# --- marshalling helpers -----------------------------------------------------------------

SWE_PROBE_FP32, SWE_PROBE_FP32X2, SWE_PROBE_FP64 = 0, 1, 2


def swe_probe_rate(kind) -> float:
    """Measured FMAs per second of the current device (kind: SWE_PROBE_*)."""
    r = ctypes.c_double(0.0)
    check(lib().swe_probe_rate(int(kind), ctypes.byref(r)), "swe_probe_rate")
    return r.value


def current_stream():
    """cudaStream_t of torch's current stream (as an int), or None."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


def _buf(a, dtype_np):
    """(pointer, row stride in elements, on_device) of a 2D array/tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype_np or a.ndim != 2 or a.strides[1] != a.itemsize:
            raise ValueError("expected a 2D %s array with unit x stride" % dtype_np)
        return a.ctypes.data, a.strides[0] // a.itemsize, 0
    import torch
    if not isinstance(a, torch.Tensor) or a.dim() != 2 or a.stride(1) != 1:
        raise ValueError("expected a 2D tensor with unit x stride")
    want = torch.float32 if dtype_np == np.float32 else torch.float64
    if a.dtype != want:
        raise ValueError("tensor dtype %s, expected %s" % (a.dtype, want))
    return a.data_ptr(), a.stride(0), 1 if a.is_cuda else 0


class Grid:
    """One nx x ny grid on the current CUDA device (owns a swe_ctx)."""

    def __init__(self, nx, ny, dx, dy, dt, g, dtype="f32", kernel=SWE_KERNEL_AUTO, depth=0, variant=None):
        o = swe_options_init()
        o.dtype = SWE_F64 if dtype in ("f64", np.float64) else SWE_F32
        o.kernel = kernel
        o.depth = depth
        o.reserved[0] = 0 if variant is None else int(variant) + 1
        self.np_dtype = np.float64 if o.dtype == SWE_F64 else np.float32
        self.nx, self.ny = nx, ny
        self.ctx = swe_create_ex(nx, ny, dx, dy, dt, g, o)

    def close(self):
        if getattr(self, "ctx", None):
            swe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, h, hu, hv, stream=None):
        bufs = [_buf(a, self.np_dtype) for a in (h, hu, hv)]
        if len({b[1] for b in bufs}) != 1 or len({b[2] for b in bufs}) != 1:
            raise ValueError("h, hu, hv must share row stride and location")
        swe_set_state(self.ctx, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1], bufs[0][2],
                      stream if stream is not None else current_stream())

    def get_state(self, out=None, stream=None, sync=True):
        """Copies the state to ``out`` (3 arrays/tensors) or new numpy arrays."""
        if out is None:
            out = [np.empty((self.ny, self.nx), self.np_dtype) for _ in range(3)]
        bufs = [_buf(a, self.np_dtype) for a in out]
        s = stream if stream is not None else current_stream()
        swe_get_state(self.ctx, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1], bufs[0][2], s)
        if sync:
            import torch
            torch.cuda.synchronize()
        return out

    def step(self, n, stream=None):
        swe_step(self.ctx, n, stream if stream is not None else current_stream())

    def set_dt(self, dt):
        swe_set_dt(self.ctx, dt)

    def mass(self, stream=None):
        return swe_mass(self.ctx, stream if stream is not None else current_stream())

    def cfl_dt(self, cfl, stream=None):
        return swe_cfl_dt(self.ctx, cfl, stream if stream is not None else current_stream())

    def run(self, n, cfl, events=None, stream=None):
        """The FP64 CFL dt, n steps with it and the FP64 mass, with one host
        synchronisation (swe_run); returns (dt, mass)."""
        return swe_run(self.ctx, n, cfl, events, stream if stream is not None else current_stream())

    def check(self, stream=None):
        return swe_check(self.ctx, stream if stream is not None else current_stream())

    def query(self, key):
        return swe_query(self.ctx, key)


# --- domain decomposition on one device -------------------------------------------------------

class Partitioned:
    """One FP32 grid split into px x py ghosted partitions (owns a swe_part)."""

    def __init__(self, nx, ny, px, py, dx, dy, dt, g):
        h = _vp()
        check(lib().swe_part_create(int(nx), int(ny), int(px), int(py), dx, dy, dt, g, ctypes.byref(h)),
              "swe_part_create")
        self.p = h.value
        self.nx, self.ny = nx, ny

    @classmethod
    def rank(cls, nx, ny, walls, dx, dy, dt, g):
        """One rank's nx x ny partition; ``walls``: bitmask of its sides on
        the grid boundary (1 left, 2 right, 4 bottom, 8 top)."""
        self = cls.__new__(cls)
        h = _vp()
        check(lib().swe_part_create_rank(int(nx), int(ny), int(walls), dx, dy, dt, g, ctypes.byref(h)),
              "swe_part_create_rank")
        self.p = h.value
        self.nx, self.ny = nx, ny
        return self

    def edges(self, out, stream=None):
        """The four edge strips into the float32 CUDA tensor ``out`` of
        6 (nx + ny) elements (layout in swe.h)."""
        check(lib().swe_part_edges(self.p, self._strip_ptr(out), stream if stream is not None else current_stream()),
              "swe_part_edges")

    def set_ghosts(self, strips, sides, stream=None):
        """The ghost strips of the sides in the bitmask ``sides`` from the
        float32 CUDA tensor ``strips`` (same layout as ``edges``)."""
        check(lib().swe_part_set_ghosts(self.p, self._strip_ptr(strips), int(sides),
                                        stream if stream is not None else current_stream()), "swe_part_set_ghosts")

    def _strip_ptr(self, t):
        import torch
        n = 6 * (self.nx + self.ny)
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.numel() == n):
            raise ValueError("expected a contiguous float32 CUDA tensor of %d elements" % n)
        return t.data_ptr()

    def close(self):
        if getattr(self, "p", None):
            lib().swe_part_destroy(self.p)
            self.p = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, h, hu, hv, stream=None):
        bufs = [_buf(a, np.float32) for a in (h, hu, hv)]
        check(lib().swe_part_set_state(self.p, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1],
                                       stream if stream is not None else current_stream()), "swe_part_set_state")

    def get_state(self, stream=None):
        out = [np.empty((self.ny, self.nx), np.float32) for _ in range(3)]
        bufs = [_buf(a, np.float32) for a in out]
        check(lib().swe_part_get_state(self.p, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1],
                                       stream if stream is not None else current_stream()), "swe_part_get_state")
        import torch
        torch.cuda.synchronize()
        return out

    def step(self, n, stream=None):
        check(lib().swe_part_step(self.p, int(n), stream if stream is not None else current_stream()),
              "swe_part_step")

    def query(self, key):
        v = _ll()
        check(lib().swe_part_query(self.p, int(key), ctypes.byref(v)), "swe_part_query")
        return v.value


# --- region front end ----------------------------------------------------------------------

def swe_region_shapes(nx, ny):
    """Extents (x, y) of the step's and the wall fill's statement groups on
    nx x ny interior cells (host only; nothing is evaluated)."""
    ext = (_i * 32)()
    n = _i()
    check(lib().swe_region_shapes(int(nx), int(ny), ext, 16, ctypes.byref(n)), "swe_region_shapes")
    return [(ext[2 * k], ext[2 * k + 1]) for k in range(min(n.value, 16))]


def _addr(p):
    return int(p.data_ptr()) if hasattr(p, "data_ptr") else int(p)


def _ptr3(planes):
    return (_vp * 3)(*[_addr(p) for p in planes])


class Region:
    """The step written as region statements (owns a swe_region).  State
    triples are caller-owned device planes of (ny + 2) rows x ``pitch``
    elements with the ghost ring (torch tensors or raw pointers)."""

    def __init__(self, dtype, nx, ny, pitch=None, variant=0):
        es = 8 if dtype == SWE_F64 else 4
        if pitch is None:
            pitch = ((nx + 2) * es + 127) // 128 * 128 // es
        h = _vp()
        check(lib().swe_region_create(int(dtype), int(nx), int(ny), int(pitch), int(variant), ctypes.byref(h)),
              "swe_region_create")
        self.r = h.value
        self.dtype, self.nx, self.ny, self.pitch = dtype, nx, ny, pitch

    def planes(self):
        """Three zeroed (ny + 2) x pitch device planes (torch)."""
        import torch
        t = torch.float64 if self.dtype == SWE_F64 else torch.float32
        return [torch.zeros((self.ny + 2, self.pitch), dtype=t, device="cuda") for _ in range(3)]

    def close(self):
        if getattr(self, "r", None):
            lib().swe_region_destroy(self.r)
            self.r = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, src, dst, dx, dy, dt, g, stream=None):
        check(lib().swe_region_step(self.r, _ptr3(src), _ptr3(dst), dx, dy, dt, g,
                                    stream if stream is not None else current_stream()), "swe_region_step")

    def walls(self, state, walls=15, stream=None):
        check(lib().swe_region_walls(self.r, _ptr3(state), int(walls),
                                     stream if stream is not None else current_stream()), "swe_region_walls")

    def step_bed(self, src, bed, dst, dx, dy, dt, g, stream=None):
        check(lib().swe_region_step_bed(self.r, _ptr3(src), _vp(_addr(bed)), _ptr3(dst), dx, dy, dt, g,
                                        stream if stream is not None else current_stream()), "swe_region_step_bed")

    def boundary(self, state, kinds, stream=None):
        """kinds per side (left, right, bottom, top): 0 none, 1 wall, 2 open."""
        check(lib().swe_region_boundary(self.r, _ptr3(state), (_i * 4)(*kinds),
                                        stream if stream is not None else current_stream()), "swe_region_boundary")

    def run_bc(self, a, b, n_steps, dx, dy, dt, g, kinds=(1, 1, 1, 1), bed=None, stream=None):
        """n_steps of (boundary, step[, over the bed]) from a; returns 1 if the result is in b."""
        in_b = _i()
        check(lib().swe_region_run_bc(self.r, _ptr3(a), _ptr3(b), _vp(_addr(bed)) if bed is not None else None,
                                      int(n_steps), (_i * 4)(*kinds), dx, dy, dt, g,
                                      stream if stream is not None else current_stream(), ctypes.byref(in_b)),
              "swe_region_run_bc")
        return in_b.value

    def run(self, a, b, n_steps, dx, dy, dt, g, walls=15, stream=None):
        """n_steps of (walls, step) from a; returns 1 if the result is in b."""
        in_b = _i()
        check(lib().swe_region_run(self.r, _ptr3(a), _ptr3(b), int(n_steps), int(walls), dx, dy, dt, g,
                                   stream if stream is not None else current_stream(), ctypes.byref(in_b)),
              "swe_region_run")
        return in_b.value

    def query(self, key):
        v = _ll()
        check(lib().swe_region_query(self.r, int(key), ctypes.byref(v)), "swe_region_query")
        return v.value


# --- batched ensembles ----------------------------------------------------------------------

def _dptr(a):
    return a.ctypes.data_as(_vp)


class Batch:
    """Many FP32 grids stepped together (owns a swe_batch)."""

    def __init__(self, sizes, dx, dy, dt, g):
        n = len(sizes)
        self.n = n
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self._nx = np.array([s[0] for s in self.sizes], np.int32)
        self._ny = np.array([s[1] for s in self.sizes], np.int32)
        self._dx = np.ascontiguousarray(np.broadcast_to(np.asarray(dx, np.float64), (n,)))
        self._dy = np.ascontiguousarray(np.broadcast_to(np.asarray(dy, np.float64), (n,)))
        dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (n,)))
        h = _vp()
        check(lib().swe_batch_create(n, _dptr(self._nx), _dptr(self._ny), _dptr(self._dx), _dptr(self._dy),
                                     _dptr(dtv), g, ctypes.byref(h)), "swe_batch_create")
        self.b = h.value

    def close(self):
        if getattr(self, "b", None):
            lib().swe_batch_destroy(self.b)
            self.b = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, i, h, hu, hv, stream=None):
        bufs = [_buf(a, np.float32) for a in (h, hu, hv)]
        check(lib().swe_batch_set_state(self.b, i, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1], bufs[0][2],
                                        stream if stream is not None else current_stream()),
              "swe_batch_set_state")

    def get_state(self, i, out=None, stream=None, sync=True):
        nx, ny = self.sizes[i]
        if out is None:
            out = [np.empty((ny, nx), np.float32) for _ in range(3)]
        bufs = [_buf(a, np.float32) for a in out]
        check(lib().swe_batch_get_state(self.b, i, bufs[0][0], bufs[1][0], bufs[2][0], bufs[0][1], bufs[0][2],
                                        stream if stream is not None else current_stream()),
              "swe_batch_get_state")
        if sync:
            import torch
            torch.cuda.synchronize()
        return out

    def set_dt(self, dt, stream=None):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (self.n,)))
        check(lib().swe_batch_set_dt(self.b, _dptr(d), stream if stream is not None else current_stream()),
              "swe_batch_set_dt")

    def step(self, n, stream=None):
        check(lib().swe_batch_step(self.b, int(n), stream if stream is not None else current_stream()),
              "swe_batch_step")

    def learned_step(self, net: "Net", n, project_mass=True, stream=None):
        """n learned coarse steps (Lax-Wendroff + corrector) in one launch."""
        check(lib().swe_batch_learned_step(self.b, net.t, int(n), int(project_mass),
                                           stream if stream is not None else current_stream()),
              "swe_batch_learned_step")

    def status(self, stream=None):
        f = np.zeros(self.n, np.int32)
        rc = lib().swe_batch_status(self.b, _dptr(f), stream if stream is not None else current_stream())
        return rc, f

    def mass(self, stream=None):
        m = np.zeros(self.n, np.float64)
        check(lib().swe_batch_mass(self.b, _dptr(m), stream if stream is not None else current_stream()),
              "swe_batch_mass")
        return m

    def cfl_dt(self, cfl, stream=None):
        d = np.zeros(self.n, np.float64)
        check(lib().swe_batch_cfl_dt(self.b, cfl, _dptr(d), stream if stream is not None else current_stream()),
              "swe_batch_cfl_dt")
        return d

    def tune(self, cache_path=None, stream=None):
        p = cache_path.encode() if cache_path else None
        check(lib().swe_batch_tune(self.b, p, stream if stream is not None else current_stream()),
              "swe_batch_tune")

    def configure(self, variant, ctas_per_sm):
        check(lib().swe_batch_configure(self.b, int(variant), int(ctas_per_sm)), "swe_batch_configure")

    def query(self, key):
        v = _ll()
        check(lib().swe_batch_query(self.b, int(key), ctypes.byref(v)), "swe_batch_query")
        return v.value

    def copy_states(self, dst_ptr, stream=None):
        """All current states into a contiguous device buffer [n][3][ny][nx]."""
        check(lib().swe_batch_copy_states(self.b, dst_ptr, stream if stream is not None else current_stream()),
              "swe_batch_copy_states")

    def state_ptr(self, i):
        """(device address of instance i's h plane, plane stride, pitch)."""
        p, ps, pi = _vp(), _ll(), _ll()
        check(lib().swe_batch_state_ptr(self.b, int(i), ctypes.byref(p), ctypes.byref(ps), ctypes.byref(pi)),
              "swe_batch_state_ptr")
        return p.value, ps.value, pi.value


# --- learned corrector -------------------------------------------------------------------------

PARAM_SHAPES = [("W1", (3, 3, 3, 32)), ("b1", (32,)), ("W2", (3, 3, 32, 32)), ("b2", (32,)),
                ("W3", (3, 3, 32, 3)), ("b3", (3,))]


def flatten_params(params) -> np.ndarray:
    """dict of arrays (W[ky][kx][c_in][c_out], b[c_out]) -> flat float32."""
    return np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k, _ in PARAM_SHAPES])


def unflatten_params(flat):
    out, o = {}, 0
    for k, shp in PARAM_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


class Net:
    """The corrector network on the current device (owns a swe_net)."""

    def __init__(self, max_images, H, W):
        h = _vp()
        check(lib().swe_net_create(int(max_images), int(H), int(W), ctypes.byref(h)), "swe_net_create")
        self.t = h.value
        self.H, self.W, self.max_images = H, W, max_images
        self.nparams = int(lib().swe_net_param_count())

    def close(self):
        if getattr(self, "t", None):
            lib().swe_net_destroy(self.t)
            self.t = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, np.float32)
        assert a.size == self.nparams
        check(lib().swe_net_set_params(self.t, a.ctypes.data), "swe_net_set_params")

    def get_params(self):
        a = np.zeros(self.nparams, np.float32)
        check(lib().swe_net_get_params(self.t, a.ctypes.data), "swe_net_get_params")
        return a

    def set_norm(self, h0, sh, su, oh, ou):
        a = np.array([h0, sh, su, oh, ou], np.float32)
        check(lib().swe_net_set_norm(self.t, a.ctypes.data), "swe_net_set_norm")

    def set_loss_weighting(self, power, floor=1.0):
        check(lib().swe_net_set_loss_weighting(self.t, float(power), float(floor)), "swe_net_set_loss_weighting")

    def prep_input(self, n, state_ptr, img_stride, plane_stride, pitch, base_ptr=None, stream=None):
        check(lib().swe_net_prep_input(self.t, n, state_ptr, base_ptr, img_stride, plane_stride, pitch,
                                       stream if stream is not None else current_stream()), "swe_net_prep_input")

    def infer(self, n, resid_ptr=None, stream=None):
        check(lib().swe_net_infer(self.t, n, resid_ptr, stream if stream is not None else current_stream()),
              "swe_net_infer")

    def apply(self, n, state_ptr, img_stride, plane_stride, pitch, project_mass=True, stream=None):
        check(lib().swe_net_apply(self.t, n, state_ptr, img_stride, plane_stride, pitch, int(project_mass),
                                  stream if stream is not None else current_stream()), "swe_net_apply")

    def correct(self, n, state_ptr, img_stride, plane_stride, pitch, project_mass=True, stream=None):
        check(lib().swe_net_correct(self.t, n, state_ptr, img_stride, plane_stride, pitch, int(project_mass),
                                    stream if stream is not None else current_stream()), "swe_net_correct")

    def make_target(self, n, next_ptr, lw_ptr, img_stride, plane_stride, pitch, target_ptr, clip=0.0, stream=None):
        check(lib().swe_net_make_target(self.t, n, next_ptr, lw_ptr, img_stride, plane_stride, pitch, clip,
                                        target_ptr, stream if stream is not None else current_stream()),
              "swe_net_make_target")

    def train_step(self, n, target_ptr, lr=1e-3, wd=0.0, clip=0.0, update=True, want_grads=False,
                   resid_ptr=None, stream=None):
        loss = _d()
        g = np.zeros(self.nparams, np.float32) if want_grads else None
        check(lib().swe_net_train_step(self.t, n, target_ptr, lr, wd, clip, int(update), ctypes.byref(loss),
                                       g.ctypes.data if g is not None else None, resid_ptr,
                                       stream if stream is not None else current_stream()), "swe_net_train_step")
        return loss.value, g

    def check(self, stream=None):
        return int(lib().swe_net_check(self.t, stream if stream is not None else current_stream()))


def swe_downsample(factor, fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc, n, stream=None):
    check(lib().swe_downsample(int(factor), fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc,
                               n, stream if stream is not None else current_stream()), "swe_downsample")


def swe_resample(src, s_img, s_plane, s_pitch, Ws, Hs, dst, d_img, d_plane, d_pitch, Wd, Hd, n, stream=None):
    check(lib().swe_resample(src, s_img, s_plane, s_pitch, Ws, Hs, dst, d_img, d_plane, d_pitch, Wd, Hd, n,
                             stream if stream is not None else current_stream()), "swe_resample")
