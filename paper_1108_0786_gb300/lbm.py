"""ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the coupled method runs in the CUDA library
``_build/liblbm.so``; this module only converts Python / numpy / torch
arguments.  ``Lattice`` raises if the library or a CUDA device is missing:
there is no CPU fallback.

PyTorch supplies device memory and streams: ``Lattice(..., torch_memory=True)``
installs torch's caching allocator as the library's allocator hook and runs
the library on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

from . import _build

OK = 0
E_ARG, E_OOM, E_OVERLAP, E_OUTSIDE, E_NAN, E_LINKS, E_TIMEOUT, E_CUDA, E_STATE, E_UNSTABLE = (
    -1, -2, -3, -4, -5, -6, -7, -8, -9, -10)
BC_PERIODIC_X, BC_PERIODIC_Y, BC_PERIODIC_Z = 1, 2, 4
SHAPE_SPHERE, SHAPE_CAPSULE = 0, 1
PREC_F64, PREC_F32, PREC_F16, PREC_BF16 = 0, 1, 2, 3
OPT_NO_FLUID = 1
OPT_OVERLAP = 4
DEBUG_EXPIRE_WAITS, DEBUG_CELL_LIST_CAP, DEBUG_ADJOINT_SERIAL, DEBUG_NO_PDL = 1, 2, 3, 4
ENSEMBLE_BATCHED, ENSEMBLE_BRANCHES = 0, 1
OPT_AVERAGE_FORCE = 2
FIELD_RHO, FIELD_U, FIELD_FLAGS, FIELD_POP = 0, 1, 2, 3
DTYPE_F64, DTYPE_F32, DTYPE_U8 = 0, 1, 2
KERNEL_NAMES = ("remap", "stream_collide", "boundary", "links", "force", "integrate")
PRECISIONS = {"f64": PREC_F64, "f32": PREC_F32, "f16": PREC_F16, "bf16": PREC_BF16}

EXPORTED = (
    "lbm_create", "lbm_create_ex", "lbm_destroy", "lbm_set_allocator", "lbm_set_stream",
    "lbm_add_body", "lbm_body_properties", "lbm_add_spring", "lbm_set_drive", "lbm_set_drive_window", "lbm_set_drive_axis",
    "lbm_set_body_state", "lbm_set_fields", "lbm_step", "lbm_sync", "lbm_steps_done",
    "lbm_average_begin", "lbm_average_stop", "lbm_average_get",
    "lbm_get_bodies", "lbm_get_bodies_async", "lbm_wait_ticket", "lbm_get_forces", "lbm_get_fields",
    "lbm_get_fields_device",
    "lbm_enable_history", "lbm_get_history", "lbm_save", "lbm_load", "lbm_time_kernels",
    "lbm_tune", "lbm_debug_set", "lbm_autotune", "lbm_kernels_per_step", "lbm_bytes_per_cell",
    "lbm_last_error",
    "lbm_momentum_exchange_static", "lbm_adjoint_record", "lbm_adjoint_backward",
    "lbm_ensemble_create", "lbm_ensemble_set_mode", "lbm_ensemble_autotune", "lbm_ensemble_step",
    "lbm_ensemble_sync", "lbm_ensemble_destroy", "lbm_ensemble_last_error",
)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(path: Optional[str] = None):
    """Load the CUDA library (no compilation); raises OSError if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise OSError(f"CUDA library {p} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    DP = ctypes.POINTER(ctypes.c_double)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "lbm_create": ([I, I, I, D, I, PP], I),
        "lbm_create_ex": ([I, I, I, D, I, I, DP, I, PP], I),
        "lbm_destroy": ([P], I),
        "lbm_set_allocator": ([P, ALLOC_FN, FREE_FN, P], I),
        "lbm_set_stream": ([P, P], I),
        "lbm_add_body": ([P, I, D, D, D, DP, DP], I),
        "lbm_add_spring": ([P, I, I, D, D, D], I),
        "lbm_set_drive": ([P, I, D, D, D], I),
        "lbm_set_drive_window": ([P, I, D], I),
        "lbm_set_drive_axis": ([P, I, DP], I),
        "lbm_set_body_state": ([P, I, DP], I),
        "lbm_set_fields": ([P, I, P, I], I),
        "lbm_step": ([P, I], I),
        "lbm_sync": ([P], I),
        "lbm_steps_done": ([P], ctypes.c_longlong),
        "lbm_get_bodies": ([P, DP], I),
        "lbm_get_bodies_async": ([P, DP, ctypes.POINTER(ctypes.c_longlong)], I),
        "lbm_wait_ticket": ([P, ctypes.c_longlong], I),
        "lbm_get_forces": ([P, DP], I),
        "lbm_get_fields": ([P, I, P, I], I),
        "lbm_get_fields_device": ([P, I, P, I], I),
        "lbm_enable_history": ([P, I], I),
        "lbm_get_history": ([P, DP, I, ctypes.POINTER(I)], I),
        "lbm_save": ([P, ctypes.c_char_p], I),
        "lbm_load": ([P, ctypes.c_char_p], I),
        "lbm_time_kernels": ([P, I, DP, I], I),
        "lbm_tune": ([P, I, I], I),
        "lbm_debug_set": ([P, I, ctypes.c_longlong], I),
        "lbm_body_properties": ([I, D, D, D, DP, DP, DP], I),
        "lbm_average_begin": ([P], I),
        "lbm_average_stop": ([P], I),
        "lbm_average_get": ([P, DP, ctypes.POINTER(ctypes.c_longlong)], I),
        "lbm_autotune": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "lbm_kernels_per_step": ([P], I),
        "lbm_bytes_per_cell": ([P], I),
        "lbm_last_error": ([P], ctypes.c_char_p),
        "lbm_momentum_exchange_static": ([P, P, P, I, I, I, I, I, I, P, P], I),
        "lbm_adjoint_record": ([P, I, I], I),
        "lbm_adjoint_backward": ([P, DP, DP, DP, DP, DP, DP, DP], I),
        "lbm_ensemble_create": ([ctypes.POINTER(P), I, PP], I),
        "lbm_ensemble_step": ([P, ctypes.POINTER(I)], I),
        "lbm_ensemble_set_mode": ([P, I], I),
        "lbm_ensemble_autotune": ([P, I, ctypes.POINTER(I)], I),
        "lbm_ensemble_sync": ([P], I),
        "lbm_ensemble_destroy": ([P], I),
        "lbm_ensemble_last_error": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


def body_properties(shape, radius, length, mass):
    """(V, I1, I2, I3) of a uniform solid sphere or capsule as lbm_add_body
    computes them, and their derivatives with respect to mass and length
    (lbm_body_properties; runs on the host)."""
    q, dm, dl = np.zeros(4), np.zeros(4), np.zeros(4)
    rc = load_library().lbm_body_properties(int(shape), float(radius), float(length), float(mass), _dp(q),
                                            _dp(dm), _dp(dl))
    if rc != OK:
        raise LbmError(rc, "bad body dimensions")
    return q, dm, dl


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Lattice:
    """One D3Q19 lattice with rigid bodies on the current CUDA device.

    Mirrors ``include/lbm.h``: ``add_body``, ``add_spring``, ``set_drive``,
    ``step``, ``bodies``, ``forces``, ``field`` ...  With ``torch_memory``
    (default) device memory comes from torch's caching allocator and work
    runs on torch's current stream.
    """

    def __init__(self, nx, ny, nz, tau, bc=7, precision="f32", g=(0.0, 0.0, 0.0), options=0,
                 torch_memory=True):
        self._lib = load_library()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        self.precision = prec
        self.g = tuple(float(v) for v in g)
        h = ctypes.c_void_p()
        gg = np.ascontiguousarray(g, dtype=np.float64)
        rc = self._lib.lbm_create_ex(nx, ny, nz, float(tau), int(bc), prec, _dp(gg), int(options),
                                     ctypes.byref(h))
        if rc != OK:
            raise LbmError(rc, "lbm_create_ex failed")
        self._h = h
        self.nbodies = 0
        self.nsprings = 0
        self.ndrives = 0
        self._callbacks = None
        if torch_memory:
            self._use_torch()

    # -- plumbing ---------------------------------------------------------
    def _use_torch(self):
        import torch
        if not torch.cuda.is_available():
            raise LbmError(E_CUDA, "no CUDA device: the library has no CPU path")
        dev = torch.cuda.current_device()
        stream = torch.cuda.current_stream(dev)

        def alloc(nbytes, ctx):
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

        def free(ptr, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self._callbacks = (ALLOC_FN(alloc), FREE_FN(free))
        self._check(self._lib.lbm_set_allocator(self._h, self._callbacks[0], self._callbacks[1], None))
        self._check(self._lib.lbm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        self._torch_stream = stream

    def _check(self, rc):
        if rc < 0:
            raise LbmError(rc, self._lib.lbm_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int):
        self._check(self._lib.lbm_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    # -- setup ------------------------------------------------------------
    def add_body(self, shape, radius, length, mass, pos, orient=(1.0, 0.0, 0.0, 0.0)):
        p = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(orient, dtype=np.float64)
        b = self._check(self._lib.lbm_add_body(self._h, int(shape), float(radius), float(length),
                                               float(mass), _dp(p), _dp(q)))
        self.nbodies += 1
        return b

    def add_spring(self, i, j, k, rest, damping):
        s = self._check(self._lib.lbm_add_spring(self._h, int(i), int(j), float(k), float(rest),
                                                 float(damping)))
        self.nsprings += 1
        return s

    def set_drive(self, body, amp, freq, phase):
        d = self._check(self._lib.lbm_set_drive(self._h, int(body), float(amp), float(freq),
                                                float(phase)))
        self.ndrives += 1
        return d

    def set_drive_window(self, term, t_off):
        return self._check(self._lib.lbm_set_drive_window(self._h, int(term), float(t_off)))

    def set_drive_axis(self, term, axis):
        a = np.ascontiguousarray(axis, dtype=np.float64)
        return self._check(self._lib.lbm_set_drive_axis(self._h, int(term), _dp(a)))

    def set_body_state(self, body, state):
        s = np.ascontiguousarray(state, dtype=np.float64)
        assert s.size == 13
        return self._check(self._lib.lbm_set_body_state(self._h, int(body), _dp(s)))

    def set_pop(self, pop):
        p = np.ascontiguousarray(pop, dtype=np.float64).reshape(-1)
        assert p.size == 19 * self.cells
        return self._check(self._lib.lbm_set_fields(self._h, FIELD_POP, p.ctypes.data_as(ctypes.c_void_p),
                                                    DTYPE_F64))

    def tune(self, cells_per_thread, min_blocks_per_sm=0):
        """Launch shape of the bulk stream-collide kernel (0: default)."""
        return self._check(self._lib.lbm_tune(self._h, int(cells_per_thread), int(min_blocks_per_sm)))

    def average_begin(self):
        """Start (or restart) the running time average of the velocity field."""
        return self._check(self._lib.lbm_average_begin(self._h))

    def average_stop(self):
        return self._check(self._lib.lbm_average_stop(self._h))

    def average(self):
        """(mean velocity [3, nz, ny, nx], steps averaged)."""
        out = np.zeros((3,) + self.shape)
        n = ctypes.c_longlong()
        self._check(self._lib.lbm_average_get(self._h, _dp(out), ctypes.byref(n)))
        return out, int(n.value)

    def debug_set(self, knob, value):
        """A check of a failure path (DEBUG_EXPIRE_WAITS, DEBUG_CELL_LIST_CAP:
        before the first step) or of a schedule (DEBUG_ADJOINT_SERIAL: the
        reverse sweep's; DEBUG_NO_PDL: the step graphs' launches; any time)."""
        return self._check(self._lib.lbm_debug_set(self._h, int(knob), int(value)))

    def autotune(self, trials=5):
        """Time the compiled bulk-kernel shapes and keep the fastest;
        returns (cells_per_thread, min_blocks_per_sm)."""
        v, m = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._lib.lbm_autotune(self._h, int(trials), ctypes.byref(v), ctypes.byref(m)))
        return v.value, m.value

    def enable_history(self, capacity):
        return self._check(self._lib.lbm_enable_history(self._h, int(capacity)))

    # -- stepping ---------------------------------------------------------
    def step(self, n=1):
        return self._check(self._lib.lbm_step(self._h, int(n)))

    def sync(self):
        return self._check(self._lib.lbm_sync(self._h))

    @property
    def steps_done(self):
        return int(self._lib.lbm_steps_done(self._h))

    # -- results ----------------------------------------------------------
    def bodies(self):
        out = np.zeros((self.nbodies, 13))
        self._check(self._lib.lbm_get_bodies(self._h, _dp(out)))
        return out

    def bodies_async(self, out):
        """Enqueue a read of the body states after the steps enqueued so far
        into ``out`` (float64 [nbodies, 13], C-contiguous; page-locked memory,
        e.g. a pinned torch tensor's ``.numpy()``, for an asynchronous copy;
        it must stay alive until the read is waited for); returns a ticket
        for ``wait``."""
        if out.dtype != np.float64 or out.shape != (self.nbodies, 13) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of shape (nbodies, 13)")
        t = ctypes.c_longlong(-1)
        self._check(self._lib.lbm_get_bodies_async(self._h, _dp(out), ctypes.byref(t)))
        return t.value

    def wait(self, ticket):
        """Wait for the read with this ticket; raises the first error the
        device had latched by then."""
        return self._check(self._lib.lbm_wait_ticket(self._h, int(ticket)))

    def forces(self):
        out = np.zeros((self.nbodies, 6))
        self._check(self._lib.lbm_get_forces(self._h, _dp(out)))
        return out

    def field(self, what, dtype=DTYPE_F64):
        nz, ny, nx = self.shape
        if what == FIELD_FLAGS:
            dtype = DTYPE_U8
            out = np.zeros((nz, ny, nx), dtype=np.uint8)
        else:
            npd = np.float64 if dtype == DTYPE_F64 else np.float32
            lead = {FIELD_RHO: (), FIELD_U: (3,), FIELD_POP: (19,)}[what]
            out = np.zeros(lead + (nz, ny, nx), dtype=npd)
        self._check(self._lib.lbm_get_fields(self._h, int(what), out.ctypes.data_as(ctypes.c_void_p),
                                             int(dtype)))
        return out

    def field_device(self, what, out_tensor, dtype=DTYPE_F64):
        """Write a field into a caller-owned CUDA tensor (enqueued, no sync)."""
        return self._check(self._lib.lbm_get_fields_device(self._h, int(what),
                                                           ctypes.c_void_p(out_tensor.data_ptr()),
                                                           int(dtype)))

    def rho(self):
        return self.field(FIELD_RHO)

    def u(self):
        return self.field(FIELD_U)

    def flags(self):
        return self.field(FIELD_FLAGS)

    def pop(self):
        return self.field(FIELD_POP)

    def history(self, max_steps=None):
        cap = max_steps if max_steps is not None else self.steps_done
        out = np.zeros((max(cap, 0), self.nbodies, 13))
        n = ctypes.c_int(0)
        self._check(self._lib.lbm_get_history(self._h, _dp(out), int(cap), ctypes.byref(n)))
        return out[: n.value]

    def save(self, path):
        return self._check(self._lib.lbm_save(self._h, os.fsencode(path)))

    def load(self, path):
        return self._check(self._lib.lbm_load(self._h, os.fsencode(path)))

    # -- reverse mode ---------------------------------------------------------
    def adjoint_record(self, n, segment=64):
        """Advance n steps keeping the recording the reverse sweep needs
        (checkpoints every ``segment`` steps)."""
        return self._check(self._lib.lbm_adjoint_record(self._h, int(n), int(segment)))

    def adjoint_backward(self, seed, want_pop=False):
        """Gradient of sum(seed * body states after the recorded run) (seed:
        nbodies x 13) as a dict: ``state``, ``prev``, ``drive`` (nd x 2: amp,
        phase), ``spring`` (ns x 3: k, rest, damping), ``body`` (nb x 5:
        mass, I1, I2, I3, volume) and, with ``want_pop``, ``pop`` (19 x
        cells)."""
        sd = np.ascontiguousarray(seed, dtype=np.float64).reshape(self.nbodies, 13)
        out = {"state": np.zeros((self.nbodies, 13)), "prev": np.zeros((self.nbodies, 13)),
               "drive": np.zeros((self.ndrives, 2)), "spring": np.zeros((self.nsprings, 3)),
               "body": np.zeros((self.nbodies, 5))}
        if want_pop:
            nz, ny, nx = self.shape
            out["pop"] = np.zeros((19, nz, ny, nx))
        keys = ("state", "prev", "drive", "spring", "body", "pop")
        ptr = [_dp(out[k]) if k in out and out[k].size else None for k in keys]
        self._check(self._lib.lbm_adjoint_backward(self._h, _dp(sd), *ptr))
        return out

    def time_kernels(self, n):
        """Average per-kernel duration in ms over n eagerly launched steps."""
        out = np.zeros(len(KERNEL_NAMES))
        self._check(self._lib.lbm_time_kernels(self._h, int(n), _dp(out), len(KERNEL_NAMES)))
        return dict(zip(KERNEL_NAMES, out.tolist()))

    @property
    def kernels_per_step(self):
        return self._check(self._lib.lbm_kernels_per_step(self._h))

    @property
    def bytes_per_cell(self):
        return self._check(self._lib.lbm_bytes_per_cell(self._h))


def from_scenario(sc, precision="f32", torch_memory=True, options=0, history=0):
    """Build a Lattice from a seeded ``workloads.Scenario``."""
    lat = Lattice(sc.nx, sc.ny, sc.nz, sc.tau, sc.bc, precision, sc.g, options, torch_memory)
    if history:
        lat.enable_history(history)
    for b in sc.bodies:
        lat.add_body(b.shape, b.radius, b.length, b.mass, b.pos, b.orient)
    for s in sc.springs:
        lat.add_spring(s.i, s.j, s.k, s.rest, s.damping)
    for d in sc.drives:
        t = lat.set_drive(d.body, d.amp, d.freq, d.phase)
        if math.isfinite(d.t_off):
            lat.set_drive_window(t, d.t_off)
        axis = tuple(getattr(d, "axis", (1.0, 0.0, 0.0)))
        if axis != (1.0, 0.0, 0.0):
            lat.set_drive_axis(t, axis)
    return lat


class Ensemble:
    """Independent lattices stepped together (``lbm_ensemble_*``): one CUDA
    graph launch advances every member that still has whole 16-step chunks
    left; by default each step is one batched launch of each per-step kernel
    over all members.  Members must share a stream (lattices created with
    torch_memory use torch's current stream)."""

    def __init__(self, lattices):
        self._lib = load_library()
        self.members = list(lattices)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        h = ctypes.c_void_p()
        rc = self._lib.lbm_ensemble_create(arr, len(self.members), ctypes.byref(h))
        if rc != OK:
            raise LbmError(rc, "lbm_ensemble_create failed: " +
                           self.members[0]._lib.lbm_last_error(self.members[0]._h).decode())
        self._h = h

    def _check(self, rc):
        if rc < 0:
            raise LbmError(rc, self._lib.lbm_ensemble_last_error(self._h).decode())
        return rc

    def step(self, steps):
        """Advance member i by steps[i] steps (an int applies to all)."""
        if isinstance(steps, int):
            steps = [steps] * len(self.members)
        arr = (ctypes.c_int * len(self.members))(*[int(v) for v in steps])
        return self._check(self._lib.lbm_ensemble_step(self._h, arr))

    def sync(self):
        return self._check(self._lib.lbm_ensemble_sync(self._h))

    def set_mode(self, mode):
        """ENSEMBLE_BATCHED (default) or ENSEMBLE_BRANCHES."""
        return self._check(self._lib.lbm_ensemble_set_mode(self._h, int(mode)))

    def autotune(self, trials=3):
        """Time the batched bulk shapes and keep the fastest; returns its
        cells per thread."""
        v = ctypes.c_int(0)
        self._check(self._lib.lbm_ensemble_autotune(self._h, int(trials), ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
