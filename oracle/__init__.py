"""FP64 CPU oracle of the coupled D3Q19 lattice Boltzmann / rigid-body step.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference that the
GPU library is checked against (Pickl et al., arXiv:1108.0786, Sec. 2.1-2.3,
Algorithms 1-2).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the GPU package and never imports it.

``build()`` compiles ``lbm_oracle.c`` with gcc (-O2, no fast-math, OpenMP)
into ``oracle/_build/liblbm_oracle.so``; ``Oracle`` drives it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_oracle.so")

BC_PERIODIC_X, BC_PERIODIC_Y, BC_PERIODIC_Z = 1, 2, 4
SHAPE_SPHERE, SHAPE_CAPSULE = 0, 1
OPT_NO_FLUID = 1
OPT_AVERAGE_FORCE = 2
FIELD_RHO, FIELD_U, FIELD_FLAGS, FIELD_POP = 0, 1, 2, 3

# error codes returned by the oracle (same numeric values as the GPU library)
E_ARG, E_OOM, E_OVERLAP, E_OUTSIDE, E_NAN, E_STATE = -1, -2, -3, -4, -5, -9

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(LIB) or
             os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                         os.path.getmtime(os.path.join(HERE, "lbm_oracle.h"))))
    if force or stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-D_DEFAULT_SOURCE", "-Wall", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path: str):
    """Load a compiled copy of the oracle (this one, or a copy a test compiled
    from an edited source) and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    DP = ctypes.POINTER(ctypes.c_double)
    lib.lbm_ref_create_ex.argtypes = [I, I, I, D, I, DP, I, ctypes.POINTER(P)]
    lib.lbm_ref_destroy.argtypes = [P]
    lib.lbm_ref_add_body.argtypes = [P, I, D, D, D, DP, DP]
    lib.lbm_ref_add_spring.argtypes = [P, I, I, D, D, D]
    lib.lbm_ref_set_drive.argtypes = [P, I, D, D, D]
    lib.lbm_ref_set_drive_window.argtypes = [P, I, D]
    lib.lbm_ref_set_drive_axis.argtypes = [P, I, DP]
    lib.lbm_ref_set_body_state.argtypes = [P, I, DP]
    lib.lbm_ref_step.argtypes = [P, I]
    lib.lbm_ref_average_begin.argtypes = [P]
    lib.lbm_ref_average_get.argtypes = [P, DP, ctypes.POINTER(ctypes.c_long)]
    lib.lbm_ref_get_bodies.argtypes = [P, DP]
    lib.lbm_ref_get_forces.argtypes = [P, DP]
    lib.lbm_ref_get_fields.argtypes = [P, I, P]
    lib.lbm_ref_set_pop.argtypes = [P, DP]
    lib.lbm_ref_steps_done.argtypes = [P]
    lib.lbm_ref_steps_done.restype = ctypes.c_long
    lib.lbm_ref_num_threads.argtypes = []
    lib.lbm_ref_set_num_threads.argtypes = [I]
    lib.lbm_ref_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), DP]
    lib.lbm_ref_equilibrium.argtypes = [D, DP, DP]
    lib.lbm_ref_body_props.argtypes = [P, I, DP]
    lib.lbm_ref_adjoint.argtypes = [P, I, DP, DP, DP, DP, DP, DP, DP]
    lib.lbm_ref_flag_digest.argtypes = [P]
    lib.lbm_ref_flag_digest.restype = ctypes.c_ulonglong
    lib.lbm_ref_last_error.argtypes = [P]
    lib.lbm_ref_last_error.restype = ctypes.c_char_p
    return lib


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().lbm_ref_num_threads())


def set_num_threads(n: int) -> int:
    """Use n OpenMP threads from now on; returns the count in use."""
    return int(_load().lbm_ref_set_num_threads(int(n)))


def lattice():
    """The oracle's velocity set e[19][3] (int) and weights w[19]."""
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    _load().lbm_ref_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    return e.astype(np.int64), w


def equilibrium(rho, u):
    """The oracle's f_eq(rho, u) for the 19 directions."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(19)
    _load().lbm_ref_equilibrium(float(rho), _dp(uu), _dp(out))
    return out


def from_scenario(sc, options=0, lib=None):
    """An Oracle holding the domain, bodies, springs and drive terms of a
    seeded scenario (any object with the fields of ``workloads.Scenario``)."""
    import math
    o = Oracle(sc.nx, sc.ny, sc.nz, sc.tau, sc.bc, sc.g, options, lib=lib)
    for b in sc.bodies:
        o.add_body(b.shape, b.radius, b.length, b.mass, b.pos, b.orient)
    for s in sc.springs:
        o.add_spring(s.i, s.j, s.k, s.rest, s.damping)
    for d in sc.drives:
        t = o.set_drive(d.body, d.amp, d.freq, d.phase)
        if math.isfinite(d.t_off):
            o.set_drive_window(t, d.t_off)
        axis = tuple(getattr(d, "axis", (1.0, 0.0, 0.0)))
        if axis != (1.0, 0.0, 0.0):
            o.set_drive_axis(t, axis)
    return o


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """ctypes wrapper of one oracle lattice (lattice units, dx = dt = 1)."""

    def __init__(self, nx, ny, nz, tau, bc=7, g=(0.0, 0.0, 0.0), options=0, lib=None):
        self._lib = lib if lib is not None else _load()
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        h = ctypes.c_void_p()
        gg = np.ascontiguousarray(g, dtype=np.float64)
        rc = self._lib.lbm_ref_create_ex(nx, ny, nz, float(tau), int(bc), _dp(gg),
                                         int(options), ctypes.byref(h))
        if rc != 0:
            raise OracleError(rc, "create failed")
        self._h = h
        self.nbodies = 0
        self.nsprings = 0
        self.ndrives = 0

    def _check(self, rc):
        if rc < 0:
            raise OracleError(rc, self._lib.lbm_ref_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_ref_destroy(self._h)
            self._h = None

    __del__ = close

    def add_body(self, shape, radius, length, mass, pos, orient=(1.0, 0.0, 0.0, 0.0)):
        p = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(orient, dtype=np.float64)
        b = self._check(self._lib.lbm_ref_add_body(self._h, int(shape), float(radius),
                                                   float(length), float(mass), _dp(p), _dp(q)))
        self.nbodies += 1
        return b

    def add_spring(self, i, j, k, rest, damping):
        s = self._check(self._lib.lbm_ref_add_spring(self._h, i, j, float(k), float(rest),
                                                     float(damping)))
        self.nsprings += 1
        return s

    def set_drive(self, body, amp, freq, phase):
        d = self._check(self._lib.lbm_ref_set_drive(self._h, body, float(amp), float(freq),
                                                    float(phase)))
        self.ndrives += 1
        return d

    def set_drive_window(self, term, t_off):
        return self._check(self._lib.lbm_ref_set_drive_window(self._h, term, float(t_off)))

    def set_drive_axis(self, term, axis):
        a = np.ascontiguousarray(axis, dtype=np.float64)
        return self._check(self._lib.lbm_ref_set_drive_axis(self._h, term, _dp(a)))

    def set_body_state(self, body, state):
        s = np.ascontiguousarray(state, dtype=np.float64)
        assert s.size == 13
        return self._check(self._lib.lbm_ref_set_body_state(self._h, body, _dp(s)))

    def set_pop(self, pop):
        p = np.ascontiguousarray(pop, dtype=np.float64).reshape(-1)
        assert p.size == 19 * self.cells
        return self._check(self._lib.lbm_ref_set_pop(self._h, _dp(p)))

    def step(self, n=1):
        return self._check(self._lib.lbm_ref_step(self._h, int(n)))

    def average_begin(self):
        return self._check(self._lib.lbm_ref_average_begin(self._h))

    def average(self):
        """(mean velocity [3, nz, ny, nx] since average_begin, steps averaged)."""
        out = np.zeros((3,) + self.shape)
        n = ctypes.c_long()
        self._check(self._lib.lbm_ref_average_get(self._h, _dp(out), ctypes.byref(n)))
        return out, int(n.value)

    @property
    def steps_done(self):
        return int(self._lib.lbm_ref_steps_done(self._h))

    def bodies(self):
        out = np.zeros((self.nbodies, 13))
        self._check(self._lib.lbm_ref_get_bodies(self._h, _dp(out)))
        return out

    def body_props(self, b):
        """(volume, I1, I2, I3) of body b, principal moments in the body frame."""
        out = np.zeros(4)
        self._check(self._lib.lbm_ref_body_props(self._h, int(b), _dp(out)))
        return out

    def forces(self):
        out = np.zeros((self.nbodies, 6))
        self._check(self._lib.lbm_ref_get_forces(self._h, _dp(out)))
        return out

    def field(self, what):
        nz, ny, nx = self.shape
        if what == FIELD_RHO:
            out = np.zeros((nz, ny, nx))
        elif what == FIELD_U:
            out = np.zeros((3, nz, ny, nx))
        elif what == FIELD_FLAGS:
            out = np.zeros((nz, ny, nx), dtype=np.uint8)
        elif what == FIELD_POP:
            out = np.zeros((19, nz, ny, nx))
        else:
            raise ValueError(what)
        self._check(self._lib.lbm_ref_get_fields(self._h, int(what), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def adjoint(self, n, seed):
        """Advance n steps and return the gradient of sum(seed * final body
        states) (seed: nbodies x 13) as a dict: ``state``, ``prev``, ``pop``,
        ``drive`` (nd x 2: amp, phase), ``spring`` (ns x 3: k, rest,
        damping), ``body`` (nb x 5: mass, I1, I2, I3, volume)."""
        sd = np.ascontiguousarray(seed, dtype=np.float64).reshape(self.nbodies, 13)
        nz, ny, nx = self.shape
        out = {"state": np.zeros((self.nbodies, 13)), "prev": np.zeros((self.nbodies, 13)),
               "pop": np.zeros((19, nz, ny, nx)), "drive": np.zeros((self.ndrives, 2)),
               "spring": np.zeros((self.nsprings, 3)), "body": np.zeros((self.nbodies, 5))}
        ptr = [_dp(out[k]) if out[k].size else None
               for k in ("state", "prev", "pop", "drive", "spring", "body")]
        self._check(self._lib.lbm_ref_adjoint(self._h, int(n), _dp(sd), *ptr))
        return out

    @property
    def flag_digest(self):
        """Running digest of the obstacle map of every step taken so far."""
        return int(self._lib.lbm_ref_flag_digest(self._h))

    def rho(self):
        return self.field(FIELD_RHO)

    def u(self):
        return self.field(FIELD_U)

    def flags(self):
        return self.field(FIELD_FLAGS)

    def pop(self):
        return self.field(FIELD_POP)
