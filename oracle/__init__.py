"""CPU FP64 oracle for the block-hydro packet task (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It never imports the CUDA library and the
CUDA library never imports it; the two share nothing but the seeded input
generators of ``paper_2507_09337_b300.workloads``, which hold none of the
scheme's arithmetic.

Contents:
  * ``oracle.c`` -- the scheme as plain per-block loops (see its header);
    wrapped here by :func:`step`, :func:`step_rk2`, :func:`stage`, :func:`dt`,
    :func:`run`, :func:`hll`, :func:`minmod`, and the two-level AMR step
    :func:`amr_step` / :func:`amr_dt` / :func:`amr_run`. Pinned by tests/test_oracle_pins.py (exact Sod solution,
    Sedov radius, conservation, symmetries, free stream, closed-form dt,
    convergence order) and tests/test_oracle_mutations.py (planted mistakes
    are caught).
  * ``exact_riemann`` -- exact Riemann solution (pinned by published Sod star
    values and integral conservation).
  * ``sedov`` -- Sedov-Taylor similarity constant (pinned by the published
    constants for gamma = 1.4 and 5/3).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import build as _build


class _OraMesh(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("nb", ctypes.c_int * 3),
        ("bs", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
    ]


def _declare(L):
    dp = ctypes.POINTER(ctypes.c_double)
    mp = ctypes.POINTER(_OraMesh)
    L.ora_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
    L.ora_minmod.restype = ctypes.c_double
    L.ora_hll.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp]
    L.ora_hll.restype = None
    L.ora_max_signal_speed.argtypes = [mp, dp]
    L.ora_max_signal_speed.restype = ctypes.c_double
    L.ora_dt.argtypes = [mp, dp]
    L.ora_dt.restype = ctypes.c_double
    L.ora_step.argtypes = [mp, dp, ctypes.c_double, dp, dp]
    L.ora_step.restype = ctypes.c_long
    L.ora_run.argtypes = [mp, dp, ctypes.c_int, dp, dp]
    L.ora_run.restype = ctypes.c_int
    L.ora_stage.argtypes = [mp, dp, dp, ctypes.c_double, dp, dp]
    L.ora_stage.restype = ctypes.c_long
    L.ora_step_rk2.argtypes = [mp, dp, ctypes.c_double, dp, dp]
    L.ora_step_rk2.restype = ctypes.c_long
    L.ora_run_scheme.argtypes = [mp, dp, ctypes.c_int, ctypes.c_int, dp, dp]
    L.ora_run_scheme.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    L.ora_amr_step.argtypes = [mp, ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
    L.ora_amr_step.restype = ctypes.c_long
    L.ora_amr_dt.argtypes = [mp, ip, ctypes.c_int, dp, dp]
    L.ora_amr_dt.restype = ctypes.c_double
    L.ora_amr_max_signal_speed.argtypes = [mp, ip, ctypes.c_int, dp, dp]
    L.ora_amr_max_signal_speed.restype = ctypes.c_double
    L.ora_set_threads.argtypes = [ctypes.c_int]
    L.ora_set_threads.restype = None
    L.ora_get_threads.argtypes = []
    L.ora_get_threads.restype = ctypes.c_int
    return L


_lib = None


def lib():
    """Load (building first if needed) the compiled oracle."""
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


@dataclass
class Mesh:
    """Uniform grid of equal blocks on the box [lo, hi] (2D: third axis unused)."""
    ndim: int
    nb: tuple
    bs: tuple
    periodic: tuple = (0, 0, 0)
    gamma: float = 1.4
    cfl: float = 0.8
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    @property
    def nvar(self) -> int:
        return self.ndim + 2

    @property
    def nblocks(self) -> int:
        return int(np.prod(self.nb))

    def shape(self) -> tuple:
        """Shape of a state array: (block, var, k, j, i)."""
        return (self.nblocks, self.nvar, self.bs[2], self.bs[1], self.bs[0])

    def c_struct(self) -> _OraMesh:
        m = _OraMesh()
        m.ndim = self.ndim
        for d in range(3):
            m.nb[d] = int(self.nb[d])
            m.bs[d] = int(self.bs[d])
            m.periodic[d] = int(self.periodic[d])
            m.lo[d] = float(self.lo[d])
            m.hi[d] = float(self.hi[d])
        m.gamma = float(self.gamma)
        m.cfl = float(self.cfl)
        return m


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check_state(mesh: Mesh, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.shape != mesh.shape():
        raise ValueError(f"state shape {U.shape} != mesh shape {mesh.shape()}")
    return U


class Variant:
    """The oracle's Python API bound to one build of oracle.c. The module-level
    functions use the default build; the mutation test binds deliberately
    broken copies of the source."""

    Mesh = Mesh

    def __init__(self, so_path: str | None = None):
        self._path = so_path
        self._L = None

    @property
    def L(self):
        if self._L is None:
            self._L = lib() if self._path is None else _declare(ctypes.CDLL(self._path))
        return self._L

    def set_threads(self, n: int) -> None:
        """OpenMP threads used by step/run (blocks are independent; results do
        not depend on the thread count)."""
        self.L.ora_set_threads(int(n))

    def get_threads(self) -> int:
        return int(self.L.ora_get_threads())

    def minmod(self, a: float, b: float) -> float:
        """minmod limiter; pinned by brute-force cases."""
        return float(self.L.ora_minmod(a, b))

    def hll(self, ndim: int, d: int, gamma: float, WL, WR) -> np.ndarray:
        """HLL flux (Davis speeds) between primitive states WL, WR along axis d;
        pinned by hand cases and by the exact Sod solution."""
        WL = np.ascontiguousarray(WL, dtype=np.float64)
        WR = np.ascontiguousarray(WR, dtype=np.float64)
        F = np.zeros(ndim + 2)
        self.L.ora_hll(ndim, d, gamma, _ptr(WL), _ptr(WR), _ptr(F))
        return F

    def max_signal_speed(self, mesh: Mesh, U: np.ndarray) -> float:
        U = _check_state(mesh, U)
        m = mesh.c_struct()
        return float(self.L.ora_max_signal_speed(ctypes.byref(m), _ptr(U)))

    def dt(self, mesh: Mesh, U: np.ndarray) -> float:
        """CFL time step of U (summed-direction rule); pinned by closed forms."""
        U = _check_state(mesh, U)
        m = mesh.c_struct()
        return float(self.L.ora_dt(ctypes.byref(m), _ptr(U)))

    def step(self, mesh: Mesh, U: np.ndarray, dt_: float):
        """One step of every block with a given dt.

        Returns (Unew, bflux, nfirst): the new state, the boundary-flux total of
        the step in cell-sum units (sum U_new = sum U - bflux up to rounding),
        and the number of cells that used the first-order fallback. Raises on a
        non-physical interior input state.
        """
        U = _check_state(mesh, U)
        Unew = np.empty_like(U)
        bf = np.zeros(mesh.nvar)
        m = mesh.c_struct()
        nf = self.L.ora_step(ctypes.byref(m), _ptr(U), float(dt_), _ptr(Unew), _ptr(bf))
        if nf < 0:
            raise FloatingPointError("non-physical interior state (rho <= 0 or p <= 0)")
        return Unew, bf, int(nf)

    def stage(self, mesh: Mesh, U: np.ndarray, dt_: float, Ubase: np.ndarray | None = None):
        """One Runge-Kutta stage with the plain MUSCL operator L (no half
        step): U + dt L(U), or with Ubase the second Heun stage
        0.5 * (Ubase + (U + dt L(U))). Returns (Unew, bflux, nfirst)."""
        U = _check_state(mesh, U)
        base = None if Ubase is None else _check_state(mesh, Ubase)
        Unew = np.empty_like(U)
        bf = np.zeros(mesh.nvar)
        m = mesh.c_struct()
        nf = self.L.ora_stage(ctypes.byref(m), _ptr(U), None if base is None else _ptr(base), float(dt_),
                              _ptr(Unew), _ptr(bf))
        if nf < 0:
            raise FloatingPointError("non-physical interior state (rho <= 0 or p <= 0)")
        return Unew, bf, int(nf)

    def step_rk2(self, mesh: Mesh, U: np.ndarray, dt_: float):
        """One Heun RK2 step (two stages of the plain MUSCL operator).
        Returns (Unew, bflux, nfirst) with sum Unew = sum U - bflux."""
        U = _check_state(mesh, U)
        Unew = np.empty_like(U)
        bf = np.zeros(mesh.nvar)
        m = mesh.c_struct()
        nf = self.L.ora_step_rk2(ctypes.byref(m), _ptr(U), float(dt_), _ptr(Unew), _ptr(bf))
        if nf < 0:
            raise FloatingPointError("non-physical interior state (rho <= 0 or p <= 0)")
        return Unew, bf, int(nf)

    def run(self, mesh: Mesh, U: np.ndarray, nsteps: int, rk2: bool = False):
        """nsteps steps (MUSCL-Hancock, or Heun RK2 when rk2), each with dt
        from the current state.

        Returns (U_final, dts, bflux_total). The input is not modified.
        """
        U = _check_state(mesh, U).copy()
        dts = np.zeros(max(nsteps, 1))
        bf = np.zeros(mesh.nvar)
        m = mesh.c_struct()
        rc = self.L.ora_run_scheme(ctypes.byref(m), _ptr(U), int(nsteps), int(bool(rk2)), _ptr(dts), _ptr(bf))
        if rc != 0:
            raise FloatingPointError("non-physical state during run")
        return U, dts[:nsteps], bf


    # ---------------------------------------------------------------- two-level AMR
    def _amr_args(self, mesh: Mesh, refined, U0: np.ndarray, U1: np.ndarray):
        U0 = _check_state(mesh, U0)
        ref = np.ascontiguousarray(refined, dtype=np.int32)
        nfine = len(ref) << mesh.ndim
        U1 = np.ascontiguousarray(U1, dtype=np.float64)
        if U1.shape != (nfine,) + mesh.shape()[1:]:
            raise ValueError(f"fine state shape {U1.shape} != {(nfine,) + mesh.shape()[1:]}")
        return U0, ref, U1

    def amr_step(self, mesh: Mesh, refined, U0: np.ndarray, U1: np.ndarray, dt_: float):
        """One two-level step with a given dt (see oracle.c, "two-level AMR"):
        mesh is the coarse level, refined the coarse block ids split into
        2^ndim fine blocks each, U0 the coarse state (all coarse blocks), U1
        the fine state [fine block][var][k][j][i]. Returns (U0new, U1new,
        nfirst); the parents of U0new are the restriction of U1new."""
        U0, ref, U1 = self._amr_args(mesh, refined, U0, U1)
        U0n, U1n = np.empty_like(U0), np.empty_like(U1)
        m = mesh.c_struct()
        ip = ref.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        nf = self.L.ora_amr_step(ctypes.byref(m), ip, len(ref), _ptr(U0), _ptr(U1), float(dt_), _ptr(U0n),
                                 _ptr(U1n))
        if nf < 0:
            raise FloatingPointError("non-physical leaf state (rho <= 0 or p <= 0)")
        return U0n, U1n, int(nf)

    def amr_dt(self, mesh: Mesh, refined, U0: np.ndarray, U1: np.ndarray) -> float:
        """CFL time step over the leaf cells of both levels."""
        U0, ref, U1 = self._amr_args(mesh, refined, U0, U1)
        m = mesh.c_struct()
        ip = ref.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        return float(self.L.ora_amr_dt(ctypes.byref(m), ip, len(ref), _ptr(U0), _ptr(U1)))

    def amr_run(self, mesh: Mesh, refined, U0: np.ndarray, U1: np.ndarray, nsteps: int):
        """nsteps two-level steps, each with the dt of its start state.
        Returns (U0, U1, dts)."""
        dts = []
        for _ in range(nsteps):
            d = self.amr_dt(mesh, refined, U0, U1)
            if not d > 0:
                raise FloatingPointError("non-physical state during an AMR run")
            U0, U1, _ = self.amr_step(mesh, refined, U0, U1, d)
            dts.append(d)
        return U0, U1, np.array(dts)


_default = Variant()
set_threads = _default.set_threads
get_threads = _default.get_threads
minmod = _default.minmod
hll = _default.hll
max_signal_speed = _default.max_signal_speed
dt = _default.dt
step = _default.step
stage = _default.stage
step_rk2 = _default.step_rk2
run = _default.run
amr_step = _default.amr_step
amr_dt = _default.amr_dt
amr_run = _default.amr_run
