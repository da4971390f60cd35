"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

The oracle is a plain C solver, serial by default, of the paper's equations
(arXiv 1810.00348, Eqs. (2)-(10), Algorithm 1).  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark import this module.  It does not import
the CUDA package and the CUDA package does not import it; both take their
inputs from ``paper_1810_00348_gb300.inputs``, which holds no solver arithmetic.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_dbl_p = ctypes.POINTER(ctypes.c_double)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", _dbl_p), ("dy", _dbl_p), ("dz", _dbl_p),
        ("solid", ctypes.POINTER(ctypes.c_ubyte)),
        ("nvx", ctypes.c_int), ("nvy", ctypes.c_int), ("nvz", ctypes.c_int),
        ("xi_x", _dbl_p), ("xi_y", _dbl_p), ("xi_z", _dbl_p),
        ("w_x", _dbl_p), ("w_y", _dbl_p), ("w_z", _dbl_p),
        ("Kn", ctypes.c_double), ("Pr", ctypes.c_double), ("omega", ctypes.c_double),
        ("face_type", ctypes.c_int * 6),
        ("T_w", ctypes.c_double * 6),
        ("U_w", (ctypes.c_double * 3) * 6),
        ("rho_in", ctypes.c_double), ("U_in", ctypes.c_double * 3), ("T_in", ctypes.c_double),
        ("T_solid", ctypes.c_double),
        ("wall_mode", ctypes.c_int),
        ("mass_rescale", ctypes.c_int),
        ("q_lagged", ctypes.c_int),
        ("order", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        lib.kgso_create.restype = ctypes.c_void_p
        lib.kgso_create.argtypes = [ctypes.POINTER(_Problem), _dbl_p]
        lib.kgso_destroy.argtypes = [ctypes.c_void_p]
        lib.kgso_iterate.restype = ctypes.c_double
        lib.kgso_iterate.argtypes = [ctypes.c_void_p]
        for name in ("kgso_get_macros", "kgso_get_rho_w", "kgso_set_rho_w"):
            getattr(lib, name).argtypes = [ctypes.c_void_p, _dbl_p]
        lib.kgso_total_mass.restype = ctypes.c_double
        lib.kgso_total_mass.argtypes = [ctypes.c_void_p]
        lib.kgso_mu_ref.restype = ctypes.c_double
        lib.kgso_mu_ref.argtypes = [ctypes.c_void_p]
        lib.kgso_equilibrium.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p]
        lib.kgso_moments.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p]
        lib.kgso_sweep.argtypes = [ctypes.c_void_p, ctypes.c_int, _dbl_p]
        lib.kgso_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.kgso_pass1_range.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        lib.kgso_pass2_range.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dbl_p, _dbl_p]
        lib.kgso_parallel.restype = ctypes.c_int
        lib.kgso_ghost.restype = ctypes.c_double
        lib.kgso_ghost.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dbl_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One oracle solver state built from an ``inputs.Problem``.  ``threads``
    > 1 sweeps that many contiguous velocity ranges concurrently, with private
    sums added in range order (same arithmetic, another summation order)."""

    def __init__(self, prob, macros0=None, threads=1):
        lib = _load()
        self.prob = prob
        self._keep = []
        P = _Problem()
        P.nx, P.ny, P.nz = prob.nx, prob.ny, prob.nz
        for name in ("dx", "dy", "dz", "xi_x", "xi_y", "xi_z", "w_x", "w_y", "w_z"):
            arr = _f64(getattr(prob, name))
            self._keep.append(arr)
            setattr(P, name, _ptr(arr))
        if prob.solid is not None:
            sol = np.ascontiguousarray(np.asarray(prob.solid, dtype=np.uint8).reshape(-1))
            self._keep.append(sol)
            P.solid = sol.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        else:
            P.solid = ctypes.POINTER(ctypes.c_ubyte)()
        P.nvx, P.nvy, P.nvz = len(prob.xi_x), len(prob.xi_y), len(prob.xi_z)
        P.Kn, P.Pr, P.omega = prob.Kn, prob.Pr, prob.omega
        for f in range(6):
            P.face_type[f] = int(prob.face_type[f])
            P.T_w[f] = float(prob.T_w[f])
            for d in range(3):
                P.U_w[f][d] = float(prob.U_w[f][d])
        P.rho_in, P.T_in = prob.rho_in, prob.T_in
        for d in range(3):
            P.U_in[d] = float(prob.U_in[d])
        P.T_solid = prob.T_solid
        P.wall_mode = int(prob.wall_mode)
        P.mass_rescale = int(prob.mass_rescale)
        P.q_lagged = int(getattr(prob, "q_lagged", 0))
        P.order = int(getattr(prob, "order", 1))
        self._P = P
        m0 = None
        if macros0 is not None:
            m0 = _f64(macros0).reshape(-1)
            self._keep.append(m0)
        self._s = lib.kgso_create(ctypes.byref(P), _ptr(m0) if m0 is not None else _dbl_p())
        if not self._s:
            raise ValueError("oracle rejected the problem")
        lib.kgso_set_threads(self._s, int(threads))
        self.ncell = prob.nx * prob.ny * prob.nz
        self.nvel = P.nvx * P.nvy * P.nvz

    def __del__(self):
        if getattr(self, "_s", None):
            _load().kgso_destroy(self._s)
            self._s = None

    def pass1_range(self, a0, a1):
        """Sums of the first pass over velocities [a0, a1): rho, rho U, rho E and
        the incoming wall fluxes, as one array [1 + 3 + 1 + 6][ncell]."""
        out = np.zeros((11, self.ncell))
        lib = _load()
        lib.kgso_pass1_range(self._s, int(a0), int(a1), _ptr(out[0]), _ptr(out[1:4]), _ptr(out[4]), _ptr(out[5:11]))
        return out

    def pass2_range(self, a0, a1, U):
        """q = 1/2 sum w c |c|^2 f over velocities [a0, a1), c = xi - U, as [3][ncell]."""
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(3, self.ncell)
        out = np.zeros((3, self.ncell))
        _load().kgso_pass2_range(self._s, int(a0), int(a1), _ptr(U), _ptr(out))
        return out

    def iterate(self, n=1):
        r = None
        for _ in range(n):
            r = _load().kgso_iterate(self._s)
        return r

    def macros(self):
        out = np.empty(8 * self.ncell)
        _load().kgso_get_macros(self._s, _ptr(out))
        return out.reshape(8, self.prob.nz, self.prob.ny, self.prob.nx)

    def rho_w(self):
        out = np.empty(6 * self.ncell)
        _load().kgso_get_rho_w(self._s, _ptr(out))
        return out.reshape(6, self.prob.nz, self.prob.ny, self.prob.nx)

    def set_rho_w(self, rw):
        a = _f64(rw).reshape(-1)
        _load().kgso_set_rho_w(self._s, _ptr(a))

    def total_mass(self):
        return _load().kgso_total_mass(self._s)

    def mu_ref(self):
        return _load().kgso_mu_ref(self._s)

    def equilibrium(self, mac):
        m = _f64(mac).reshape(8)
        out = np.empty(self.nvel)
        _load().kgso_equilibrium(self._s, _ptr(m), _ptr(out))
        return out

    def moments(self, f):
        fa = _f64(f).reshape(-1)
        out = np.empty(8)
        _load().kgso_moments(self._s, _ptr(fa), _ptr(out))
        return out

    def sweep(self, a):
        out = np.empty(self.ncell)
        _load().kgso_sweep(self._s, int(a), _ptr(out))
        return out.reshape(self.prob.nz, self.prob.ny, self.prob.nx)

    def ghost(self, c, face, a):
        return _load().kgso_ghost(self._s, int(c), int(face), int(a))


def parallel_build() -> bool:
    """The oracle library runs its optional velocity ranges on several threads."""
    return bool(_load().kgso_parallel())
