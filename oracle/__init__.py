"""Plain FP64 single-threaded CPU oracle of the thermal LBM-PIBM-DEM step.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path
(``paper_1502_01159_gb300``) never does, and the two share no code.  The
arithmetic lives in ``pibm_oracle.c`` (each step cites the equation of
Zhang et al., arXiv 1502.01159, that it follows); this module only loads it and
marshals arguments.

Parity status: the lattice (Eqs lbm2-lbm3.5, lbm9, lbm12.5), the PIBM coupling
(Eqs lbm5-lbm13), the contact search and the contact laws are pinned by the
closed-form, invariant and brute-force tests under ``tests/``.  Full-case
sedimentation trajectories are "parity unpinned" beyond those component pins
and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pibm_oracle.c")
_HDR = os.path.join(_HERE, "pibm_oracle.h")
_LIB = os.path.join(_HERE, "libpibm_oracle.so")

PERIODIC, WALL = 0, 1
ADIABATIC, ISOTHERMAL = 0, 1
SPRING_DASHPOT, HERTZ_MD = 0, 1
FIELDS = {"rho": 0, "ux": 1, "uy": 2, "uz": 3, "T": 4, "FBx": 5, "FBy": 6, "FBz": 7, "QB": 8}


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("Ra", C.c_double), ("Pr", C.c_double), ("U_c", C.c_double), ("L_c", C.c_double),
        ("T_ref", C.c_double), ("T_init", C.c_double),
        ("buoyancy", C.c_int), ("gravity_axis", C.c_int),
        ("body_force", C.c_double * 3), ("g_particle", C.c_double * 3),
        ("dem_substeps", C.c_int), ("kappa_T", C.c_double), ("cell_size", C.c_double),
        ("nu_dT", C.c_double), ("pibm", C.c_int), ("flow_q", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so cell and contact
    decisions follow the written IEEE operation order)."""
    fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if fresh and not force:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, D, I = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        sig = {
            "orc_create": (P, [C.POINTER(_Params)]),
            "orc_destroy": (None, [P]),
            "orc_set_wall": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double]),
            "orc_set_contact_law": (C.c_int, [P, C.c_int] + [C.c_double] * 7),
            "orc_set_particles": (C.c_int, [P, C.c_int, D, D, D, D, D, D, D, C.POINTER(C.c_ubyte)]),
            "orc_set_markers": (C.c_int, [P, C.c_int, D, D, D]),
            "orc_set_populations": (C.c_int, [P, D, D]),
            "orc_step": (C.c_int, [P, C.c_int]),
            "orc_read_field": (C.c_int, [P, C.c_int, D]),
            "orc_read_populations": (C.c_int, [P, D, D]),
            "orc_read_particles": (C.c_int, [P, D, D, D, D]),
            "orc_read_particle_forces": (C.c_int, [P, D, D, D]),
            "orc_read_contact_forces": (C.c_int, [P, D, D]),
            "orc_set_hydro_jacobian": (C.c_int, [P, D]),
            "orc_set_particle_model": (C.c_int, [P, C.c_int]),
            "orc_nusselt": (C.c_double, [P]),
            "orc_contacts": (C.c_int, [P, I, C.c_int]),
            "orc_contacts_bruteforce": (C.c_int, [P, I, C.c_int]),
            "orc_cells": (C.c_int, [P, I, I]),
            "orc_point_contacts": (C.c_int, [C.c_int, D, D, I, C.c_int]),
            "orc_point_cells": (C.c_int, [C.c_int, I, C.c_double, C.c_int, D, D, I, I]),
            "orc_diagnostics": (C.c_int, [P, D]),
            "orc_relaxation": (C.c_int, [P, D]),
            "orc_time": (C.c_long, [P]),
            "orc_lagrange_weights": (C.c_int, [C.c_double, C.c_int, D]),
            "orc_delta_h": (C.c_double, [C.c_double]),
            "orc_md_path": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


class Oracle:
    """One simulation held by the C oracle.  ``case`` is a workload dict (see
    ``workloads.py``): lattice, physics parameters, walls, contact law,
    particles and static markers."""

    def __init__(self, case: dict):
        self.case = case
        p = _Params()
        p.dim = case["dim"]
        p.nx, p.ny, p.nz = case["shape"]
        p.Ra, p.Pr, p.U_c, p.L_c = case["Ra"], case["Pr"], case["U_c"], case["L_c"]
        p.T_ref, p.T_init = case["T_ref"], case["T_init"]
        p.buoyancy, p.gravity_axis = int(case["buoyancy"]), case["gravity_axis"]
        p.body_force = (C.c_double * 3)(*case["body_force"])
        p.g_particle = (C.c_double * 3)(*case["g_particle"])
        p.dem_substeps = case["dem_substeps"]
        p.kappa_T, p.cell_size, p.nu_dT = case["kappa_T"], case["cell_size"], case["nu_dT"]
        p.pibm = int(case["pibm"])
        p.flow_q = int(case.get("flow_q", 0))
        self.L = lib()
        self.h = self.L.orc_create(C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the lattice description")
        self.dim = p.dim
        self.shape = (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        self.Q, self.QG = (9, 5) if self.dim == 2 else ((15, 7) if p.flow_q == 15 else (19, 7))
        for face, (kind, thermal, Tw) in enumerate(case["walls"]):
            self.L.orc_set_wall(self.h, face, kind, thermal, Tw)
        law = case.get("contact")
        if law is not None:
            self.L.orc_set_contact_law(self.h, law["law"], law["E"], law["poisson"], law["mu"],
                                       law["kn"], law["kt"], law["gamma_n"], law["gamma_t"])
        if case.get("particle_model", "resolved") == "point":
            self.L.orc_set_particle_model(self.h, 1)
        if case.get("particles") is not None:
            self.set_particles(case["particles"])
        if case.get("markers") is not None:
            m = case["markers"]
            X = _f64(m["X"], (-1, 3))
            A, T = _f64(m["A"]), _f64(m["T"])
            if self.L.orc_set_markers(self.h, len(A), _dp(X), _dp(A), _dp(T)) != 0:
                raise ValueError("oracle rejected the markers")

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    __del__ = close

    def set_contact_law(self, law, E, poisson, mu, kn, kt, gamma_n, gamma_t):
        self.L.orc_set_contact_law(self.h, int(law), float(E), float(poisson), float(mu), float(kn), float(kt),
                                   float(gamma_n), float(gamma_t))

    def set_particles(self, parts: dict):
        X = _f64(parts["X"], (-1, 3))
        n = X.shape[0]
        z3 = np.zeros((n, 3))
        U = _f64(parts.get("U", z3), (-1, 3))
        W = _f64(parts.get("W", z3), (-1, 3))
        R, rho = _f64(parts["R"]), _f64(parts["rho_p"])
        Tp = _f64(parts.get("T_p", np.zeros(n)))
        Cp = _f64(parts.get("heat_cap"))
        fixed = parts.get("fixed")
        fx = None
        if fixed is not None:
            fixed = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
            fx = fixed.ctypes.data_as(C.POINTER(C.c_ubyte))
        self._keep = (X, U, W, R, rho, Tp, Cp, fixed)
        rc = self.L.orc_set_particles(self.h, n, _dp(X), _dp(U), _dp(W), _dp(R), _dp(rho), _dp(Tp), _dp(Cp), fx)
        if rc != 0:
            raise ValueError("oracle rejected the particles")
        self.np = n

    def set_populations(self, f=None, g=None):
        f = _f64(f)
        g = _f64(g)
        self.L.orc_set_populations(self.h, _dp(f), _dp(g))

    def step(self, n: int = 1):
        self.L.orc_step(self.h, int(n))

    @property
    def t(self) -> int:
        return int(self.L.orc_time(self.h))

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.N)
        if self.L.orc_read_field(self.h, FIELDS[name], _dp(out)) != 0:
            raise ValueError(name)
        return out.reshape(self.shape)

    def populations(self):
        f = np.empty(self.Q * self.N)
        g = np.empty(self.QG * self.N)
        self.L.orc_read_populations(self.h, _dp(f), _dp(g))
        return f.reshape((self.Q,) + self.shape), g.reshape((self.QG,) + self.shape)

    def particles(self):
        n = getattr(self, "np", 0)
        X, U, W, T = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        self.L.orc_read_particles(self.h, _dp(X), _dp(U), _dp(W), _dp(T))
        return {"X": X, "U": U, "W": W, "T_p": T}

    def particle_forces(self):
        n = getattr(self, "np", 0)
        F, T, H = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        self.L.orc_read_particle_forces(self.h, _dp(F), _dp(T), _dp(H))
        return {"F": F, "T": T, "H": H}

    def set_hydro_jacobian(self, J=None):
        """n x 19 Jacobian (J_FU row-major, J_TW row-major, J_HT) or None."""
        if J is None:
            self.L.orc_set_hydro_jacobian(self.h, None)
            self._J = None
        else:
            self._J = _f64(J, (-1, 19))
            self.L.orc_set_hydro_jacobian(self.h, _dp(self._J))

    def contact_forces(self):
        n = getattr(self, "np", 0)
        F, T = np.empty((n, 3)), np.empty((n, 3))
        self.L.orc_read_contact_forces(self.h, _dp(F), _dp(T))
        return F, T

    def nusselt(self) -> float:
        return float(self.L.orc_nusselt(self.h))

    def md_path(self, n, a, Fn, ds):
        """Tangential force after each update of one contact with the
        Mindlin-Deresiewicz history (law 2), along the prescribed normal forces
        Fn[k] and displacement increments ds[k] (k x 3), contact radius a."""
        n = _f64(n)
        Fn = _f64(Fn)
        ds = _f64(ds, (-1, 3))
        out = np.zeros((len(Fn), 3))
        rc = self.L.orc_md_path(self.h, _dp(n), float(a), len(Fn), _dp(Fn), _dp(ds), _dp(out))
        if rc != 0:
            raise ValueError("the contact law is not the Mindlin-Deresiewicz history law")
        return out

    def _pairs(self, fn):
        n = fn(self.h, None, 0)
        buf = np.zeros(2 * max(n, 1), dtype=np.int32)
        fn(self.h, buf.ctypes.data_as(C.POINTER(C.c_int)), n)
        return buf[: 2 * n].reshape(n, 2)

    def contacts(self) -> np.ndarray:
        return self._pairs(self.L.orc_contacts)

    def contacts_bruteforce(self) -> np.ndarray:
        return self._pairs(self.L.orc_contacts_bruteforce)

    def cells(self):
        n = getattr(self, "np", 0)
        c = np.zeros(max(n, 1), dtype=np.int32)
        nc = np.zeros(3, dtype=np.int32)
        self.L.orc_cells(self.h, c.ctypes.data_as(C.POINTER(C.c_int)), nc.ctypes.data_as(C.POINTER(C.c_int)))
        return c[:n], tuple(int(v) for v in nc)

    def diagnostics(self) -> dict:
        out = np.empty(6)
        self.L.orc_diagnostics(self.h, _dp(out))
        return dict(zip(["mass", "heat", "ke", "min_height", "umax", "nonfinite"], out.tolist()))

    def relaxation(self) -> dict:
        out = np.empty(5)
        self.L.orc_relaxation(self.h, _dp(out))
        return dict(zip(["nu", "alpha", "tau_f", "tau_g", "buoy"], out.tolist()))


def delta_h(a: float) -> float:
    return float(lib().orc_delta_h(float(a)))


def lagrange_weights(x: float, npts: int = 4):
    w = np.empty(npts)
    base = lib().orc_lagrange_weights(float(x), int(npts), _dp(w))
    return int(base), w


def point_contacts(X, R) -> np.ndarray:
    """Brute-force contact pairs (i < j, sorted) of a bare point set."""
    X = _f64(X, (-1, 3))
    R = _f64(R)
    n = lib().orc_point_contacts(len(R), _dp(X), _dp(R), None, 0)
    buf = np.zeros(2 * max(n, 1), dtype=np.int32)
    lib().orc_point_contacts(len(R), _dp(X), _dp(R), buf.ctypes.data_as(C.POINTER(C.c_int)), n)
    return buf[: 2 * n].reshape(n, 2)


def point_cells(dim, shape, cell_size, X, R):
    """Cell of each point under the cell-grid definition shared with the library."""
    X = _f64(X, (-1, 3))
    R = _f64(R)
    nl = np.asarray(shape, dtype=np.int32)
    c = np.zeros(max(len(R), 1), dtype=np.int32)
    nc = np.zeros(3, dtype=np.int32)
    I = C.POINTER(C.c_int)
    lib().orc_point_cells(dim, nl.ctypes.data_as(I), float(cell_size), len(R), _dp(X), _dp(R),
                          c.ctypes.data_as(I), nc.ctypes.data_as(I))
    return c[: len(R)], tuple(int(v) for v in nc)
