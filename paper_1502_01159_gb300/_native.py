"""ctypes binding of libpibm.so (include/pibm.h).  Argument marshalling only:
every step of the lattice update, the coupling and the DEM runs in the CUDA
kernels of the library.  PyTorch provides the device memory (through the
allocator hook of pibm_create) and the stream."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpibm.so")

PIBM_OK, PIBM_ERR_ARG, PIBM_ERR_OOM, PIBM_ERR_CUDA, PIBM_ERR_STATE, PIBM_ERR_UNSTABLE, PIBM_ERR_TIMEOUT = range(7)
PERIODIC, WALL = 0, 1
ADIABATIC, ISOTHERMAL = 0, 1
SPRING_DASHPOT, HERTZ_MD, HERTZ_MD_HIST = 0, 1, 2
STORE_F32, STORE_F64, STORE_F16, STORE_BF16 = 0, 1, 2, 3
(TUNE_DEM_PARTICLES_PER_CTA, TUNE_LATTICE_ROW_TILES, TUNE_LATTICE_THREADS, TUNE_WIDE_INDEX, TUNE_TC_WAIT_POLLS,
 TUNE_COUPLING_THREADS, TUNE_COUPLING_ORDER, TUNE_LATTICE_PAIRS) = range(8)
STORAGE = {"f32": STORE_F32, "f64": STORE_F64, "f16": STORE_F16, "bf16": STORE_BF16}
FIELDS = {"rho": 0, "ux": 1, "uy": 2, "uz": 3, "T": 4, "FBx": 5, "FBy": 6, "FBz": 7, "QB": 8}

# every symbol include/pibm.h declares, with (restype, argtypes)
_P, _D, _I32, _U8 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
_F = C.POINTER(C.c_float)
SURROGATE_PARAMS, SURROGATE_NORM = 9691, 38
HYDRO_JACOBIAN = 19  # J_FU (9), J_TW (9), J_HT per particle


class pibm_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("storage", C.c_int),
        ("Ra", C.c_double), ("Pr", C.c_double), ("U_c", C.c_double), ("L_c", C.c_double),
        ("T_ref", C.c_double), ("T_init", C.c_double),
        ("buoyancy", C.c_int), ("gravity_axis", C.c_int),
        ("body_force", C.c_double * 3), ("g_particle", C.c_double * 3),
        ("dem_substeps", C.c_int), ("kappa_T", C.c_double), ("cell_size", C.c_double),
        ("nu_dT", C.c_double), ("pibm", C.c_int), ("flow_q", C.c_int),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class pibm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


SIGNATURES = {
    "pibm_create": (C.c_int, [C.POINTER(pibm_desc), _P, C.POINTER(pibm_allocator), C.POINTER(_P)]),
    "pibm_destroy": (C.c_int, [_P]),
    "pibm_set_wall": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double]),
    "pibm_set_contact_law": (C.c_int, [_P, C.c_int] + [C.c_double] * 7),
    "pibm_set_particles": (C.c_int, [_P, C.c_int, _D, _D, _D, _D, _D, _D, _D, _U8]),
    "pibm_set_markers": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "pibm_set_populations": (C.c_int, [_P, _D, _D]),
    "pibm_step": (C.c_int, [_P, C.c_int]),
    "pibm_read_field": (C.c_int, [_P, C.c_int, _D, C.c_size_t]),
    "pibm_read_populations": (C.c_int, [_P, _D, _D]),
    "pibm_read_particles": (C.c_int, [_P, _D, _D, _D, _D]),
    "pibm_read_particle_forces": (C.c_int, [_P, _D, _D, _D]),
    "pibm_nusselt": (C.c_int, [_P, _D]),
    "pibm_read_contacts": (C.c_int, [_P, _I32, C.c_int, C.POINTER(C.c_int)]),
    "pibm_read_cells": (C.c_int, [_P, _I32, _I32]),
    "pibm_diagnostics": (C.c_int, [_P, _D]),
    "pibm_relaxation": (C.c_int, [_P, _D]),
    "pibm_time": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "pibm_kernels_per_step": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "pibm_step_timed": (C.c_int, [_P, _D]),
    "pibm_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "pibm_save": (C.c_int, [_P, C.c_char_p]),
    "pibm_load": (C.c_int, [_P, C.c_char_p]),
    "pibm_contacts_static": (C.c_int, [_P, _P, C.c_int, C.c_int, _I32, C.c_double, _P, C.c_int, _P, _P]),
    "pibm_set_particle_model": (C.c_int, [_P, C.c_int]),
    "pibm_read_features": (C.c_int, [_P, _D]),
    "pibm_surrogate_set_params": (C.c_int, [_P, _F, _F]),
    "pibm_surrogate_get_params": (C.c_int, [_P, _F, _F]),
    "pibm_surrogate_infer": (C.c_int, [_P, _F, C.c_int, _F]),
    "pibm_surrogate_gradient": (C.c_int, [_P, _F, _F, C.c_int, _F, _D]),
    "pibm_surrogate_train": (C.c_int, [_P, _D, _D, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_uint64, _D]),
    "pibm_surrogate_enable": (C.c_int, [_P, C.c_int, C.c_double, C.c_double]),
    "pibm_surrogate_stats": (C.c_int, [_P, _D]),
    "pibm_set_hydro_jacobian": (C.c_int, [_P, _D]),
    "pibm_read_hydro_jacobian": (C.c_int, [_P, _D, C.POINTER(C.c_int)]),
    "pibm_ensemble_create": (C.c_int, [C.POINTER(pibm_desc), C.c_int, _P, C.POINTER(pibm_allocator), C.POINTER(_P)]),
    "pibm_ensemble_destroy": (C.c_int, [_P]),
    "pibm_ensemble_box": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "pibm_ensemble_step": (C.c_int, [_P, C.c_int]),
    "pibm_ensemble_kernels_per_step": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "pibm_ensemble_autotune": (C.c_int, [_P, C.c_int, _I32]),
    "pibm_ensemble_last_error": (C.c_int, [_P, C.c_char_p, C.c_size_t]),
    "pibm_status_string": (C.c_char_p, [C.c_int]),
    "pibm_last_error": (C.c_int, [_P, C.c_char_p, C.c_size_t]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpibm.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PibmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


def desc_from_case(case: dict) -> pibm_desc:
    """The C descriptor of a workload dict (see workloads.py)."""
    d = pibm_desc()
    d.dim = case["dim"]
    d.nx, d.ny, d.nz = case["shape"]
    d.storage = STORAGE[case.get("storage", "f32")]
    d.Ra, d.Pr, d.U_c, d.L_c = case["Ra"], case["Pr"], case["U_c"], case["L_c"]
    d.T_ref, d.T_init = case["T_ref"], case["T_init"]
    d.buoyancy, d.gravity_axis = int(case["buoyancy"]), case["gravity_axis"]
    d.body_force = (C.c_double * 3)(*case["body_force"])
    d.g_particle = (C.c_double * 3)(*case["g_particle"])
    d.dem_substeps = case["dem_substeps"]
    d.kappa_T, d.cell_size, d.nu_dT = case["kappa_T"], case["cell_size"], case["nu_dT"]
    d.pibm = int(case["pibm"])
    d.flow_q = int(case.get("flow_q", 0))
    return d


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator.  Each
    allocation is a uint8 CUDA tensor kept alive until the library frees it."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = pibm_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports PIBM_ERR_OOM
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _do_free(self, ptr, user):
        self.live.pop(ptr, None)


class Simulation:
    """One library context built from a workload dict (see workloads.py).

    Method names follow the C ABI without the ``pibm_`` prefix.  With
    ``use_torch=True`` (default) device memory comes from PyTorch and the
    work is ordered on a dedicated torch CUDA stream."""

    def __init__(self, case: dict, use_torch: bool = True, device: int = 0, _handle=None):
        self.L = load()
        self.case = case
        d = desc_from_case(case)
        self.desc = d
        self.dim = d.dim
        self.shape = (d.nz, d.ny, d.nx)
        self.N = d.nx * d.ny * d.nz
        self.Q, self.QG = (9, 5) if self.dim == 2 else ((15, 7) if d.flow_q == 15 else (19, 7))
        self.np = 0
        self.allocator = None
        self.stream = None
        self._owned = _handle is None
        if _handle is not None:  # a box of an ensemble: the ensemble owns the context
            self.h = _handle
        else:
            stream_ptr = None
            alloc_ptr = None
            if use_torch:
                import torch
                dev = torch.device("cuda", device)
                self.stream = torch.cuda.Stream(device=dev)
                stream_ptr = C.c_void_p(self.stream.cuda_stream)
                self.allocator = TorchAllocator(dev)
                alloc_ptr = C.byref(self.allocator.struct)
            h = C.c_void_p()
            st = self.L.pibm_create(C.byref(d), stream_ptr, alloc_ptr, C.byref(h))
            if st != PIBM_OK:
                buf = C.create_string_buffer(512)
                self.L.pibm_last_error(None, buf, 512)
                raise PibmError(st, "pibm_create: " + buf.value.decode())
            self.h = h
        for face, (kind, thermal, Tw) in enumerate(case["walls"]):
            self.set_wall(face, kind, thermal, Tw)
        if case.get("particle_model", "resolved") == "point":
            self._check(self.L.pibm_set_particle_model(self.h, 1), "pibm_set_particle_model")
        law = case.get("contact")
        if law is not None:
            self.set_contact_law(law["law"], law["E"], law["poisson"], law["mu"], law["kn"], law["kt"],
                                 law["gamma_n"], law["gamma_t"])
        if case.get("particles") is not None:
            self.set_particles(case["particles"])
        if case.get("markers") is not None:
            m = case["markers"]
            self.set_markers(m["X"], m["A"], m["T"])

    # ------------------------------------------------------------ plumbing
    def _check(self, st, what):
        if st != PIBM_OK:
            buf = C.create_string_buffer(512)
            self.L.pibm_last_error(self.h, buf, 512)
            raise PibmError(st, f"{what}: {buf.value.decode()}")

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self.L.pibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ set-up
    def set_wall(self, face, kind, thermal, T_w):
        self._check(self.L.pibm_set_wall(self.h, face, kind, thermal, float(T_w)), "pibm_set_wall")

    def set_contact_law(self, law, E, poisson, mu, kn, kt, gamma_n, gamma_t):
        self._check(self.L.pibm_set_contact_law(self.h, law, E, poisson, mu, kn, kt, gamma_n, gamma_t),
                    "pibm_set_contact_law")

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
            fx = fixed.ctypes.data_as(_U8)
        st = self.L.pibm_set_particles(self.h, n, _dp(X), _dp(U), _dp(W), _dp(R), _dp(rho), _dp(Tp), _dp(Cp), fx)
        self._check(st, "pibm_set_particles")
        self.np = n

    def set_markers(self, X, A, T):
        X = _f64(X, (-1, 3))
        A, T = _f64(A), _f64(T)
        self._check(self.L.pibm_set_markers(self.h, len(A), _dp(X), _dp(A), _dp(T)), "pibm_set_markers")

    def set_populations(self, f=None, g=None):
        f, g = _f64(f), _f64(g)
        self._check(self.L.pibm_set_populations(self.h, _dp(f), _dp(g)), "pibm_set_populations")

    # ------------------------------------------------------------ stepping
    def step(self, n: int = 1):
        self._check(self.L.pibm_step(self.h, int(n)), "pibm_step")

    def step_timed(self):
        """One step (a replay of the step graph with event-record nodes); returns per-kernel-group device times in ms:
        collide-and-stream, DEM, coupling, whole step."""
        ms = np.zeros(4)
        self._check(self.L.pibm_step_timed(self.h, _dp(ms)), "pibm_step_timed")
        return dict(zip(["stream_collide", "dem", "coupling", "step"], ms.tolist()))

    # ------------------------------------------------------------ read-back
    def read_field(self, name: str, out=None) -> np.ndarray:
        """The field as (nz, ny, nx) FP64; out: optional C-contiguous float64 array
        of N elements to receive it (for instance in pinned host memory)."""
        if out is None:
            out = np.empty(self.N)
        elif out.dtype != np.float64 or out.size != self.N or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array of N elements")
        self._check(self.L.pibm_read_field(self.h, FIELDS[name], _dp(out), self.N), "pibm_read_field")
        return out.reshape(self.shape)

    def read_populations(self):
        f = np.empty(self.Q * self.N)
        g = np.empty(self.QG * self.N)
        self._check(self.L.pibm_read_populations(self.h, _dp(f), _dp(g)), "pibm_read_populations")
        return f.reshape((self.Q,) + self.shape), g.reshape((self.QG,) + self.shape)

    def read_particles(self, out=None):
        """Positions, velocities, spins (n x 3) and temperatures (n); out: optional
        dict of C-contiguous float64 arrays of those shapes to receive them."""
        n = self.np
        if out is None:
            out = {"X": np.empty((n, 3)), "U": np.empty((n, 3)), "W": np.empty((n, 3)), "T_p": np.empty(n)}
        for k, shape in (("X", (n, 3)), ("U", (n, 3)), ("W", (n, 3)), ("T_p", (n,))):
            a = out[k]
            if a.dtype != np.float64 or a.shape != shape or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"out[{k!r}] must be a C-contiguous float64 array of shape {shape}")
        self._check(self.L.pibm_read_particles(self.h, _dp(out["X"]), _dp(out["U"]), _dp(out["W"]), _dp(out["T_p"])),
                    "pibm_read_particles")
        return out

    def read_particle_forces(self):
        n = self.np
        F, T, H = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        self._check(self.L.pibm_read_particle_forces(self.h, _dp(F), _dp(T), _dp(H)), "pibm_read_particle_forces")
        return {"F": F, "T": T, "H": H}

    def nusselt(self) -> float:
        v = C.c_double()
        self._check(self.L.pibm_nusselt(self.h, C.byref(v)), "pibm_nusselt")
        return v.value

    def read_contacts(self) -> np.ndarray:
        n = C.c_int()
        self._check(self.L.pibm_read_contacts(self.h, None, 0, C.byref(n)), "pibm_read_contacts")
        buf = np.zeros(2 * max(n.value, 1), dtype=np.int32)
        self._check(self.L.pibm_read_contacts(self.h, buf.ctypes.data_as(_I32), n.value, C.byref(n)),
                    "pibm_read_contacts")
        return buf[: 2 * n.value].reshape(-1, 2)

    def read_cells(self):
        c = np.zeros(max(self.np, 1), dtype=np.int32)
        nc = np.zeros(3, dtype=np.int32)
        self._check(self.L.pibm_read_cells(self.h, c.ctypes.data_as(_I32), nc.ctypes.data_as(_I32)),
                    "pibm_read_cells")
        return c[: self.np], tuple(int(v) for v in nc)

    def diagnostics(self) -> dict:
        out = np.empty(6)
        self._check(self.L.pibm_diagnostics(self.h, _dp(out)), "pibm_diagnostics")
        return dict(zip(["mass", "heat", "ke", "min_height", "umax", "nonfinite"], out.tolist()))

    def relaxation(self) -> dict:
        out = np.empty(5)
        self._check(self.L.pibm_relaxation(self.h, _dp(out)), "pibm_relaxation")
        return dict(zip(["nu", "alpha", "tau_f", "tau_g", "buoy"], out.tolist()))

    @property
    def t(self) -> int:
        v = C.c_int64()
        self._check(self.L.pibm_time(self.h, C.byref(v)), "pibm_time")
        return v.value

    def save(self, path: str):
        self._check(self.L.pibm_save(self.h, str(path).encode()), "pibm_save")

    def load(self, path: str):
        self._check(self.L.pibm_load(self.h, str(path).encode()), "pibm_load")

    def set_tuning(self, knob: int, value: int):
        self._check(self.L.pibm_set_tuning(self.h, knob, value), "pibm_set_tuning")

    # ------------------------------------------------ learned surrogate
    def read_features(self):
        out = np.empty((self.np, 12))
        self._check(self.L.pibm_read_features(self.h, _dp(out)), "pibm_read_features")
        return out

    def surrogate_set_params(self, params, norm):
        p = np.ascontiguousarray(params, dtype=np.float32)
        q = np.ascontiguousarray(norm, dtype=np.float32)
        self._check(self.L.pibm_surrogate_set_params(self.h, p.ctypes.data_as(_F), q.ctypes.data_as(_F)),
                    "pibm_surrogate_set_params")

    def surrogate_get_params(self):
        p = np.empty(SURROGATE_PARAMS, dtype=np.float32)
        q = np.empty(SURROGATE_NORM, dtype=np.float32)
        self._check(self.L.pibm_surrogate_get_params(self.h, p.ctypes.data_as(_F), q.ctypes.data_as(_F)),
                    "pibm_surrogate_get_params")
        return p, q

    def surrogate_infer(self, Xn):
        """Standardised inputs (rows x 12) -> standardised outputs (rows x 7), tensor cores."""
        Xn = np.asarray(Xn, dtype=np.float32)
        rows = Xn.shape[0]
        inp = np.zeros((rows, 16), dtype=np.float32)
        inp[:, :12] = Xn
        out = np.empty((rows, 8), dtype=np.float32)
        self._check(self.L.pibm_surrogate_infer(self.h, inp.ctypes.data_as(_F), rows, out.ctypes.data_as(_F)),
                    "pibm_surrogate_infer")
        return out[:, :7]

    def surrogate_gradient(self, Xn, Yn):
        X = np.ascontiguousarray(Xn, dtype=np.float32)
        Y = np.ascontiguousarray(Yn, dtype=np.float32)
        g = np.empty(SURROGATE_PARAMS, dtype=np.float32)
        loss = C.c_double()
        self._check(self.L.pibm_surrogate_gradient(self.h, X.ctypes.data_as(_F), Y.ctypes.data_as(_F), X.shape[0],
                                                   g.ctypes.data_as(_F), C.byref(loss)), "pibm_surrogate_gradient")
        return g, loss.value

    def surrogate_train(self, feat, targ, epochs=10, batch=1024, lr=1e-3, seed=0):
        F = np.ascontiguousarray(feat, dtype=np.float64)
        T = np.ascontiguousarray(targ, dtype=np.float64)
        losses = np.zeros(max(epochs, 1))
        self._check(self.L.pibm_surrogate_train(self.h, _dp(F), _dp(T), F.shape[0], epochs, batch, lr, seed,
                                                _dp(losses)), "pibm_surrogate_train")
        return losses[:epochs]

    def surrogate_enable(self, on=True, bound=0.01, delta=0.25):
        self._check(self.L.pibm_surrogate_enable(self.h, int(on), float(bound), float(delta)), "pibm_surrogate_enable")

    def surrogate_stats(self):
        out = np.zeros(3)
        self._check(self.L.pibm_surrogate_stats(self.h, _dp(out)), "pibm_surrogate_stats")
        return {"on_steps": int(out[0]), "off_steps": int(out[1]), "last_error": float(out[2])}

    def set_hydro_jacobian(self, J=None):
        if J is None:
            self._check(self.L.pibm_set_hydro_jacobian(self.h, None), "pibm_set_hydro_jacobian")
        else:
            J = np.ascontiguousarray(J, dtype=np.float64).reshape(-1, HYDRO_JACOBIAN)
            self._check(self.L.pibm_set_hydro_jacobian(self.h, _dp(J)), "pibm_set_hydro_jacobian")

    def read_hydro_jacobian(self):
        J = np.empty((self.np, HYDRO_JACOBIAN))
        on = C.c_int()
        self._check(self.L.pibm_read_hydro_jacobian(self.h, _dp(J), C.byref(on)), "pibm_read_hydro_jacobian")
        return J, bool(on.value)

    def kernels_per_step(self) -> int:
        v = C.c_int()
        self._check(self.L.pibm_kernels_per_step(self.h, C.byref(v)), "pibm_kernels_per_step")
        return v.value


def contacts_static(X, R, dim, shape, cell_size, cap=None, stream=None):
    """pibm_contacts_static on torch CUDA tensors X (n x 3 float64) and R (n
    float64): the contact pairs computed without any device allocation by the
    library.  The output buffers are the caller's (allocated here by torch);
    returns (pairs n_pairs x 2 int32 tensor, flag)."""
    import torch
    L = load()
    n = int(R.numel())
    if cap is None:
        cap = 8 * max(n, 1)
    pairs = torch.zeros(2 * max(cap, 1), dtype=torch.int32, device=R.device)
    count = torch.zeros(2, dtype=torch.int32, device=R.device)
    nl = (C.c_int32 * 3)(*shape)
    s = stream if stream is not None else torch.cuda.current_stream(R.device)
    st = L.pibm_contacts_static(C.c_void_p(X.data_ptr()), C.c_void_p(R.data_ptr()), n, dim, nl, float(cell_size),
                                C.c_void_p(pairs.data_ptr()), cap, C.c_void_p(count.data_ptr()),
                                C.c_void_p(s.cuda_stream))
    if st != PIBM_OK:
        buf = C.create_string_buffer(512)
        L.pibm_last_error(None, buf, 512)
        raise PibmError(st, buf.value.decode())
    s.synchronize()
    total, flag = (int(v) for v in count.tolist())
    return pairs[: 2 * min(total, cap)].view(-1, 2), flag


class Ensemble:
    """Independent boxes advanced together, one graph launch per step
    (pibm_ensemble_*).  ``boxes[b]`` is a Simulation view of box b for set-up
    and read-back; the ensemble owns the contexts."""

    def __init__(self, cases, use_torch: bool = True, device: int = 0):
        self.L = load()
        n = len(cases)
        descs = (pibm_desc * n)(*[desc_from_case(c) for c in cases])
        self.allocator = None
        self.stream = None
        stream_ptr = alloc_ptr = None
        if use_torch:
            import torch
            dev = torch.device("cuda", device)
            self.stream = torch.cuda.Stream(device=dev)
            stream_ptr = C.c_void_p(self.stream.cuda_stream)
            self.allocator = TorchAllocator(dev)
            alloc_ptr = C.byref(self.allocator.struct)
        h = C.c_void_p()
        st = self.L.pibm_ensemble_create(descs, n, stream_ptr, alloc_ptr, C.byref(h))
        if st != PIBM_OK:
            buf = C.create_string_buffer(512)
            self.L.pibm_last_error(None, buf, 512)
            raise PibmError(st, "pibm_ensemble_create: " + buf.value.decode())
        self.h = h
        self.boxes = []
        for b, case in enumerate(cases):
            bh = C.c_void_p()
            self._check(self.L.pibm_ensemble_box(self.h, b, C.byref(bh)), "pibm_ensemble_box")
            self.boxes.append(Simulation(case, _handle=bh))

    def _check(self, st, what):
        if st != PIBM_OK:
            buf = C.create_string_buffer(512)
            self.L.pibm_ensemble_last_error(self.h, buf, 512)
            raise PibmError(st, f"{what}: {buf.value.decode()}")

    def step(self, n: int = 1):
        self._check(self.L.pibm_ensemble_step(self.h, int(n)), "pibm_ensemble_step")

    def autotune(self, reps: int = 2):
        """Launch shapes chosen by timing; returns [(lattice threads, row tiles,
        DEM particles per CTA)] per box (0 = default).  Advances every box
        5 reps + 16 (reps + 4) steps."""
        out = np.zeros(3 * len(self.boxes), dtype=np.int32)
        self._check(self.L.pibm_ensemble_autotune(self.h, int(reps), out.ctypes.data_as(_I32)),
                    "pibm_ensemble_autotune")
        return [tuple(int(v) for v in out[3 * b:3 * b + 3]) for b in range(len(self.boxes))]

    def kernels_per_step(self) -> int:
        n = C.c_int()
        self._check(self.L.pibm_ensemble_kernels_per_step(self.h, C.byref(n)), "pibm_ensemble_kernels_per_step")
        return n.value

    @property
    def t(self):
        return self.boxes[0].t

    def close(self):
        if getattr(self, "h", None):
            for b in self.boxes:
                b.h = None
            self.L.pibm_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
