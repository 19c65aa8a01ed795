"""ctypes wrapper of the FP64 CPU oracle (tfkt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and
by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. Nothing in
the product path (the CUDA library and its binding) may import this module.

The oracle restates the two-fluid kinetic scheme of arXiv 2201.10132, Sec. VI
(D2Q9 solvent + D4Q25 polymer hyper-lattice, trapezoidal g-scheme) with the
Kolmogorov forcing of Sec. VII; see tfkt_oracle.c for the step and its readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfkt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtfkt_oracle.so")

NFIELDS = 12
FIELDS = ["rho_s", "psi_tot", "ux", "uy", "cxx", "cxy", "cyy", "thxx", "thxy", "thyy",
          "qrms", "vort"]
NDIAG = 8
DIAGS = ["mass_s", "mass_p", "px", "py", "ke", "enstrophy", "qrms_mean", "ey2"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tfkt_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Phys(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("q_side", ctypes.c_int32),
                ("q_radius", ctypes.c_double), ("re", ctypes.c_double), ("wi", ctypes.c_double),
                ("beta", ctypes.c_double), ("u0", ctypes.c_double),
                ("k_periods", ctypes.c_int32), ("tau2", ctypes.c_double),
                ("ell", ctypes.c_double), ("fene_b", ctypes.c_double),
                ("qe_model", ctypes.c_int32)]


class Lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("q_side", ctypes.c_int32),
                ("q_radius", ctypes.c_double), ("tau1", ctypes.c_double),
                ("tau2", ctypes.c_double), ("H", ctypes.c_double), ("kappa", ctypes.c_double),
                ("ell", ctypes.c_double), ("psi_tot", ctypes.c_double),
                ("sigma_q2", ctypes.c_double), ("a0", ctypes.c_double), ("kf", ctypes.c_double),
                ("u0", ctypes.c_double), ("nu", ctypes.c_double), ("nu_s", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("lambda_h", ctypes.c_double),
                ("fene_b", ctypes.c_double), ("qe_model", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int32)
        L.orc_map_params.argtypes = [ctypes.POINTER(_Phys), ctypes.POINTER(Lattice)]
        L.orc_map_params.restype = ctypes.c_int
        L.orc_d2q9.argtypes = [I, D, I]
        L.orc_d4q25.argtypes = [I, D, I]
        L.orc_create.argtypes = [ctypes.POINTER(Lattice)]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_nq.argtypes = [P]
        L.orc_nq.restype = ctypes.c_int32
        L.orc_q_nodes.argtypes = [P, D, D]
        L.orc_psi0.argtypes = [P, D]
        L.orc_init.argtypes = [P, D, ctypes.c_int32]
        for n in ("orc_get_g", "orc_set_g", "orc_get_gpost", "orc_set_gpost"):
            getattr(L, n).argtypes = [P, D, D]
        L.orc_set_imposed_gradient.argtypes = [P, D, ctypes.c_int32]
        L.orc_collide.argtypes = [P]
        L.orc_stream.argtypes = [P]
        L.orc_step.argtypes = [P, ctypes.c_int32]
        L.orc_fields.argtypes = [P, D, D, D]
        L.orc_diagnostics.argtypes = [P, D]
        L.orc_set_threads.argtypes = [ctypes.c_int32]
        L.orc_set_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def map_params(nx, ny, q_side, q_radius, re, wi, beta, u0, k_periods=1, tau2=0.0,
               ell=0.0, fene_b=0.0, qe_model=0) -> Lattice:
    """Physical (Re, Wi, beta, U0, grid) -> lattice parameters; ValueError if invalid.
    tau2: the momentum relaxation time (<= 0: equal to the stress relaxation time)."""
    p = _Phys(nx, ny, q_side, q_radius, re, wi, beta, u0, k_periods, tau2, ell, fene_b, qe_model)
    out = Lattice()
    if lib().orc_map_params(ctypes.byref(p), ctypes.byref(out)) != 0:
        raise ValueError("invalid physical parameters")
    return out


def d2q9():
    c = np.zeros((9, 2), np.int32)
    w = np.zeros(9)
    o = np.zeros(9, np.int32)
    lib().orc_d2q9(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                   o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return c, w, o


def d4q25():
    c = np.zeros((25, 4), np.int32)
    w = np.zeros(25)
    o = np.zeros(25, np.int32)
    lib().orc_d4q25(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                    o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return c, w, o


def set_threads(n: int) -> int:
    return int(lib().orc_set_threads(n))


class Oracle:
    """One oracle run. Arrays: g_s[ny, nx, 9], g_p[ny, nx, nq, 25]."""

    def __init__(self, lattice: Lattice):
        self.lat = lattice
        self._h = lib().orc_create(ctypes.byref(lattice))
        self.nx, self.ny = lattice.nx, lattice.ny
        self.nq = int(lib().orc_nq(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # -- tables
    def q_nodes(self):
        qx = np.zeros(self.nq)
        qy = np.zeros(self.nq)
        lib().orc_q_nodes(self._h, _dp(qx), _dp(qy))
        return qx, qy

    def psi0(self):
        p = np.zeros(self.nq)
        lib().orc_psi0(self._h, _dp(p))
        return p

    # -- state
    def init(self, perturb: np.ndarray | None = None, ic_mode: int = 0):
        if perturb is not None:
            perturb = np.ascontiguousarray(perturb, dtype=np.float64)
            assert perturb.shape == (2, self.ny, self.nx)
        lib().orc_init(self._h, _dp(perturb), ic_mode)

    def _alloc(self):
        return (np.zeros((self.ny, self.nx, 9)), np.zeros((self.ny, self.nx, self.nq, 25)))

    def get_g(self):
        gs, gp = self._alloc()
        lib().orc_get_g(self._h, _dp(gs), _dp(gp))
        return gs, gp

    def set_g(self, gs=None, gp=None):
        gs = None if gs is None else np.ascontiguousarray(gs, dtype=np.float64)
        gp = None if gp is None else np.ascontiguousarray(gp, dtype=np.float64)
        lib().orc_set_g(self._h, _dp(gs), _dp(gp))

    def get_gpost(self):
        gs, gp = self._alloc()
        lib().orc_get_gpost(self._h, _dp(gs), _dp(gp))
        return gs, gp

    def set_gpost(self, gs=None, gp=None):
        gs = None if gs is None else np.ascontiguousarray(gs, dtype=np.float64)
        gp = None if gp is None else np.ascontiguousarray(gp, dtype=np.float64)
        lib().orc_set_gpost(self._h, _dp(gs), _dp(gp))

    def impose_gradient(self, G=None):
        """G[a][b] = d_a U_b held fixed in the Q-space drift; None restores the computed one."""
        if G is None:
            lib().orc_set_imposed_gradient(self._h, None, 0)
        else:
            g = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(4))
            lib().orc_set_imposed_gradient(self._h, _dp(g), 1)

    # -- stepping
    def collide(self):
        lib().orc_collide(self._h)

    def stream(self):
        lib().orc_stream(self._h)

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    # -- observables
    def fields(self, with_psi: bool = False, with_e: bool = False):
        out = np.zeros((NFIELDS, self.ny, self.nx))
        psi = np.zeros((self.ny, self.nx, self.nq)) if with_psi else None
        e = np.zeros((2, self.ny, self.nx)) if with_e else None
        lib().orc_fields(self._h, _dp(out), _dp(psi), _dp(e))
        d = {k: out[i] for i, k in enumerate(FIELDS)}
        if with_psi:
            d["psi"] = psi
        if with_e:
            d["ex"], d["ey"] = e[0], e[1]
        return d

    def diagnostics(self):
        out = np.zeros(NDIAG)
        lib().orc_diagnostics(self._h, _dp(out))
        return dict(zip(DIAGS, out.tolist()))
