"""Python binding of libtfkt (include/tfkt.h): argument marshalling only.

Every step of the two-fluid kinetic scheme runs in the library's CUDA kernels.
There is no CPU fallback: if the in-tree library is missing or cannot be
loaded, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields as dc_fields

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libtfkt.so")

FP64, FP32, FP16 = 0, 1, 2
FIELDS = ["rho_s", "psi_tot", "ux", "uy", "cxx", "cxy", "cyy", "thxx", "thxy", "thyy", "qrms",
          "vort"]
KERNELS = ["moments", "step", "fused", "fixup"]
DIAGS = ["mass_s", "mass_p", "px", "py", "ke", "enstrophy", "qrms_mean", "ey2", "umax",
         "qrms_max"]
STATUS = {0: "TFKT_OK", 1: "TFKT_EINVAL", 2: "TFKT_ENOMEM", 3: "TFKT_ECUDA", 4: "TFKT_ENAN",
          5: "TFKT_ESTATE", 6: "TFKT_EIO", 7: "TFKT_ETIMEOUT"}
EINVAL, ENAN, EIO, ETIMEOUT = 1, 4, 6, 7


class TfktError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("q_side", ctypes.c_int32),
                ("q_radius", ctypes.c_double), ("re", ctypes.c_double), ("wi", ctypes.c_double),
                ("beta", ctypes.c_double), ("u0", ctypes.c_double),
                ("k_periods", ctypes.c_int32), ("tau2", ctypes.c_double),
                ("ell", ctypes.c_double), ("ic_mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("fene_b", ctypes.c_double),
                ("qe_model", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nq", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tau1", ctypes.c_double),
                ("tau2", ctypes.c_double), ("H", ctypes.c_double), ("kappa", ctypes.c_double),
                ("ell", ctypes.c_double), ("psi_tot", ctypes.c_double),
                ("sigma_q2", ctypes.c_double), ("a0", ctypes.c_double), ("kf", ctypes.c_double),
                ("nu", ctypes.c_double), ("nu_s", ctypes.c_double), ("eta_p", ctypes.c_double),
                ("lambda_h", ctypes.c_double), ("step", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t), ("pitch", ctypes.c_size_t),
                ("bytes_per_node_step", ctypes.c_size_t), ("fene_b", ctypes.c_double),
                ("qe_model", ctypes.c_int32)]


class LpmOpts(ctypes.Structure):
    """Mirror of tfkt_lpm_opts."""
    _fields_ = [("K", ctypes.c_int32), ("tile", ctypes.c_int32), ("threshold", ctypes.c_float),
                ("mode", ctypes.c_int32), ("inject_wait_timeout", ctypes.c_int32)]


LPM_NET, LPM_FROZEN = 0, 1
QE_MOMENTUM, QE_STRESS = 0, 1
MLP_IN, MLP_HID, MLP_OUT = 40, 64, 3
MLP_NWEIGHTS = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT
MLP_NPARAM = MLP_NWEIGHTS + 2 * MLP_IN + 2 * MLP_OUT


@dataclass
class Params:
    """Mirror of tfkt_params (physical description of one Kolmogorov run)."""
    nx: int
    ny: int
    q_side: int
    q_radius: float
    re: float
    wi: float
    beta: float
    u0: float = 0.05
    k_periods: int = 1
    tau2: float = 0.0
    ell: float = 0.0
    ic_mode: int = 0
    precision: int = FP64
    fene_b: float = 0.0     # 0: Hookean springs; > 0: FENE extensibility b
    qe_model: int = 0       # QE_MOMENTUM or QE_STRESS

    def _c(self) -> _Params:
        return _Params(*(getattr(self, f.name) for f in dc_fields(self)))

    @classmethod
    def from_workload(cls, w, precision: int = FP64):
        return cls(w.nx, w.ny, w.q_side, w.q_radius, w.re, w.wi, w.beta, w.u0, w.k_periods,
                   w.tau2, 0.0, w.ic_mode, precision)


_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree libtfkt.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtfkt.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, S = ctypes.c_void_p, ctypes.c_int
        D = ctypes.POINTER(ctypes.c_double)
        L.tfkt_required_bytes.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_size_t)]
        L.tfkt_create.argtypes = [ctypes.POINTER(_Params), D, P, ctypes.c_size_t, P,
                                  ctypes.POINTER(P)]
        L.tfkt_step.argtypes = [P, ctypes.c_int64]
        L.tfkt_step_profiled.argtypes = [P, ctypes.c_int64, D, ctypes.POINTER(ctypes.c_int64)]
        L.tfkt_moments.argtypes = [P, ctypes.c_uint32, P, ctypes.c_size_t, ctypes.c_int]
        L.tfkt_psi.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int]
        L.tfkt_moments_noalloc.argtypes = [ctypes.POINTER(_Params), P, ctypes.c_uint32, P,
                                           ctypes.c_size_t, P]
        L.tfkt_moments_noalloc.restype = S
        L.tfkt_diagnostics.argtypes = [P, D]
        L.tfkt_populations.argtypes = [P, D, ctypes.c_size_t]
        L.tfkt_get_info.argtypes = [P, ctypes.POINTER(_Info)]
        L.tfkt_lattice.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.tfkt_sync.argtypes = [P]
        L.tfkt_destroy.argtypes = [P]
        L.tfkt_save.argtypes = [P, ctypes.c_char_p]
        L.tfkt_load.argtypes = [P, ctypes.c_char_p]
        L.tfkt_batch_required_bytes.argtypes = [ctypes.POINTER(_Params), ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]
        L.tfkt_batch_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int32,
                                         ctypes.POINTER(D), P, ctypes.c_size_t, P,
                                         ctypes.POINTER(P)]
        L.tfkt_batch_step.argtypes = [P, ctypes.c_int64]
        L.tfkt_batch_run.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P)]
        L.tfkt_batch_destroy.argtypes = [P]
        L.tfkt_batch_tile_height.argtypes = [P, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_float)]
        L.tfkt_batch_tile_height.restype = S
        L.tfkt_batch_plan.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_float)]
        L.tfkt_batch_plan.restype = S
        for n in ("tfkt_batch_required_bytes", "tfkt_batch_create", "tfkt_batch_step",
                  "tfkt_batch_run", "tfkt_batch_destroy"):
            getattr(L, n).restype = S
        F = ctypes.POINTER(ctypes.c_float)
        L.tfkt_mlp_create.argtypes = [F, P, ctypes.POINTER(P)]
        L.tfkt_mlp_destroy.argtypes = [P]
        L.tfkt_mlp_get.argtypes = [P, F]
        L.tfkt_mlp_set.argtypes = [P, F]
        L.tfkt_mlp_forward.argtypes = [P, P, ctypes.c_int64, P]
        L.tfkt_mlp_loss_grad.argtypes = [P, P, P, ctypes.c_int64, D, P]
        L.tfkt_mlp_adam.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float]
        L.tfkt_lpm_run.argtypes = [P, P, ctypes.POINTER(LpmOpts), ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int64)]
        L.tfkt_lpm_features.argtypes = [P, ctypes.c_int32, P, P]
        L.tfkt_lpm_targets.argtypes = [P, P, P]
        for n in ("tfkt_mlp_create", "tfkt_mlp_destroy", "tfkt_mlp_get", "tfkt_mlp_set",
                  "tfkt_mlp_forward", "tfkt_mlp_loss_grad", "tfkt_mlp_adam", "tfkt_lpm_run",
                  "tfkt_lpm_features", "tfkt_lpm_targets"):
            getattr(L, n).restype = S
        L.tfkt_slab_required_bytes.argtypes = [ctypes.POINTER(_Params), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_size_t)]
        L.tfkt_slab_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int32, ctypes.c_int32, D,
                                       P, ctypes.c_size_t, P, ctypes.POINTER(P)]
        L.tfkt_slab_halo_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.tfkt_slab_halo_pack.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t, ctypes.c_int]
        L.tfkt_slab_halo_unpack.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t, ctypes.c_int]
        I32 = ctypes.POINTER(ctypes.c_int32)
        L.tfkt_slab_rows.argtypes = [P, I32, I32, I32]
        for n in ("tfkt_slab_required_bytes", "tfkt_slab_create", "tfkt_slab_halo_bytes",
                  "tfkt_slab_halo_pack", "tfkt_slab_halo_unpack", "tfkt_slab_rows"):
            getattr(L, n).restype = S
        L.tfkt_status_string.argtypes = [S]
        L.tfkt_status_string.restype = ctypes.c_char_p
        L.tfkt_last_error.restype = ctypes.c_char_p
        for n in ("tfkt_required_bytes", "tfkt_create", "tfkt_step", "tfkt_step_profiled",
                  "tfkt_moments", "tfkt_psi",
                  "tfkt_diagnostics", "tfkt_populations", "tfkt_get_info", "tfkt_lattice",
                  "tfkt_sync", "tfkt_destroy", "tfkt_save", "tfkt_load"):
            getattr(L, n).restype = S
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise TfktError(status, where, lib().tfkt_last_error().decode())


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def required_bytes(p: Params) -> int:
    n = ctypes.c_size_t()
    _check(lib().tfkt_required_bytes(ctypes.byref(p._c()), ctypes.byref(n)), "tfkt_required_bytes")
    return n.value


def lattice():
    c9 = np.zeros((9, 2), np.int32)
    c25 = np.zeros((25, 4), np.int32)
    _check(lib().tfkt_lattice(c9.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              c25.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "tfkt_lattice")
    return c9, c25


def moments_noalloc(p: Params, pops_ptr: int, mask: int, dst_ptr: int, dst_bytes: int,
                    stream: int | None = None):
    """tfkt_moments_noalloc: fields from a device population buffer into device memory,
    using the library's static scratch instead of any allocation."""
    _check(lib().tfkt_moments_noalloc(ctypes.byref(p._c()), pops_ptr, mask, dst_ptr, dst_bytes,
                                      stream), "tfkt_moments_noalloc")


def field_mask(names) -> int:
    m = 0
    for n in names:
        m |= 1 << FIELDS.index(n)
    return m


class Solver:
    """One tfkt context. workspace: optional device buffer (e.g. a torch uint8
    tensor) of at least required_bytes(params), kept alive by the solver;
    stream: optional cudaStream_t handle (int), e.g. torch's cuda_stream."""

    def __init__(self, params: Params, perturb: np.ndarray | None = None, workspace=None,
                 stream: int | None = None):
        self.params = params
        self._workspace = workspace
        if perturb is not None:
            perturb = np.ascontiguousarray(perturb, dtype=np.float64)
            assert perturb.shape == (2, params.ny, params.nx)
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr = workspace.data_ptr()
            ws_bytes = workspace.numel() * workspace.element_size()
        h = ctypes.c_void_p()
        _check(lib().tfkt_create(ctypes.byref(params._c()),
                                 None if perturb is None else _dptr(perturb), ws_ptr, ws_bytes,
                                 stream, ctypes.byref(h)), "tfkt_create")
        self._h = h
        self.info = self.get_info()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().tfkt_destroy(self._h), "tfkt_destroy")
            self._h = ctypes.c_void_p()
        self._workspace = None   # a closed context no longer keeps the caller's buffer alive

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- the C-ABI calls
    def step(self, n: int = 1):
        _check(lib().tfkt_step(self._h, int(n)), "tfkt_step")

    def step_profiled(self, n: int, kernel_ms: np.ndarray, launches: np.ndarray):
        """tfkt_step_profiled: adds per-kernel milliseconds and launch counts."""
        assert kernel_ms.dtype == np.float64 and launches.dtype == np.int64
        _check(lib().tfkt_step_profiled(self._h, int(n), _dptr(kernel_ms),
                                        launches.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "tfkt_step_profiled")

    def sync(self):
        _check(lib().tfkt_sync(self._h), "tfkt_sync")

    def save(self, path: str):
        """Checkpoint the current state to `path` (tfkt_save)."""
        _check(lib().tfkt_save(self._h, os.fsencode(path)), "tfkt_save")

    def load(self, path: str):
        """Restore a checkpoint written for the same parameters (tfkt_load)."""
        _check(lib().tfkt_load(self._h, os.fsencode(path)), "tfkt_load")

    def get_info(self) -> dict:
        i = _Info()
        _check(lib().tfkt_get_info(self._h, ctypes.byref(i)), "tfkt_get_info")
        return {k: getattr(i, k) for k, _ in _Info._fields_}

    def moments(self, names=FIELDS, out=None) -> dict:
        """Fields as float64 [ny, nx] arrays (host), or into a device buffer `out`
        (a tensor with data_ptr()) when given; returns {name: array} for host."""
        names = [n for n in FIELDS if n in names]
        mask = field_mask(names)
        ny, nx = self.params.ny, self.params.nx
        if out is not None:
            nbytes = out.numel() * out.element_size()
            _check(lib().tfkt_moments(self._h, mask, out.data_ptr(), nbytes, 1), "tfkt_moments")
            return {}
        buf = np.empty((len(names), ny, nx), np.float64)
        _check(lib().tfkt_moments(self._h, mask, buf.ctypes.data, buf.nbytes, 0), "tfkt_moments")
        return {n: buf[k] for k, n in enumerate(names)}

    def moments_into(self, mask: int, host: np.ndarray):
        _check(lib().tfkt_moments(self._h, mask, host.ctypes.data, host.nbytes, 0),
               "tfkt_moments")

    def psi(self) -> np.ndarray:
        ny, nx, nq = self.params.ny, self.params.nx, self.info["nq"]
        buf = np.empty((ny, nx, nq), np.float64)
        _check(lib().tfkt_psi(self._h, buf.ctypes.data, buf.nbytes, 0), "tfkt_psi")
        return buf

    def diagnostics(self) -> dict:
        out = np.zeros(len(DIAGS))
        _check(lib().tfkt_diagnostics(self._h, _dptr(out)), "tfkt_diagnostics")
        return dict(zip(DIAGS, out.tolist()))

    def diagnostics_into(self, out: np.ndarray):
        _check(lib().tfkt_diagnostics(self._h, _dptr(out)), "tfkt_diagnostics")

    def populations(self) -> np.ndarray:
        """Stored post-collision g' as float64 [9 + 25 nq, ny, nx]."""
        ny, nx, nq = self.params.ny, self.params.nx, self.info["nq"]
        buf = np.empty((9 + 25 * nq, ny, nx), np.float64)
        _check(lib().tfkt_populations(self._h, _dptr(buf), buf.nbytes), "tfkt_populations")
        return buf


def batch_required_bytes(runs) -> int:
    arr = (_Params * len(runs))(*[r._c() for r in runs])
    n = ctypes.c_size_t()
    _check(lib().tfkt_batch_required_bytes(arr, len(runs), ctypes.byref(n)),
           "tfkt_batch_required_bytes")
    return n.value


# ---------------------------------------------------------------- slabs in y
SLAB_GHOST = 8
SLAB_LOW, SLAB_HIGH = 0, 1


def slab_required_bytes(p: Params, ny_local: int) -> int:
    n = ctypes.c_size_t()
    _check(lib().tfkt_slab_required_bytes(ctypes.byref(p._c()), ny_local, ctypes.byref(n)),
           "tfkt_slab_required_bytes")
    return n.value


class Slab(Solver):
    """A slab of one run (tfkt_slab_*): owned global rows [y0, y0 + ny_local) plus
    SLAB_GHOST ghost rows on each side. `params` describe the whole run; the arrays
    the Solver calls return cover the slab's ny_local + 2 SLAB_GHOST local rows
    (owned rows: SLAB_GHOST ... SLAB_GHOST + ny_local - 1). perturb: the whole run's
    perturbation at the slab's local rows, [2, ny_local + 2 SLAB_GHOST, nx]."""

    def __init__(self, params: Params, y0: int, ny_local: int, perturb: np.ndarray | None = None,
                 workspace=None, stream: int | None = None):
        from dataclasses import replace
        ny_ext = ny_local + 2 * SLAB_GHOST
        self.run_params = params
        self.params = replace(params, ny=ny_ext)    # the shapes of the local arrays
        self.y0, self.ny_local = y0, ny_local
        self._workspace = workspace
        if perturb is not None:
            perturb = np.ascontiguousarray(perturb, dtype=np.float64)
            assert perturb.shape == (2, ny_ext, params.nx)
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr = workspace.data_ptr()
            ws_bytes = workspace.numel() * workspace.element_size()
        h = ctypes.c_void_p()
        _check(lib().tfkt_slab_create(ctypes.byref(params._c()), y0, ny_local,
                                      None if perturb is None else _dptr(perturb), ws_ptr,
                                      ws_bytes, stream, ctypes.byref(h)), "tfkt_slab_create")
        self._h = h
        self.info = self.get_info()

    def halo_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().tfkt_slab_halo_bytes(self._h, ctypes.byref(n)), "tfkt_slab_halo_bytes")
        return n.value

    def pack(self, side: int, ptr: int, nbytes: int, device: bool):
        _check(lib().tfkt_slab_halo_pack(self._h, side, ctypes.c_void_p(ptr), nbytes, int(device)),
               "tfkt_slab_halo_pack")

    def unpack(self, side: int, ptr: int, nbytes: int, device: bool):
        _check(lib().tfkt_slab_halo_unpack(self._h, side, ctypes.c_void_p(ptr), nbytes,
                                           int(device)), "tfkt_slab_halo_unpack")

    def rows(self):
        y0, n, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tfkt_slab_rows(self._h, ctypes.byref(y0), ctypes.byref(n), ctypes.byref(g)),
               "tfkt_slab_rows")
        return y0.value, n.value, g.value

    def owned(self, a: np.ndarray, axis: int = -2) -> np.ndarray:
        """The owned rows of a local array whose y axis is `axis` (fields [..., y, x]:
        -2; psi [y, x, q]: 0)."""
        return np.take(a, np.arange(SLAB_GHOST, SLAB_GHOST + self.ny_local), axis=axis)


class _RunView(Solver):
    """A run of a batch: the context calls of Solver, without ownership."""

    def __init__(self, handle, params):
        self.params = params
        self._workspace = None
        self._h = handle
        self.info = self.get_info()

    def close(self):
        self._h = ctypes.c_void_p()

    def step(self, n: int = 1):
        raise TfktError(1, "step", "advance a batch with Batch.step")


class Batch:
    """tfkt_batch: independent runs advanced together by one launch per kernel per step."""

    def __init__(self, runs, perturbs=None, workspace=None, stream: int | None = None):
        self.params = list(runs)
        n = len(self.params)
        arr = (_Params * n)(*[r._c() for r in self.params])
        self._perturbs = None
        pp = None
        if perturbs is not None:
            self._perturbs = [None if p is None else np.ascontiguousarray(p, dtype=np.float64)
                              for p in perturbs]
            pp = (ctypes.POINTER(ctypes.c_double) * n)(
                *[_dptr(p) if p is not None else ctypes.POINTER(ctypes.c_double)()
                  for p in self._perturbs])
        self._workspace = workspace
        ws_ptr = workspace.data_ptr() if workspace is not None else None
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        h = ctypes.c_void_p()
        _check(lib().tfkt_batch_create(arr, n, pp, ws_ptr, ws_bytes, stream, ctypes.byref(h)),
               "tfkt_batch_create")
        self._h = h

    def step(self, n: int = 1):
        _check(lib().tfkt_batch_step(self._h, int(n)), "tfkt_batch_step")

    def tile_height(self):
        """(tile height of the launch, timed ms per step at heights 4, 8, 16)."""
        ty = ctypes.c_int32()
        ms = (ctypes.c_float * 3)()
        _check(lib().tfkt_batch_tile_height(self._h, ctypes.byref(ty), ms), "tfkt_batch_tile_height")
        return int(ty.value), [float(v) for v in ms]

    def plan(self):
        """{"per_run": bool, "tile_height": int, "ms": {"4", "8", "16", "per_run": timed ms per step}}."""
        pr, ty = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 4)()
        _check(lib().tfkt_batch_plan(self._h, ctypes.byref(pr), ctypes.byref(ty), ms), "tfkt_batch_plan")
        return {"per_run": bool(pr.value), "tile_height": int(ty.value),
                "ms": dict(zip(("4", "8", "16", "per_run"), [float(v) for v in ms]))}

    def run(self, i: int) -> Solver:
        r = ctypes.c_void_p()
        _check(lib().tfkt_batch_run(self._h, int(i), ctypes.byref(r)), "tfkt_batch_run")
        return _RunView(r, self.params[i])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().tfkt_batch_destroy(self._h), "tfkt_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------- learned macro-step
def pack_mlp(W1, b1, W2, b2, W3, b3, mx, sx, mt, st) -> np.ndarray:
    """The packed FP32 parameter vector of tfkt_lpm.h."""
    parts = [np.asarray(v, dtype=np.float32).ravel() for v in (W1, b1, W2, b2, W3, b3, mx, sx, mt, st)]
    out = np.concatenate(parts)
    assert out.size == MLP_NPARAM
    return out


def unpack_mlp(v: np.ndarray) -> dict:
    shapes = [("W1", (MLP_HID, MLP_IN)), ("b1", (MLP_HID,)), ("W2", (MLP_HID, MLP_HID)),
              ("b2", (MLP_HID,)), ("W3", (MLP_OUT, MLP_HID)), ("b3", (MLP_OUT,)),
              ("mx", (MLP_IN,)), ("sx", (MLP_IN,)), ("mt", (MLP_OUT,)), ("st", (MLP_OUT,))]
    out, k = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = np.asarray(v[k:k + n], dtype=np.float32).reshape(shp)
        k += n
    return out


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """The learned macro-step's network on the device (tfkt_mlp_*). Device arrays are
    passed as integer pointers (e.g. torch.Tensor.data_ptr())."""

    def __init__(self, params: np.ndarray, stream: int | None = None):
        v = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        _check(lib().tfkt_mlp_create(_fptr(v), ctypes.c_void_p(stream or 0), ctypes.byref(h)),
               "tfkt_mlp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().tfkt_mlp_destroy(self._h), "tfkt_mlp_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self) -> np.ndarray:
        v = np.zeros(MLP_NPARAM, np.float32)
        _check(lib().tfkt_mlp_get(self._h, _fptr(v)), "tfkt_mlp_get")
        return v

    def set(self, params: np.ndarray):
        v = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().tfkt_mlp_set(self._h, _fptr(v)), "tfkt_mlp_set")

    def forward(self, X_ptr: int, n: int, Y_ptr: int):
        _check(lib().tfkt_mlp_forward(self._h, ctypes.c_void_p(X_ptr), n, ctypes.c_void_p(Y_ptr)),
               "tfkt_mlp_forward")

    def loss_grad(self, X_ptr: int, T_ptr: int, n: int, grad_ptr: int | None = None) -> float:
        loss = ctypes.c_double()
        _check(lib().tfkt_mlp_loss_grad(self._h, ctypes.c_void_p(X_ptr), ctypes.c_void_p(T_ptr), n,
                                        ctypes.byref(loss), ctypes.c_void_p(grad_ptr or 0)),
               "tfkt_mlp_loss_grad")
        return loss.value

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(lib().tfkt_mlp_adam(self._h, lr, beta1, beta2, eps), "tfkt_mlp_adam")


def lpm_run(solver: Solver, net: Mlp | None, nblocks: int, K: int = 8, tile: int = 32,
            threshold: float = 0.25, mode: int = LPM_NET, inject_wait_timeout: bool = False) -> int:
    """Run learned blocks on a solver; returns the number of tiles that fell back.
    inject_wait_timeout (tests only): the network kernel's waits run out (TFKT_ETIMEOUT)."""
    o = LpmOpts(K, tile, threshold, mode, int(inject_wait_timeout))
    flagged = ctypes.c_int64()
    _check(lib().tfkt_lpm_run(solver._h, net._h if net is not None else None, ctypes.byref(o),
                              nblocks, ctypes.byref(flagged)), "tfkt_lpm_run")
    return int(flagged.value)


def lpm_features(solver: Solver, K: int, X_ptr: int, Cdep_ptr: int):
    _check(lib().tfkt_lpm_features(solver._h, K, ctypes.c_void_p(X_ptr), ctypes.c_void_p(Cdep_ptr)),
           "tfkt_lpm_features")


def lpm_targets(solver: Solver, Cdep_ptr: int, T_ptr: int):
    _check(lib().tfkt_lpm_targets(solver._h, ctypes.c_void_p(Cdep_ptr), ctypes.c_void_p(T_ptr)),
           "tfkt_lpm_targets")
