"""ctypes binding of ``liblasto_poisson.so`` with the C ABI's names.

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device memory and streams come from PyTorch; pointers are passed as
plain integers.  The library must be built (``build.build()``) and a CUDA
device present: there is no CPU path, and loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

LASTO_OK, LASTO_ERR_INVALID_ARG, LASTO_ERR_GEOMETRY, LASTO_ERR_NONFINITE = 0, 1, 2, 3
LASTO_ERR_NOT_CONVERGED, LASTO_ERR_TIMEOUT, LASTO_ERR_CUDA, LASTO_ERR_NO_MEMORY = 4, 5, 6, 7
LASTO_PREC_FP64, LASTO_PREC_MIXED = 0, 1
LASTO_CYCLE_V, LASTO_CYCLE_FV, LASTO_CYCLE_PCG = 0, 1, 2
LASTO_BC_MULTIPOLE, LASTO_BC_ZERO, LASTO_BC_EXACT = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "GEOMETRY", 3: "NONFINITE", 4: "NOT_CONVERGED", 5: "TIMEOUT",
                6: "CUDA", 7: "NO_MEMORY"}

_P = ctypes.c_void_p


class lasto_config(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("max_atoms", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("precision", ctypes.c_int), ("cycle", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("rel_tol", ctypes.c_double), ("n_theta", ctypes.c_int),
                ("n_phi", ctypes.c_int), ("launch", ctypes.c_int), ("boundary", ctypes.c_int),
                ("nu_coarse", ctypes.c_int), ("nu_fine", ctypes.c_int)]


class lasto_cluster(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("pos", _P), ("Z", _P), ("R", _P), ("slater_w", _P),
                ("slater_zeta", _P), ("c_lm", _P), ("n", ctypes.c_int * 3), ("x", _P), ("y", _P), ("z", _P),
                ("centre", ctypes.c_double * 3)]


class lasto_raw_cluster(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("pos", _P), ("Z", _P), ("R", _P), ("n", ctypes.c_int * 3), ("x", _P),
                ("y", _P), ("z", _P), ("centre", ctypes.c_double * 3), ("density", _P), ("n_rad", ctypes.c_int),
                ("r_min", ctypes.c_double), ("rho00", _P)]


class lasto_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("outer", ctypes.c_int), ("guess", ctypes.c_int)]


EXPORTS = ["lasto_config_default", "lasto_poisson_create", "lasto_poisson_solve", "lasto_poisson_solve_raw",
           "lasto_op_raw_deposit", "lasto_poisson_destroy",
           "lasto_poisson_last_error", "lasto_poisson_kernel_counts", "lasto_mesh_axis", "lasto_op_sphere_params", "lasto_op_deposit",
           "lasto_op_deposit_noalloc",
           "lasto_op_multipoles", "lasto_op_boundary_fill", "lasto_op_boundary_exact", "lasto_op_apply", "lasto_op_residual", "lasto_op_smooth",
           "lasto_op_smooth_f32", "lasto_op_smooth_split_f32", "lasto_op_smooth_slab", "lasto_op_smooth_slab_f32", "lasto_op_smooth_wave_f32", "lasto_selftest_bounded_wait",
           "lasto_probe_fma", "lasto_op_restrict", "lasto_op_prolong_add", "lasto_op_coarse_solve",
           "lasto_op_project", "lasto_op_sphere_density", "lasto_op_inner_solve", "lasto_op_interstitial_hs", "lasto_guess_param_count", "lasto_poisson_set_guess",
           "lasto_poisson_tune_table", "lasto_poisson_set_tune_table", "lasto_nn_conv3d_fwd", "lasto_nn_pack_weights", "lasto_nn_conv3d_fwd_tc", "lasto_nn_conv3d_dgrad", "lasto_nn_conv3d_wgrad", "lasto_nn_conv3d_dgrad_tc", "lasto_nn_conv3d_wgrad_tc",
           "lasto_nn_relu_grad", "lasto_nn_to_bf16", "lasto_nn_copy_channels", "lasto_nn_down", "lasto_nn_up",
           "lasto_nn_mse", "lasto_nn_adam", "lasto_nn_guess_features", "lasto_nn_guess_grid"]

_lib = None

# the learned guess network's convolutions, in the order of lasto_poisson_set_guess's parameters
GUESS_LAYERS = ["e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "bta", "btb", "d3a", "d3b", "d2a", "d2b", "d1a", "d1b", "out"]
GUESS_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_pd_33.npz")


def _declare(L):
    i, d, vp = ctypes.c_int, ctypes.c_double, _P
    ip = ctypes.POINTER(ctypes.c_int)
    cfgp, clp, stp = ctypes.POINTER(lasto_config), ctypes.POINTER(lasto_cluster), ctypes.POINTER(lasto_stats)
    sig = {
        "lasto_config_default": (None, [cfgp]),
        "lasto_poisson_create": (i, [cfgp, ctypes.POINTER(vp)]),
        "lasto_poisson_solve": (i, [vp, clp, i, vp, vp, vp, stp, vp]),
        "lasto_poisson_solve_raw": (i, [vp, ctypes.POINTER(lasto_raw_cluster), i, vp, vp, vp, stp, vp]),
        "lasto_op_raw_deposit": (i, [ctypes.POINTER(lasto_raw_cluster), vp, vp, vp, vp]),
        "lasto_poisson_destroy": (None, [vp]),
        "lasto_poisson_last_error": (ctypes.c_char_p, [vp]),
        "lasto_poisson_kernel_counts": (i, [vp, ip, ip, ip]),
        "lasto_guess_param_count": (ctypes.c_size_t, []),
        "lasto_poisson_tune_table": (i, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "lasto_poisson_set_tune_table": (i, [vp, ctypes.c_char_p]),
        "lasto_poisson_set_guess": (i, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t, ctypes.POINTER(d)]),
        "lasto_mesh_axis": (i, [i, d, d, d, d, d, vp, vp, vp]),
        "lasto_op_sphere_params": (i, [clp, vp, vp, vp, vp, vp, vp]),
        "lasto_op_deposit": (i, [clp, i, vp, vp, vp, vp]),
        "lasto_op_deposit_noalloc": (i, [clp, i, vp, vp, vp, vp]),
        "lasto_op_multipoles": (i, [ip, vp, vp, vp, vp, ctypes.POINTER(d), vp, vp]),
        "lasto_op_boundary_fill": (i, [ip, vp, vp, vp, ctypes.POINTER(d), vp, vp, vp]),
        "lasto_op_boundary_exact": (i, [clp, vp, vp]),
        "lasto_op_apply": (i, [ip, vp, vp, vp, vp, vp, vp]),
        "lasto_op_residual": (i, [ip, vp, vp, vp, vp, vp, vp, vp]),
        "lasto_op_smooth": (i, [ip, vp, vp, vp, vp, vp, i, i, vp]),
        "lasto_op_smooth_f32": (i, [ip, vp, vp, vp, vp, vp, i, i, vp]),
        "lasto_op_smooth_split_f32": (i, [ip, vp, vp, vp, vp, vp, i, i, vp]),
        "lasto_op_smooth_slab": (i, [ip, vp, vp, vp, vp, vp, vp, i, i, i, ip, vp]),
        "lasto_op_smooth_slab_f32": (i, [ip, vp, vp, vp, vp, vp, vp, i, i, i, ip, vp]),
        "lasto_op_smooth_wave_f32": (i, [ip, vp, vp, vp, vp, vp, vp, i, i, i, i, vp]),
        "lasto_selftest_bounded_wait": (i, [d, vp, vp]),
        "lasto_probe_fma": (i, [i, i, i, vp, vp]),
        "lasto_op_restrict": (i, [ip, vp, vp, vp, vp, vp, vp]),
        "lasto_op_prolong_add": (i, [ip, vp, vp, vp, vp, vp, vp]),
        "lasto_op_coarse_solve": (i, [ip, vp, vp, vp, vp, vp, vp]),
        "lasto_op_project": (i, [ip, vp, vp, vp, vp, i, vp, vp, i, i, vp, vp, vp]),
        "lasto_op_sphere_density": (i, [clp, i, d, i, i, vp, vp, vp]),
        "lasto_op_inner_solve": (i, [i, vp, vp, i, d, vp, vp, vp, vp]),
        "lasto_op_interstitial_hs": (i, [ip, vp, vp, vp, i, vp, vp, i, ip, ip, ctypes.POINTER(ctypes.c_double), vp,
                                         vp, vp, i, ctypes.POINTER(lasto_hs_stats), vp]),
        "lasto_nn_conv3d_fwd": (i, [i, ip, i, i, vp, vp, vp, i, vp, i, i, vp, i, i, vp]),
        "lasto_nn_pack_weights": (i, [i, i, vp, vp, vp]),
        "lasto_nn_conv3d_fwd_tc": (i, [i, ip, i, i, vp, vp, vp, i, vp, i, i, vp, i, i, vp, vp]),
        "lasto_nn_conv3d_dgrad": (i, [i, ip, i, i, vp, vp, vp, vp, vp]),
        "lasto_nn_conv3d_wgrad": (i, [i, ip, i, i, vp, vp, vp, vp, vp, vp]),
        "lasto_nn_conv3d_dgrad_tc": (i, [i, ip, i, i, vp, vp, vp, vp, vp, vp, vp]),
        "lasto_nn_conv3d_wgrad_tc": (i, [i, ip, i, i, vp, vp, vp, vp, vp, vp, vp]),
        "lasto_nn_relu_grad": (i, [ctypes.c_size_t, vp, vp, vp, vp, vp]),
        "lasto_nn_to_bf16": (i, [ctypes.c_size_t, vp, vp, vp]),
        "lasto_nn_copy_channels": (i, [ctypes.c_size_t, i, vp, i, i, vp, i, i, i, vp]),
        "lasto_nn_down": (i, [i, ip, i, vp, vp, i, vp]),
        "lasto_nn_up": (i, [i, ip, i, vp, vp, i, i, i, vp]),
        "lasto_nn_mse": (i, [ctypes.c_size_t, vp, vp, vp, ctypes.c_float, vp, vp, vp]),
        "lasto_nn_adam": (i, [ctypes.c_size_t, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, i, vp, vp]),
        "lasto_nn_guess_features": (i, [ip, vp, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp,
                                        vp]),
        "lasto_nn_guess_grid": (i, [ip, vp, i, ctypes.c_float, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load the CUDA library; raises if it is missing or no CUDA device is visible."""
    global _lib
    if _lib is None:
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built: {_build.LIB}")
        _lib = ctypes.CDLL(_build.LIB)
        _declare(_lib)
    return _lib


def lib_path() -> str:
    return _build.LIB


# ------------------------------------------------------------------ marshalling helpers
def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors, contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _n3(n):
    return (ctypes.c_int * 3)(*[int(v) for v in n])


def _check(st, what):
    if st != LASTO_OK:
        raise RuntimeError(f"{what} failed: {STATUS_NAMES.get(st, st)}")


def lasto_config_default() -> lasto_config:
    c = lasto_config()
    load().lasto_config_default(ctypes.byref(c))
    return c


def lasto_mesh_axis(n, centre, half_width, h_min, h_max, p_max=6.0, device="cuda", stream=None, info=False):
    x = torch.empty(n, dtype=torch.float64, device=device)
    inf = torch.empty(5, dtype=torch.float64, device=device) if info else None
    st = load().lasto_mesh_axis(int(n), float(centre), float(half_width), float(h_min), float(h_max), float(p_max),
                                _ptr(x), _ptr(inf), _stream(stream))
    _check(st, "lasto_mesh_axis")
    return (x, inf) if info else x


class DeviceCluster:
    """A cluster's arrays on the device plus its mesh axes built by ``lasto_mesh_axis``."""

    def __init__(self, cl, device="cuda", stream=None, axes=None):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(device)
        self.src = cl
        self.n_atoms = int(cl.pos.shape[0])
        self.pos, self.Z, self.R = f(cl.pos), f(cl.Z), f(cl.R)
        self.w, self.zeta, self.clm = f(cl.slater_w), f(cl.slater_zeta), f(cl.c_lm)
        self.n = (int(cl.n),) * 3
        self.centre = tuple(float(c) for c in cl.centre)
        if axes is None:
            axes = [lasto_mesh_axis(cl.n, self.centre[a], cl.half_width, cl.h_min, cl.h_max, cl.p_max, device, stream)
                    for a in range(3)]
        else:
            axes = [f(a) for a in axes]
        self.x, self.y, self.z = axes

    def struct(self) -> lasto_cluster:
        c = lasto_cluster()
        c.n_atoms = self.n_atoms
        c.pos, c.Z, c.R = _ptr(self.pos), _ptr(self.Z), _ptr(self.R)
        c.slater_w, c.slater_zeta, c.c_lm = _ptr(self.w), _ptr(self.zeta), _ptr(self.clm)
        c.n = _n3(self.n)
        c.x, c.y, c.z = _ptr(self.x), _ptr(self.y), _ptr(self.z)
        c.centre = (ctypes.c_double * 3)(*self.centre)
        return c

    @property
    def N(self):
        return self.n[0] * self.n[1] * self.n[2]


class Poisson:
    """Owns one ``lasto_poisson`` handle."""

    def __init__(self, n_max=129, max_atoms=561, max_batch=1, precision=LASTO_PREC_FP64, cycle=LASTO_CYCLE_PCG,
                 nu1=4, nu2=4, max_cycles=50, rel_tol=1e-10, n_theta=16, n_phi=32, launch=0, boundary=0,
                 nu_coarse=4, nu_fine=0):
        L = load()
        cfg = lasto_config_default()
        cfg.n_max, cfg.max_atoms, cfg.max_batch = n_max, max_atoms, max_batch
        cfg.precision, cfg.cycle, cfg.nu1, cfg.nu2 = precision, cycle, nu1, nu2
        cfg.max_cycles, cfg.rel_tol, cfg.n_theta, cfg.n_phi = max_cycles, rel_tol, n_theta, n_phi
        cfg.launch = launch
        cfg.boundary = boundary
        cfg.nu_coarse = nu_coarse
        cfg.nu_fine = nu_fine
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = L.lasto_poisson_create(ctypes.byref(cfg), ctypes.byref(h))
        _check(st, "lasto_poisson_create")
        self.h = h
        self._pending = []   # (event, stats array) of solves whose stats are still to be written

    def close(self):
        if getattr(self, "h", None):
            load().lasto_poisson_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def kernel_counts(self):
        """(once per solve, per CG iteration / V-cycle, per defect-correction step) kernel launches."""
        f, it, ou = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().lasto_poisson_kernel_counts(self.h, ctypes.byref(f), ctypes.byref(it), ctypes.byref(ou)),
               "lasto_poisson_kernel_counts")
        return f.value, it.value, ou.value

    def last_error(self) -> str:
        return load().lasto_poisson_last_error(self.h).decode()

    def tune_table(self) -> str:
        """The smoother choices measured so far, one line per level shape."""
        L = load()
        n = L.lasto_poisson_tune_table(self.h, None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        L.lasto_poisson_tune_table(self.h, buf, n + 1)
        return buf.value.decode()

    def set_tune_table(self, text: str):
        st = load().lasto_poisson_set_tune_table(self.h, text.encode())
        if st != LASTO_OK:
            raise RuntimeError(f"lasto_poisson_set_tune_table failed: {STATUS_NAMES.get(st, st)}: {self.last_error()}")

    def solve_raw(self, clusters, v_lm, potential=None, guess=None, stats=True, stream=None):
        """lasto_poisson_solve_raw on RawCluster inputs (grid density + rho_00 tables)."""
        if not isinstance(clusters, (list, tuple)):
            clusters = [clusters]
        arr = (lasto_raw_cluster * len(clusters))(*[c.struct() for c in clusters])
        self._keep = (clusters, arr)
        st_arr = (lasto_stats * len(clusters))() if stats else None
        st = load().lasto_poisson_solve_raw(self.h, arr, len(clusters), _ptr(v_lm), _ptr(potential), _ptr(guess),
                                            st_arr, _stream(stream))
        if st != LASTO_OK:
            raise RuntimeError(f"lasto_poisson_solve_raw failed: {STATUS_NAMES.get(st, st)}: {self.last_error()}")
        self._hold(st_arr, stream)
        return st_arr

    def _hold(self, st_arr, stream):
        """The library writes a solve's stats into st_arr from the stream, after the solve: keep the
        array alive until that has happened (an event after the call), even if the caller drops it."""
        self._pending = [(ev, a) for ev, a in self._pending if not ev.query()]
        if st_arr is not None:
            ev = torch.cuda.Event()
            ev.record(stream if stream is not None else torch.cuda.current_stream())
            self._pending.append((ev, st_arr))

    def set_guess(self, weights=GUESS_WEIGHTS):
        """Load the learned initial-guess network (an .npz of per-layer weights [27][cin][cout],
        biases and the JSON input/output scales); None removes it."""
        L = load()
        if weights is None:
            _check(L.lasto_poisson_set_guess(self.h, None, 0, None), "lasto_poisson_set_guess")
            return
        import json
        z = np.load(weights)
        flat = np.concatenate([np.concatenate([np.asarray(z[k + ".w"], dtype=np.float32).ravel(),
                                               np.asarray(z[k + ".b"], dtype=np.float32).ravel()])
                               for k in GUESS_LAYERS])
        if flat.size != L.lasto_guess_param_count():
            raise ValueError(f"guess network: {flat.size} parameters, expected {L.lasto_guess_param_count()}")
        sc = json.loads(str(z["scales"]))
        scales = (ctypes.c_double * 4)(sc["s0"], sc["s1"], sc["h_ref"], sc["out"])
        flat = np.ascontiguousarray(flat)
        st = L.lasto_poisson_set_guess(self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), flat.size, scales)
        if st != LASTO_OK:
            raise RuntimeError(f"lasto_poisson_set_guess failed: {STATUS_NAMES.get(st, st)}: {self.last_error()}")

    def solve(self, clusters, v_lm, potential=None, guess=None, stats=True, stream=None):
        """Enqueue one solve of the DeviceClusters; returns the host stats array (valid after sync)."""
        if not isinstance(clusters, (list, tuple)):
            clusters = [clusters]
        arr = (lasto_cluster * len(clusters))(*[c.struct() for c in clusters])
        self._keep = (clusters, arr)
        st_arr = (lasto_stats * len(clusters))() if stats else None
        st = load().lasto_poisson_solve(self.h, arr, len(clusters), _ptr(v_lm), _ptr(potential), _ptr(guess),
                                        st_arr, _stream(stream))
        if st != LASTO_OK:
            raise RuntimeError(f"lasto_poisson_solve failed: {STATUS_NAMES.get(st, st)}: {self.last_error()}")
        self._hold(st_arr, stream)
        return st_arr


# ------------------------------------------------------------------ single operations
def lasto_op_sphere_params(dc: DeviceCluster, stream=None):
    na = dc.n_atoms
    q, rhoR, drhoR = (torch.empty(na, dtype=torch.float64, device=dc.pos.device) for _ in range(3))
    coef = torch.empty((na, 3), dtype=torch.float64, device=dc.pos.device)
    status = torch.zeros(1, dtype=torch.int32, device=dc.pos.device)
    c = dc.struct()
    _check(load().lasto_op_sphere_params(ctypes.byref(c), _ptr(q), _ptr(rhoR), _ptr(drhoR), _ptr(coef),
                                         _ptr(status), _stream(stream)), "lasto_op_sphere_params")
    return q, rhoR, drhoR, coef, status


def lasto_op_deposit(dc: DeviceCluster, precision=LASTO_PREC_FP64, stream=None):
    n = dc.n
    b = torch.empty((n[2], n[1], n[0]), dtype=torch.float64, device=dc.pos.device)
    owner = torch.empty((n[2], n[1], n[0]), dtype=torch.int32, device=dc.pos.device)
    status = torch.zeros(1, dtype=torch.int32, device=dc.pos.device)
    c = dc.struct()
    _check(load().lasto_op_deposit(ctypes.byref(c), int(precision), _ptr(b), _ptr(owner), _ptr(status),
                                   _stream(stream)), "lasto_op_deposit")
    return b, owner, status


def _check_buffer(t, name, dtype, count, device):
    """A caller buffer the C ABI writes without a length: checked here, before any launch."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is required")
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name}: must live on {device}, got {t.device}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {dtype} required, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() < count:
        raise ValueError(f"{name}: at least {count} elements required, got {t.numel()}")


def lasto_op_deposit_noalloc(dc: DeviceCluster, b, owner=None, status=None, precision=LASTO_PREC_FP64, stream=None):
    """Allocation-free deposit into caller buffers: b (float64, >= N elements), optional owner
    (int32, >= N) and status (int32, >= 1, zeroed by the caller: the kernels only raise it).
    The buffers are checked here because the C entry point takes no lengths."""
    dev = dc.pos.device
    _check_buffer(b, "b", torch.float64, dc.N, dev)
    if owner is not None:
        _check_buffer(owner, "owner", torch.int32, dc.N, dev)
    if status is not None:
        _check_buffer(status, "status", torch.int32, 1, dev)
    c = dc.struct()
    _check(load().lasto_op_deposit_noalloc(ctypes.byref(c), int(precision), _ptr(b), _ptr(owner), _ptr(status),
                                           _stream(stream)), "lasto_op_deposit_noalloc")
    return b


def _axes(x, y, z):
    n = (len(x), len(y), len(z))
    return _n3(n), _ptr(x), _ptr(y), _ptr(z)


def lasto_op_multipoles(x, y, z, b, centre=(0.0, 0.0, 0.0), stream=None):
    Q = torch.empty(25, dtype=torch.float64, device=b.device)
    c = (ctypes.c_double * 3)(*centre)
    _check(load().lasto_op_multipoles(*_axes(x, y, z), _ptr(b), c, _ptr(Q), _stream(stream)), "lasto_op_multipoles")
    return Q


def lasto_op_boundary_fill(x, y, z, Q, u, centre=(0.0, 0.0, 0.0), stream=None):
    c = (ctypes.c_double * 3)(*centre)
    _check(load().lasto_op_boundary_fill(*_axes(x, y, z), c, _ptr(Q), _ptr(u), _stream(stream)),
           "lasto_op_boundary_fill")
    return u


def lasto_op_apply(x, y, z, u, stream=None):
    out = torch.empty_like(u)
    _check(load().lasto_op_apply(*_axes(x, y, z), _ptr(u), _ptr(out), _stream(stream)), "lasto_op_apply")
    return out


def lasto_op_residual(x, y, z, u, b, stream=None):
    out = torch.empty_like(u)
    _check(load().lasto_op_residual(*_axes(x, y, z), _ptr(u), _ptr(b), _ptr(out), _stream(stream)),
           "lasto_op_residual")
    return out


def lasto_op_smooth(x, y, z, u, b, sweeps=1, threads=256, stream=None):
    """`sweeps` red-black sweeps in place on u (FP64 or FP32); threads 0 = one block per row."""
    fn = load().lasto_op_smooth if u.dtype == torch.float64 else load().lasto_op_smooth_f32
    _check(fn(*_axes(x, y, z), _ptr(u), _ptr(b), int(sweeps), int(threads), _stream(stream)), "lasto_op_smooth")
    return u


SPLIT_STAGED = 1   # threads value of the plane-staged split half sweep


def lasto_op_smooth_split(x, y, z, u, b, sweeps=1, threads=256, stream=None):
    """`sweeps` FP32 red-black sweeps in place on u and b held in colour-split storage
    (split_colours); threads = SPLIT_STAGED runs the plane-staged kernel."""
    _check(load().lasto_op_smooth_split_f32(*_axes(x, y, z), _ptr(u), _ptr(b), int(sweeps), int(threads),
                                            _stream(stream)), "lasto_op_smooth_split_f32")
    return u


def split_colours(a):
    """A natural-order node array in colour-split storage: the even flat indices, then the odd ones."""
    return torch.cat([a[0::2], a[1::2]])


def merge_colours(a):
    """Inverse of split_colours."""
    h = (a.numel() + 1) // 2
    out = torch.empty_like(a)
    out[0::2] = a[:h]
    out[1::2] = a[h:]
    return out


def lasto_op_smooth_slab(x, y, z, u_in, u_out, b, sweeps=None, ns=1, first=0, tile=(32, 8, 16), stream=None):
    """`sweeps` (default ns) red-black sweeps from u_in into u_out, ns fused per pass (FP64 or FP32)."""
    fn = load().lasto_op_smooth_slab if u_in.dtype == torch.float64 else load().lasto_op_smooth_slab_f32
    sweeps = ns if sweeps is None else sweeps
    _check(fn(*_axes(x, y, z), _ptr(u_in), _ptr(u_out), _ptr(b), int(sweeps), int(ns), int(first), _n3(tile),
              _stream(stream)), "lasto_op_smooth_slab")
    return u_out


def lasto_op_smooth_wave(x, y, z, u_in, u_out, b, sweeps=1, first=0, tile=(60, 16), stream=None):
    """`sweeps` FP32 red-black sweeps from u_in into u_out as z-wavefront passes (one sweep each)."""
    _check(load().lasto_op_smooth_wave_f32(*_axes(x, y, z), _ptr(u_in), _ptr(u_out), _ptr(b), int(sweeps), int(first),
                                           int(tile[0]), int(tile[1]), _stream(stream)),
           "lasto_op_smooth_wave_f32")
    return u_out


def lasto_selftest_bounded_wait(seconds, status, stream=None):
    """One device thread waits on an mbarrier nothing arrives at for `seconds`, then raises
    status (int32 device tensor) to LASTO_ERR_TIMEOUT."""
    _check_buffer(status, "status", torch.int32, 1, status.device)
    _check(load().lasto_selftest_bounded_wait(float(seconds), _ptr(status), _stream(stream)),
           "lasto_selftest_bounded_wait")
    return status


PROBE_FLOP_PER_THREAD_ITER = 2 * 8 * 16


def lasto_probe_fma(precision, blocks, iters, out, stream=None):
    """FMA-chain throughput probe; out: float64 (precision 0) or float32 (1) tensor of blocks*256."""
    _check_buffer(out, "out", torch.float64 if precision == 0 else torch.float32, blocks * 256, out.device)
    _check(load().lasto_probe_fma(int(precision), int(blocks), int(iters), _ptr(out), _stream(stream)),
           "lasto_probe_fma")
    return out


def lasto_op_restrict(x, y, z, r, stream=None):
    bc = torch.empty(((len(z) + 1) // 2, (len(y) + 1) // 2, (len(x) + 1) // 2), dtype=torch.float64, device=r.device)
    _check(load().lasto_op_restrict(*_axes(x, y, z), _ptr(r), _ptr(bc), _stream(stream)), "lasto_op_restrict")
    return bc


def lasto_op_prolong_add(x, y, z, ec, u, stream=None):
    _check(load().lasto_op_prolong_add(*_axes(x, y, z), _ptr(ec), _ptr(u), _stream(stream)), "lasto_op_prolong_add")
    return u


def lasto_op_coarse_solve(x, y, z, b, stream=None):
    e = torch.empty_like(b)
    _check(load().lasto_op_coarse_solve(*_axes(x, y, z), _ptr(b), _ptr(e), _stream(stream)), "lasto_op_coarse_solve")
    return e


def lasto_op_project(x, y, z, u, pos, R, n_theta=16, n_phi=32, stream=None):
    na = int(R.shape[0])
    vlm = torch.empty((na, 25), dtype=torch.float64, device=u.device)
    status = torch.zeros(1, dtype=torch.int32, device=u.device)
    _check(load().lasto_op_project(*_axes(x, y, z), _ptr(u), na, _ptr(pos), _ptr(R), int(n_theta), int(n_phi),
                                   _ptr(vlm), _ptr(status), _stream(stream)), "lasto_op_project")
    return vlm, status


def lasto_op_sphere_density(dc: DeviceCluster, n_rad=429, r_min=1e-5, n_theta=16, n_phi=32, stream=None):
    """rho_LM(r_j) [n_atoms][25][n_rad] inside every sphere (Eq. 3.7 at each radius)."""
    out = torch.empty((dc.n_atoms, 25, n_rad), dtype=torch.float64, device=dc.pos.device)
    status = torch.zeros(1, dtype=torch.int32, device=dc.pos.device)
    c = dc.struct()
    _check(load().lasto_op_sphere_density(ctypes.byref(c), int(n_rad), float(r_min), int(n_theta), int(n_phi),
                                          _ptr(out), _ptr(status), _stream(stream)), "lasto_op_sphere_density")
    return out, status


def lasto_op_inner_solve(R, Z, rho_lm, v_R, r_min=1e-5, stream=None):
    """V_LM(r_j) [n_atoms][25][n_rad] inside every sphere (Eq. 3.4-3.5, Dirichlet values v_R)."""
    v = torch.empty_like(rho_lm)
    _check(load().lasto_op_inner_solve(int(R.shape[0]), _ptr(R), _ptr(Z), int(rho_lm.shape[2]), float(r_min),
                                       _ptr(rho_lm), _ptr(v_R), _ptr(v), _stream(stream)), "lasto_op_inner_solve")
    return v


class lasto_hs_stats(ctypes.Structure):
    _fields_ = [("interstitial_nodes", ctypes.c_longlong), ("chunks", ctypes.c_int), ("tile", ctypes.c_int),
                ("ms_list", ctypes.c_float), ("ms_tables", ctypes.c_float), ("ms_contract", ctypes.c_float),
                ("ms_mirror", ctypes.c_float)]


# the basis of Table 1 per Pd atom: (n, l, zeta) of 4d, 5d, 5s, 5p, 6s, 6p, 4f
PD_BASIS = [(4, 2, 2.20), (5, 2, 2.60), (5, 0, 1.00), (5, 1, 1.00), (6, 0, 2.00), (6, 1, 2.00), (4, 3, 1.60)]

LASTO_HS_DEFAULT, LASTO_HS_SIMT, LASTO_HS_TENSOR = 0, 1, 2


def lasto_op_interstitial_hs(x, y, z, pos, R, V, basis=PD_BASIS, mode=LASTO_HS_DEFAULT, stream=None, stats=None):
    """(S, H) [M][M] over the nodes outside every sphere (Eq. 3.11-3.14, grid-point form);
    V the potential energy at the nodes [nz][ny][nx]; M = n_atoms * sum(2l + 1).  stats: an
    optional lasto_hs_stats filled with the node count and stage times."""
    n = (ctypes.c_int * 3)(int(x.shape[0]), int(y.shape[0]), int(z.shape[0]))
    bn = (ctypes.c_int * len(basis))(*[int(b[0]) for b in basis])
    bl = (ctypes.c_int * len(basis))(*[int(b[1]) for b in basis])
    bz = (ctypes.c_double * len(basis))(*[float(b[2]) for b in basis])
    na = int(R.shape[0])
    M = na * sum(2 * int(b[1]) + 1 for b in basis)
    S = torch.empty((M, M), dtype=torch.float64, device=x.device)
    H = torch.empty_like(S)
    _check(load().lasto_op_interstitial_hs(n, _ptr(x), _ptr(y), _ptr(z), na, _ptr(pos), _ptr(R), len(basis), bn, bl,
                                           bz, _ptr(V), _ptr(S), _ptr(H), int(mode),
                                           ctypes.byref(stats) if stats is not None else None, _stream(stream)),
           "lasto_op_interstitial_hs")
    return S, H


def lasto_op_boundary_exact(dc: DeviceCluster, u, stream=None):
    """The six faces of u set to the exact superposition of the atoms' potentials."""
    c = dc.struct()
    _check(load().lasto_op_boundary_exact(ctypes.byref(c), _ptr(u), _stream(stream)), "lasto_op_boundary_exact")
    return u


class RawCluster:
    """A raw-density input on the device: atoms, mesh axes, the electron density at every node
    and each sphere's spherical component rho_00 on the logarithmic radial mesh."""

    def __init__(self, pos, Z, R, x, y, z, centre, density, rho00, r_min=1e-5, device="cuda"):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(device) \
            if not isinstance(a, torch.Tensor) else a.contiguous()
        self.pos, self.Z, self.R = f(pos), f(Z), f(R)
        self.x, self.y, self.z = f(x), f(y), f(z)
        self.density, self.rho00 = f(density), f(rho00)
        self.centre = tuple(float(c) for c in centre)
        self.r_min = float(r_min)
        self.n_atoms = int(self.R.shape[0])
        self.n = (int(self.x.shape[0]), int(self.y.shape[0]), int(self.z.shape[0]))

    def struct(self):
        c = lasto_raw_cluster()
        c.n_atoms = self.n_atoms
        c.pos, c.Z, c.R = _ptr(self.pos), _ptr(self.Z), _ptr(self.R)
        c.n = (ctypes.c_int * 3)(*self.n)
        c.x, c.y, c.z = _ptr(self.x), _ptr(self.y), _ptr(self.z)
        c.centre = (ctypes.c_double * 3)(*self.centre)
        c.density = _ptr(self.density)
        c.n_rad = int(self.rho00.shape[1])
        c.r_min = self.r_min
        c.rho00 = _ptr(self.rho00)
        return c


def lasto_op_raw_deposit(rc: RawCluster, stream=None):
    n = rc.n[0] * rc.n[1] * rc.n[2]
    b = torch.empty(n, dtype=torch.float64, device=rc.x.device)
    owner = torch.empty(n, dtype=torch.int32, device=rc.x.device)
    status = torch.zeros(1, dtype=torch.int32, device=rc.x.device)
    c = rc.struct()
    _check(load().lasto_op_raw_deposit(ctypes.byref(c), _ptr(b), _ptr(owner), _ptr(status), _stream(stream)),
           "lasto_op_raw_deposit")
    return b, owner, status
