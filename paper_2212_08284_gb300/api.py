"""Thin Python binding of libankh (include/ankh.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
kernels of libankh.so.  Functions keep the C names (ankh_create,
ankh_energy, ankh_energy_forces, ankh_destroy, ...).  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

``AnkhEnergy`` is a torch.autograd.Function whose backward scales the
gradients produced by the library's adjoint (dE/dx, dE/dq, dE/dmu,
dE/dTheta) by the incoming grad_output.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libankh.so")

ANKH_OK, ANKH_EINVAL, ANKH_ENOMEM, ANKH_ECUDA, ANKH_ETIMEOUT, ANKH_ENUMERIC, ANKH_ENOTCONV = range(7)
ANKH_INCLUDE_REC = 1
ANKH_MIXED = 2
ANKH_NONPERIODIC = 4
ANKH_FMM = 8

# buffer ids of ankh_debug_copy
BUF_PERM, BUF_START, BUF_M, BUF_RHO, BUF_PSI, BUF_SCELL, BUF_D = range(7)

EXPORTED = ["ankh_default_params", "ankh_create", "ankh_create_cached", "ankh_energy", "ankh_energy_forces",
            "ankh_energy_forces_host", "ankh_last_terms", "ankh_get_info", "ankh_debug_copy",
            "ankh_ldm", "ankh_set_timing", "ankh_stage_times", "ankh_bin_sort_noalloc", "ankh_destroy",
            "ankh_last_error", "ankh_version", "ankh_create_batch", "ankh_energy_forces_batch",
            "ankh_batch_box", "ankh_destroy_batch", "ankh_induce", "ankh_measure_fp32_peak", "ankh_debug_fft", "ankh_accuracy_rule",
            "ankh_launch_count", "ankh_batch_launch_count", "ankh_batch_set_timing", "ankh_batch_near_ms"]
STAGES = ["sort", "self", "p2m", "merge", "fft_fwd", "spectral", "corr", "near", "fft_inv", "l2p",
          "unused", "reduce"]


class AnkhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ankh error {code}: {msg}")
        self.code = code


class ankh_params(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("n_cells", ctypes.c_int), ("Lu", ctypes.c_int),
                ("Lc", ctypes.c_int), ("max_order", ctypes.c_int), ("flags", ctypes.c_uint)]


class ankh_info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("Lu", ctypes.c_int), ("Lc", ctypes.c_int),
                ("nf", ctypes.c_int), ("n_atoms", ctypes.c_int64), ("box", ctypes.c_double),
                ("h", ctypes.c_double), ("xi", ctypes.c_double), ("precompute_ms", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("tables_from_cache", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libankh.so (build it first with paper_2212_08284_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise OSError(f"{path} not found: run paper_2212_08284_gb300/build.py (nvcc, sm_103a)")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        lib.ankh_default_params.argtypes = [ctypes.POINTER(ankh_params)]
        lib.ankh_default_params.restype = None
        lib.ankh_create.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ankh_params),
                                    ctypes.POINTER(vp)]
        lib.ankh_create.restype = ctypes.c_int
        lib.ankh_create_cached.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ankh_params),
                                           ctypes.c_char_p, ctypes.POINTER(vp)]
        lib.ankh_create_cached.restype = ctypes.c_int
        lib.ankh_energy.argtypes = [vp, vp, vp, vp, vp, dp, vp]
        lib.ankh_energy.restype = ctypes.c_int
        lib.ankh_energy_forces.argtypes = [vp, vp, vp, vp, vp, dp, vp, vp, vp, vp, vp, vp]
        lib.ankh_energy_forces.restype = ctypes.c_int
        lib.ankh_energy_forces_host.argtypes = [vp, vp, vp, vp, vp, dp, vp, vp, vp, vp, vp, vp]
        lib.ankh_energy_forces_host.restype = ctypes.c_int
        lib.ankh_induce.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, vp, dp,
                                    ctypes.POINTER(ctypes.c_int), vp]
        lib.ankh_induce.restype = ctypes.c_int
        lib.ankh_last_terms.argtypes = [vp, dp]
        lib.ankh_last_terms.restype = ctypes.c_int
        lib.ankh_get_info.argtypes = [vp, ctypes.POINTER(ankh_info)]
        lib.ankh_get_info.restype = ctypes.c_int
        lib.ankh_debug_copy.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int64), vp]
        lib.ankh_debug_copy.restype = ctypes.c_int
        lib.ankh_ldm.argtypes = [vp]
        lib.ankh_ldm.restype = ctypes.c_int
        lib.ankh_set_timing.argtypes = [vp, ctypes.c_int]
        lib.ankh_set_timing.restype = ctypes.c_int
        lib.ankh_stage_times.argtypes = [vp, dp]
        lib.ankh_stage_times.restype = ctypes.c_int
        lib.ankh_bin_sort_noalloc.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, vp, vp, vp]
        lib.ankh_bin_sort_noalloc.restype = ctypes.c_int
        lib.ankh_create_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ankh_params),
                                          ctypes.POINTER(vp)]
        lib.ankh_create_batch.restype = ctypes.c_int
        lib.ankh_energy_forces_batch.argtypes = [vp, vp, vp, vp, vp, dp, vp, vp, vp, vp, vp, vp]
        lib.ankh_energy_forces_batch.restype = ctypes.c_int
        lib.ankh_batch_box.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
        lib.ankh_batch_box.restype = ctypes.c_int
        lib.ankh_launch_count.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.ankh_launch_count.restype = ctypes.c_int
        lib.ankh_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.ankh_batch_launch_count.restype = ctypes.c_int
        lib.ankh_batch_set_timing.argtypes = [vp, ctypes.c_int]
        lib.ankh_batch_set_timing.restype = ctypes.c_int
        lib.ankh_batch_near_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.ankh_batch_near_ms.restype = ctypes.c_int
        lib.ankh_destroy_batch.argtypes = [vp]
        lib.ankh_destroy_batch.restype = None
        lib.ankh_destroy.argtypes = [vp]
        lib.ankh_destroy.restype = None
        lib.ankh_last_error.argtypes = []
        lib.ankh_last_error.restype = ctypes.c_char_p
        lib.ankh_accuracy_rule.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.ankh_accuracy_rule.restype = ctypes.c_int
        lib.ankh_debug_fft.argtypes = [vp, vp, vp, ctypes.c_int, dp, vp, vp]
        lib.ankh_debug_fft.restype = ctypes.c_int
        lib.ankh_measure_fp32_peak.argtypes = [dp, dp, vp]
        lib.ankh_measure_fp32_peak.restype = ctypes.c_int
        lib.ankh_version.argtypes = []
        lib.ankh_version.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != ANKH_OK:
        raise AnkhError(rc, load_library().ankh_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ankh_default_params() -> ankh_params:
    p = ankh_params()
    load_library().ankh_default_params(ctypes.byref(p))
    return p


def ankh_create(box_edge: float, n_atoms: int, params: ankh_params | None = None) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.ankh_create(float(box_edge), int(n_atoms),
                           ctypes.byref(params) if params is not None else None, ctypes.byref(h)))
    return h


def ankh_create_cached(box_edge: float, n_atoms: int, params: ankh_params | None, cache_dir: str) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.ankh_create_cached(float(box_edge), int(n_atoms), ctypes.byref(params) if params is not None else None,
                                  os.fsencode(cache_dir), ctypes.byref(h)))
    return h


def ankh_destroy(h) -> None:
    if h:
        load_library().ankh_destroy(h)


def _check_tensor(t, shape_tail, name):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}")
    return t


def ankh_energy(h, x, q, mu=None, theta=None, stream=None) -> float:
    """Energy (e^2/A) of the box; tensors are float32 CUDA tensors."""
    _check_tensor(x, (3,), "x"); _check_tensor(mu, (3,), "mu"); _check_tensor(theta, (6,), "theta")
    E = ctypes.c_double()
    _check(load_library().ankh_energy(h, _ptr(x), _ptr(q), _ptr(mu), _ptr(theta), ctypes.byref(E),
                                      _stream_ptr(stream)))
    return E.value


def ankh_induce(h, x, q, mu, theta, alpha, mu_ind, tol: float = 1e-6, max_iter: int = 50, stream=None):
    """Induced dipoles (conjugate gradients on the ANKH field) into mu_ind
    (N x 3 float32 CUDA tensor).  Returns (E_pol, iterations)."""
    _check_tensor(x, (3,), "x"); _check_tensor(mu_ind, (3,), "mu_ind")
    E = ctypes.c_double()
    it = ctypes.c_int()
    _check(load_library().ankh_induce(h, _ptr(x), _ptr(q), _ptr(mu), _ptr(theta), _ptr(alpha), float(tol),
                                      int(max_iter), _ptr(mu_ind), ctypes.byref(E), ctypes.byref(it),
                                      _stream_ptr(stream)))
    return E.value, it.value


def ankh_energy_forces(h, x, q, mu=None, theta=None, dEdx=None, dEdq=None, dEdmu=None, dEdtheta=None,
                       torque=None, stream=None, sync: bool = True):
    """Energy and its gradient; output tensors are filled in place.  Returns E
    (float) when sync is True, else None."""
    _check_tensor(x, (3,), "x")
    E = ctypes.c_double()
    _check(load_library().ankh_energy_forces(h, _ptr(x), _ptr(q), _ptr(mu), _ptr(theta),
                                             ctypes.byref(E) if sync else None, _ptr(dEdx), _ptr(dEdq),
                                             _ptr(dEdmu), _ptr(dEdtheta), _ptr(torque), _stream_ptr(stream)))
    return E.value if sync else None


def ankh_energy_forces_host(h, x, q, mu=None, theta=None, dEdx=None, dEdq=None, dEdmu=None,
                            dEdtheta=None, torque=None, stream=None) -> float:
    """Host-buffer variant: numpy float32 arrays in and out (copies inside the call)."""
    import numpy as np

    def p(a):
        if a is None:
            return None
        assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(a.ctypes.data)

    def pt(t):
        # pinned torch CPU tensors
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    conv = (lambda a: pt(a) if hasattr(a, "data_ptr") else p(a))
    E = ctypes.c_double()
    _check(load_library().ankh_energy_forces_host(h, conv(x), conv(q), conv(mu), conv(theta),
                                                  ctypes.byref(E), conv(dEdx), conv(dEdq), conv(dEdmu),
                                                  conv(dEdtheta), conv(torque), _stream_ptr(stream)))
    return E.value


def ankh_last_terms(h):
    t = (ctypes.c_double * 6)()
    _check(load_library().ankh_last_terms(h, t))
    keys = ["near", "far", "far_k0", "correction", "self", "total"]
    return dict(zip(keys, list(t)))


def ankh_set_timing(h, enable: bool = True) -> None:
    _check(load_library().ankh_set_timing(h, 1 if enable else 0))


def ankh_stage_times(h) -> dict:
    """Per-stage device milliseconds of the last call (timing must be on)."""
    t = (ctypes.c_double * len(STAGES))()
    _check(load_library().ankh_stage_times(h, t))
    return dict(zip(STAGES, list(t)))


def ankh_accuracy_rule(n_atoms: int, Lu: int, max_order: int = 2):
    """(hmin, hmax) leaf-edge range of the accuracy table for N atoms at order
    Lu (max_order 0: charges only), or None when not calibrated."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = load_library().ankh_accuracy_rule(int(n_atoms), int(max_order), int(Lu), ctypes.byref(lo),
                                           ctypes.byref(hi))
    return (lo.value, hi.value) if rc == ANKH_OK else None


def ankh_debug_fft(h, rho, D, mode: int, out, stream=None) -> float:
    """The far-field transform step alone (tests): mode 0 forward transform of
    rho into out (complex64), mode 1 energy term (returned) and phi into out."""
    E = ctypes.c_double(0.0)
    _check(load_library().ankh_debug_fft(h, _ptr(rho), _ptr(D), int(mode), ctypes.byref(E), _ptr(out),
                                         _stream_ptr(stream)))
    return E.value


def ankh_measure_fp32_peak(stream=None) -> tuple[float, float]:
    """FP32 FMA throughput of the current device: (TFLOP/s, ms per launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ankh_measure_fp32_peak(ctypes.byref(t), ctypes.byref(ms), _stream_ptr(stream)))
    return t.value, ms.value


def ankh_bin_sort_noalloc(x, box_edge: float, n_cells: int, perm, leaf_start, stream=None) -> None:
    """Leaf binning + stable sort into caller tensors (int32 perm[N],
    leaf_start[n^3+1]) using the library's static scratch (no allocation)."""
    _check(load_library().ankh_bin_sort_noalloc(_ptr(x), int(x.shape[0]), float(box_edge), int(n_cells),
                                                _ptr(perm), _ptr(leaf_start), _stream_ptr(stream)))


def ankh_get_info(h) -> dict:
    info = ankh_info()
    _check(load_library().ankh_get_info(h, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in ankh_info._fields_}


def ankh_ldm(h) -> int:
    return int(load_library().ankh_ldm(h))


def ankh_debug_copy(h, which: int, dtype=None, stream=None):
    """Copy an internal buffer of the last call into a new CUDA tensor."""
    import torch
    nb = ctypes.c_int64()
    _check(load_library().ankh_debug_copy(h, int(which), None, ctypes.byref(nb), _stream_ptr(stream)))
    if dtype is None:
        dtype = torch.int32 if which in (BUF_PERM, BUF_START, BUF_SCELL) else torch.float32
    out = torch.empty(nb.value // 4, dtype=dtype, device="cuda")
    _check(load_library().ankh_debug_copy(h, int(which), ctypes.c_void_p(out.data_ptr()), ctypes.byref(nb),
                                          _stream_ptr(stream)))
    return out


class Ankh:
    """Owning wrapper of one handle (one cubic box, fixed N)."""

    def __init__(self, box_edge: float, n_atoms: int, xi: float = 0.01, n_cells: int = 0, Lu: int = 0,
                 Lc: int = 0, max_order: int = 2, include_rec: bool = True, mixed: bool = True,
                 nonperiodic: bool = False, fmm: bool = False, cache_dir: str | None = None):
        p = ankh_default_params()
        p.xi = xi
        p.n_cells = n_cells
        p.Lu = Lu
        p.Lc = Lc
        p.max_order = max_order
        p.flags = ((ANKH_INCLUDE_REC if include_rec else 0) | (ANKH_MIXED if mixed else 0)
                   | (ANKH_NONPERIODIC if nonperiodic else 0) | (ANKH_FMM if fmm else 0))
        self.n_atoms = int(n_atoms)
        self.box = float(box_edge)
        self.h = ankh_create_cached(box_edge, n_atoms, p, cache_dir) if cache_dir else ankh_create(box_edge, n_atoms, p)

    def close(self):
        if self.h:
            ankh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return ankh_get_info(self.h)

    def energy(self, x, q, mu=None, theta=None):
        return ankh_energy(self.h, x, q, mu, theta)

    def energy_forces(self, x, q, mu=None, theta=None, torques: bool = False):
        import torch
        n = x.shape[0]
        dev = x.device
        g = {"dEdx": torch.empty((n, 3), device=dev), "dEdq": torch.empty(n, device=dev),
             "dEdmu": torch.empty((n, 3), device=dev), "dEdtheta": torch.empty((n, 6), device=dev)}
        if torques:
            g["torque"] = torch.empty((n, 3), device=dev)
        E = ankh_energy_forces(self.h, x, q, mu, theta, **g)
        return E, g

    def terms(self):
        return ankh_last_terms(self.h)

    def induce(self, x, q, mu, theta, alpha, tol: float = 1e-6, max_iter: int = 50):
        """Induced dipoles of point polarizabilities alpha (N); returns
        (mu_ind N x 3 tensor, E_pol, iterations)."""
        import torch
        out = torch.empty((self.n_atoms, 3), device=x.device, dtype=torch.float32)
        E, it = ankh_induce(self.h, x, q, mu, theta, alpha, out, tol=tol, max_iter=max_iter)
        return out, E, it


def ankh_create_batch(box_edges, n_atoms, params: ankh_params | None = None) -> ctypes.c_void_p:
    lib = load_library()
    nb = len(box_edges)
    be = (ctypes.c_double * nb)(*[float(v) for v in box_edges])
    na = (ctypes.c_int64 * nb)(*[int(v) for v in n_atoms])
    h = ctypes.c_void_p()
    _check(lib.ankh_create_batch(nb, be, na, ctypes.byref(params) if params is not None else None,
                                 ctypes.byref(h)))
    return h


def ankh_destroy_batch(h) -> None:
    if h:
        load_library().ankh_destroy_batch(h)


def ankh_energy_forces_batch(h, nbox: int, x, q, mu=None, theta=None, dEdx=None, dEdq=None, dEdmu=None,
                             dEdtheta=None, torque=None, stream=None):
    """All boxes of a batch; arrays are concatenated in box order.  Returns a
    list of nbox energies."""
    E = (ctypes.c_double * nbox)()
    _check(load_library().ankh_energy_forces_batch(h, _ptr(x), _ptr(q), _ptr(mu), _ptr(theta), E, _ptr(dEdx),
                                                   _ptr(dEdq), _ptr(dEdmu), _ptr(dEdtheta), _ptr(torque),
                                                   _stream_ptr(stream)))
    return list(E)


def ankh_launch_count(h, forces: bool) -> int:
    """Kernels one evaluation on h launches (the library's own count)."""
    out = ctypes.c_int()
    _check(load_library().ankh_launch_count(h, 1 if forces else 0, ctypes.byref(out)))
    return int(out.value)


def ankh_batch_launch_count(b) -> int:
    """Kernels one batched evaluation launches."""
    out = ctypes.c_int()
    _check(load_library().ankh_batch_launch_count(b, ctypes.byref(out)))
    return int(out.value)


def ankh_batch_set_timing(b, enable: bool) -> None:
    _check(load_library().ankh_batch_set_timing(b, 1 if enable else 0))


def ankh_batch_near_ms(b) -> float:
    """Duration of the batched near field in the last timed batch call (ms)."""
    out = ctypes.c_double()
    _check(load_library().ankh_batch_near_ms(b, ctypes.byref(out)))
    return float(out.value)


def ankh_batch_box(h, i: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(load_library().ankh_batch_box(h, int(i), ctypes.byref(out)))
    return out


class AnkhBatch:
    """Owning wrapper of a batch of independent boxes (replicas)."""

    def __init__(self, box_edges, n_atoms, xi: float = 0.01, n_cells: int = 0, Lu: int = 0, Lc: int = 0,
                 max_order: int = 2, include_rec: bool = True, mixed: bool = True, nonperiodic: bool = False):
        p = ankh_default_params()
        p.xi, p.n_cells, p.Lu, p.Lc, p.max_order = xi, n_cells, Lu, Lc, max_order
        p.flags = ((ANKH_INCLUDE_REC if include_rec else 0) | (ANKH_MIXED if mixed else 0)
                   | (ANKH_NONPERIODIC if nonperiodic else 0))
        self.n_atoms = [int(v) for v in n_atoms]
        self.nbox = len(self.n_atoms)
        self.h = ankh_create_batch(box_edges, self.n_atoms, p)

    def close(self):
        if self.h:
            ankh_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy_forces(self, x, q, mu=None, theta=None, out=None, torques: bool = False):
        import torch
        n = x.shape[0]
        dev = x.device
        if out is None:
            out = {"dEdx": torch.empty((n, 3), device=dev), "dEdq": torch.empty(n, device=dev),
                   "dEdmu": torch.empty((n, 3), device=dev), "dEdtheta": torch.empty((n, 6), device=dev)}
            if torques:
                out["torque"] = torch.empty((n, 3), device=dev)
        E = ankh_energy_forces_batch(self.h, self.nbox, x, q, mu, theta, **out)
        return E, out


def _autograd():
    import torch

    class AnkhEnergy(torch.autograd.Function):
        """E = AnkhEnergy.apply(model, x, q, mu, theta); backward uses the exact
        adjoint computed in the same library call."""

        @staticmethod
        def forward(ctx, model, x, q, mu, theta):
            E, g = model.energy_forces(x.detach().contiguous(), q.detach().contiguous(),
                                       None if mu is None else mu.detach().contiguous(),
                                       None if theta is None else theta.detach().contiguous())
            ctx.save_for_backward(g["dEdx"], g["dEdq"], g["dEdmu"], g["dEdtheta"])
            ctx.has_mu = mu is not None
            ctx.has_theta = theta is not None
            return torch.tensor(E, dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, gout):
            gx, gq, gmu, gth = ctx.saved_tensors
            s = gout.to(torch.float32)
            return (None, gx * s, gq * s, gmu * s if ctx.has_mu else None,
                    gth * s if ctx.has_theta else None)

    return AnkhEnergy


_AE = None


def ankh_energy_autograd(model: Ankh, x, q, mu=None, theta=None):
    """Differentiable energy (torch.float64 scalar on the device)."""
    global _AE
    if _AE is None:
        _AE = _autograd()
    return _AE.apply(model, x, q, mu, theta)
