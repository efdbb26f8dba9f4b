"""FP64 classical Ewald oracle for periodic point multipoles (Python side).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path.

The quantity is the periodic multipole Coulomb energy of the paper's Eq. 1,
evaluated by Ewald summation with tin-foil boundary conditions (Sec. 3,
Eq. ewald; the reciprocal-space prefactors are restated in their standard
form because the printed ones are garbled).  See ``ewald.c`` for the formulas.

Multipole layout (10 per atom): q, mu(3), Theta(6: xx, xy, xz, yy, yz, zz).
Gradient layout (13 per atom): dE/dx(3), dE/dq, dE/dmu(3), dE/dTheta(6,
derivative with respect to the six stored entries).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald.c")
_SO = os.path.join(_HERE, "_ewald_oracle.so")
_lock = threading.Lock()
_lib = None

NMP = 10
NGR = 13


def build(force: bool = False) -> str:
    """Compile ewald.c into a shared library next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.or_version.restype = ctypes.c_int
        lib.or_bfun.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
        lib.or_pair_tensor.argtypes = [dp, dp, dp, dp, dp]
        lib.or_pair_scalar.argtypes = [dp, dp, dp, dp, dp]
        lib.or_pair_csr.argtypes = [ctypes.c_int64, dp, dp, i64p, i32p, dp, ctypes.c_double,
                                    ctypes.c_int, dp, dp, ctypes.c_int]
        lib.or_pair_csr.restype = ctypes.c_int
        lib.or_ewald_real.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, i64p, ctypes.c_int64, dp, dp,
                                      ctypes.c_int]
        lib.or_ewald_real.restype = ctypes.c_int
        lib.or_ewald_rec.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int64, dp, dp, ctypes.c_int]
        lib.or_ewald_rec.restype = ctypes.c_int
        lib.or_ewald_self.argtypes = [ctypes.c_int64, dp, ctypes.c_double, ctypes.c_double,
                                      dp, dp, dp]
        lib.or_ewald_self.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nthreads_default() -> int:
    return int(os.environ.get("ANKH_ORACLE_THREADS", os.cpu_count() or 1))


def pack_multipoles(q, mu=None, theta=None) -> np.ndarray:
    """(N,10) float64 array [q, mu, Theta6] from separate arrays."""
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    mp = np.zeros((n, NMP), dtype=np.float64)
    mp[:, 0] = q
    if mu is not None:
        mp[:, 1:4] = np.asarray(mu, dtype=np.float64)
    if theta is not None:
        mp[:, 4:10] = np.asarray(theta, dtype=np.float64)
    return mp


def bfun(r: float, a: float, lmax: int = 5) -> np.ndarray:
    lib = _load()
    out = np.zeros(lmax + 1)
    lib.or_bfun(float(r), float(a), int(lmax), _dp(out))
    return out


def pair(r, mi, mk, a: float, tensor: bool = False) -> np.ndarray:
    """One ordered pair term: [e, de/dr(3), de/dq_i, de/dmu_i(3), de/dTheta_i(6)]."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    B = bfun(float(np.linalg.norm(r)), a, 5)
    mi = np.ascontiguousarray(mi, dtype=np.float64)
    mk = np.ascontiguousarray(mk, dtype=np.float64)
    out = np.zeros(14)
    (lib.or_pair_tensor if tensor else lib.or_pair_scalar)(_dp(r), _dp(B), _dp(mi), _dp(mk), _dp(out))
    return out


def pair_csr(x, mp, rowptr, col, shift, a: float, tensor: bool = False, grad: bool = True,
             nthreads: int | None = None):
    """Sum over an ordered pair list (CSR by target).  Returns (sum e, grad N x 13)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    mp = np.ascontiguousarray(mp, dtype=np.float64)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    shift = np.ascontiguousarray(shift, dtype=np.float64)
    n = x.shape[0]
    E = np.zeros(1)
    g = np.zeros((n, NGR)) if grad else None
    rc = lib.or_pair_csr(n, _dp(x), _dp(mp), rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(shift), float(a),
                         int(tensor), _dp(E), _dp(g) if grad else ctypes.POINTER(ctypes.c_double)(),
                         nthreads or nthreads_default())
    if rc != 0:
        raise MemoryError("or_pair_csr failed")
    return float(E[0]), g


def ewald_params(box: float, n_atoms: int, tol: float = 1e-12, ratio: float = 8.0):
    """Splitting parameter alpha, real cutoff and reciprocal cutoff.

    alpha balances the real- and reciprocal-space work, alpha ~ sqrt(pi)
    (ratio * N / V^2)^(1/6) (the classic Perram/Petersen/de Leeuw optimum);
    the cutoffs follow from erfc(alpha rc) ~ exp(-s^2) = tol and
    exp(-kc^2 / 4 alpha^2) = tol (Kolafa-Perram style estimates)."""
    V = box ** 3
    s = math.sqrt(-math.log(tol))
    alpha = math.sqrt(math.pi) * (ratio * n_atoms / V ** 2) ** (1.0 / 6.0)
    # keep the real-space cutoff within a few boxes for tiny systems
    alpha = max(alpha, s / (3.0 * box))
    rc = s / alpha
    kc = 2.0 * alpha * s
    return alpha, rc, kc


def ewald(x, mp, box: float, alpha: float | None = None, rc: float | None = None,
          kc: float | None = None, tol: float = 1e-12, grad: bool = True,
          tensor: bool = False, nthreads: int | None = None) -> dict:
    """Full Ewald energy (and gradient) of a periodic multipole system.

    Returns a dict with E, E_real, E_rec, E_self, E_neut, grad (N x 13) and the
    parameters used."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    mp = np.ascontiguousarray(mp, dtype=np.float64)
    n = x.shape[0]
    a0, rc0, kc0 = ewald_params(box, n, tol)
    alpha = a0 if alpha is None else alpha
    rc = (rc0 * a0 / alpha) if rc is None else rc
    kc = (kc0 * alpha / a0) if kc is None else kc
    nt = nthreads or nthreads_default()
    g = np.zeros((n, NGR)) if grad else None
    gp = _dp(g) if grad else ctypes.POINTER(ctypes.c_double)()
    Er, Ek, Es, En = (np.zeros(1) for _ in range(4))
    null64 = ctypes.POINTER(ctypes.c_int64)()
    if lib.or_ewald_real(n, _dp(x), _dp(mp), box, alpha, rc, int(tensor), null64, 0,
                         _dp(Er), gp, nt):
        raise MemoryError("or_ewald_real failed")
    if lib.or_ewald_rec(n, _dp(x), _dp(mp), box, alpha, kc, 1, _dp(Ek), gp, nt):
        raise MemoryError("or_ewald_rec failed")
    lib.or_ewald_self(n, _dp(mp), box, alpha, _dp(Es), _dp(En), gp)
    return {"E": float(Er[0] + Ek[0] + Es[0] + En[0]), "E_real": float(Er[0]),
            "E_rec": float(Ek[0]), "E_self": float(Es[0]), "E_neut": float(En[0]),
            "grad": g, "alpha": alpha, "rc": rc, "kc": kc}


def ewald_rec_only(x, mp, box: float, alpha: float, kc: float, grad: bool = False,
                   kstride: int = 1, nthreads: int | None = None):
    """Reciprocal-space term alone (optionally every kstride-th k-vector)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    mp = np.ascontiguousarray(mp, dtype=np.float64)
    n = x.shape[0]
    g = np.zeros((n, NGR)) if grad else None
    gp = _dp(g) if grad else ctypes.POINTER(ctypes.c_double)()
    Ek = np.zeros(1)
    lib.or_ewald_rec(n, _dp(x), _dp(mp), box, alpha, kc, int(kstride), _dp(Ek), gp,
                     nthreads or nthreads_default())
    return float(Ek[0]), g


def ewald_real_rows(x, mp, box: float, alpha: float, rc: float, targets, grad: bool = False,
                    nthreads: int | None = None):
    """Real-space rows of the listed target atoms only (1/2 sum over those rows)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    mp = np.ascontiguousarray(mp, dtype=np.float64)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    n = x.shape[0]
    g = np.zeros((n, NGR)) if grad else None
    gp = _dp(g) if grad else ctypes.POINTER(ctypes.c_double)()
    Er = np.zeros(1)
    lib.or_ewald_real(n, _dp(x), _dp(mp), box, alpha, rc, 0,
                      t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), t.shape[0], _dp(Er), gp,
                      nthreads or nthreads_default())
    return float(Er[0]), g


def direct_nonperiodic(x, mp, grad: bool = True, tensor: bool = False, nthreads: int | None = None):
    """E = 1/2 sum_{i != j} D_i D_j 1/|x_i - x_j| (Eq. relerrnonperio, no images),
    by the same pair evaluators with the bare kernel (a = 0), FP64.
    Returns (E, grad N x 13 or None)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    jj = np.concatenate([np.concatenate([np.arange(i), np.arange(i + 1, n)]) for i in range(n)]) if n > 1 \
        else np.zeros(0, dtype=np.int64)
    rowptr = np.arange(n + 1, dtype=np.int64) * (n - 1)
    e, g = pair_csr(x, mp, rowptr, jj, np.zeros((len(jj), 3)), 0.0, tensor=tensor, grad=grad,
                    nthreads=nthreads)
    return 0.5 * e, g


def direct_nonperiodic_rows(x, mp, targets, tensor: bool = False, nthreads: int | None = None):
    """Gradient rows (len(targets) x 13) of the non-periodic direct sum for the
    given target atoms only (all sources j != i), FP64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    targets = np.asarray(targets, dtype=np.int64)
    xs = np.concatenate([x[targets], x])
    mps = np.concatenate([mp[targets], mp])
    nt = len(targets)
    cols = [np.concatenate([np.arange(nt, nt + t), np.arange(nt + t + 1, nt + n)]) for t in targets]
    rowptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int64)
    rowptr = np.concatenate([rowptr, np.full(n, rowptr[-1], dtype=np.int64)])
    col = np.concatenate(cols)
    _, g = pair_csr(xs, mps, rowptr, col, np.zeros((len(col), 3)), 0.0, tensor=tensor, grad=True,
                    nthreads=nthreads)
    return g[:nt]
