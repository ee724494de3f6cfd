"""CPU oracle for the exact Gaussian log-likelihood (Eq. 1) with a Matern
covariance (Eq. 2), evaluated as in Algorithm 2.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path: the arithmetic lives in ``egs_oracle.c`` (plain FP64 C) and in
this file, where NumPy/SciPy library routines serve as whole steps of
Algorithm 2 (``dpotrf`` -> ``scipy.linalg.cholesky``, ``dtrsm`` ->
``scipy.linalg.solve_triangular``) for sizes where the textbook C Cholesky
would be too slow.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, SciPy's independent Bessel routine, brute-force determinants and
inverses in long double, and invariances of Eq. 1.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libegs_oracle.so")
_SRC = os.path.join(_HERE, "egs_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/libegs_oracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i64 = ctypes.c_double, ctypes.c_int64
    P = ctypes.POINTER
    pd = P(ctypes.c_double)
    lib.ora_bessel_k.restype = d
    lib.ora_bessel_k.argtypes = [d, d]
    lib.ora_bessel_k_scaled.restype = d
    lib.ora_bessel_k_scaled.argtypes = [d, d, d]
    lib.ora_matern.restype = d
    lib.ora_matern.argtypes = [pd, d]
    lib.ora_cov_matrix.restype = None
    lib.ora_cov_matrix.argtypes = [i64, pd, pd, pd, pd]
    lib.ora_cov_cross.restype = None
    lib.ora_cov_cross.argtypes = [i64, pd, pd, i64, pd, pd, pd, pd]
    lib.ora_cholesky.restype = i64
    lib.ora_cholesky.argtypes = [i64, pd]
    lib.ora_forward_solve.restype = None
    lib.ora_forward_solve.argtypes = [i64, pd, pd, pd]
    lib.ora_loglik.restype = i64
    lib.ora_loglik.argtypes = [i64, pd, pd, pd, pd, pd]
    lib.ora_brute_logdet.restype = ctypes.c_int
    lib.ora_brute_logdet.argtypes = [i64, pd, P(ctypes.c_longdouble)]
    lib.ora_brute_quad.restype = ctypes.c_int
    lib.ora_brute_quad.argtypes = [i64, pd, pd, P(ctypes.c_longdouble)]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------
# Eq. 2 and its special function
# ----------------------------------------------------------------------------

def bessel_k(nu: float, x) -> np.ndarray:
    """K_nu(x) by the integral representation (DLMF 10.32.9), trapezoidal rule."""
    lib = _load()
    xs = np.atleast_1d(_f64(x))
    return np.array([lib.ora_bessel_k(float(nu), float(v)) for v in xs]).reshape(np.shape(x))


def bessel_k_scaled(nu: float, x, h: float = 0.05) -> np.ndarray:
    """e^x K_nu(x) with trapezoid step h (capped at 0.2/sqrt(x))."""
    lib = _load()
    xs = np.atleast_1d(_f64(x))
    return np.array([lib.ora_bessel_k_scaled(float(nu), float(v), float(h)) for v in xs]).reshape(np.shape(x))


def matern(theta, r) -> np.ndarray:
    """Eq. 2 at distances r (C(0) = theta1)."""
    lib = _load()
    th = _f64(theta)
    rs = np.atleast_1d(_f64(r))
    return np.array([lib.ora_matern(_p(th), float(v)) for v in rs]).reshape(np.shape(r))


EARTH_RADIUS_KM = 6371.0


def gcd_dist(locs1, locs2, radius: float = EARTH_RADIUS_KM) -> np.ndarray:
    """Great-circle distances (Section 7.4) between (longitude, latitude)
    pairs in degrees, by the haversine formula
    hav(d / r) = hav(phi2 - phi1) + cos(phi1) cos(phi2) hav(lambda2 - lambda1),
    hav(t) = (1 - cos t) / 2, d = 2 r asin(sqrt(hav(d / r)))."""
    a, b = _f64(locs1), _f64(locs2)
    lam1, phi1 = np.radians(a[0])[:, None], np.radians(a[1])[:, None]
    lam2, phi2 = np.radians(b[0])[None, :], np.radians(b[1])[None, :]
    h = (1.0 - np.cos(phi2 - phi1)) / 2.0 + np.cos(phi1) * np.cos(phi2) * (1.0 - np.cos(lam2 - lam1)) / 2.0
    return 2.0 * radius * np.arcsin(np.sqrt(np.clip(h, 0.0, 1.0)))


def cov_matrix_gcd(locs, theta) -> np.ndarray:
    """Sigma(theta) with great-circle distances in km (locations in degrees)."""
    d = gcd_dist(locs, locs)
    np.fill_diagonal(d, 0.0)
    return matern(theta, d.reshape(-1)).reshape(d.shape)


def loglik_gcd(locs, z, theta) -> dict:
    """Eq. 1 by Algorithm 2 (LAPACK steps) on the great-circle Sigma."""
    import scipy.linalg as sla

    S = cov_matrix_gcd(locs, theta)
    n = S.shape[0]
    try:
        L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(-1) from exc
    y = sla.solve_triangular(L, _f64(z), lower=True, check_finite=False)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    quad = float(y @ y)
    return {"loglik": -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2.0 * math.pi),
            "logdet": logdet, "quad": quad}


def cov_matrix(locs, theta) -> np.ndarray:
    """Dense Sigma(theta) (Section 2): Sigma_ij = C(||s_i - s_j||; theta)."""
    lib = _load()
    locs = _f64(locs)
    n = locs.shape[1]
    x, y = _f64(locs[0]), _f64(locs[1])
    th = _f64(theta)
    S = np.empty((n, n))
    lib.ora_cov_matrix(n, _p(x), _p(y), _p(th), _p(S))
    return S


def cov_cross(locs1, locs2, theta) -> np.ndarray:
    """Sigma_12 between the columns of locs1 (rows) and locs2 (columns)."""
    lib = _load()
    a, b = _f64(locs1), _f64(locs2)
    m, n = a.shape[1], b.shape[1]
    th = _f64(theta)
    S = np.empty((m, n))
    lib.ora_cov_cross(m, _p(_f64(a[0])), _p(_f64(a[1])), n, _p(_f64(b[0])), _p(_f64(b[1])), _p(th), _p(S))
    return S


# ----------------------------------------------------------------------------
# Algorithm 2 with the textbook C routines (small n)
# ----------------------------------------------------------------------------

class NotPositiveDefinite(Exception):
    def __init__(self, column: int):
        super().__init__("matrix is not positive definite at column %d" % column)
        self.column = column


def cholesky(S) -> np.ndarray:
    """Textbook left-looking Cholesky; returns L (lower, zero upper)."""
    lib = _load()
    A = _f64(S).copy()
    fail = lib.ora_cholesky(A.shape[0], _p(A))
    if fail >= 0:
        raise NotPositiveDefinite(int(fail))
    return A


def forward_solve(L, z) -> np.ndarray:
    lib = _load()
    L = _f64(L)
    z = _f64(z)
    y = np.empty_like(z)
    lib.ora_forward_solve(L.shape[0], _p(L), _p(z), _p(y))
    return y


def loglik(locs, z, theta) -> dict:
    """Eq. 1 by Algorithm 2 with the C routines.  Returns l, logdet, quad."""
    lib = _load()
    locs = _f64(locs)
    n = locs.shape[1]
    out = np.empty(3)
    fail = lib.ora_loglik(n, _p(_f64(locs[0])), _p(_f64(locs[1])), _p(_f64(z)), _p(_f64(theta)), _p(out))
    if fail == -2:
        raise MemoryError("oracle: allocation failed")
    if fail >= 0:
        raise NotPositiveDefinite(int(fail))
    return {"loglik": float(out[0]), "logdet": float(out[1]), "quad": float(out[2])}


# ----------------------------------------------------------------------------
# Algorithm 2 with LAPACK as the dpotrf / dtrsm steps (larger n)
# ----------------------------------------------------------------------------

def loglik_lapack(locs, z, theta, return_factor: bool = False) -> dict:
    """Eq. 1 by Algorithm 2, with LAPACK dpotrf and a triangular solve as steps."""
    import scipy.linalg as sla

    S = cov_matrix(locs, theta)
    n = S.shape[0]
    try:
        L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(-1) from exc
    y = sla.solve_triangular(L, _f64(z), lower=True, check_finite=False)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    quad = float(y @ y)
    out = {"loglik": -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2.0 * math.pi),
           "logdet": logdet, "quad": quad}
    if return_factor:
        out["L"] = L
        out["y"] = y
    return out


def loglik_ind(locs, z, theta, block: int) -> dict:
    """The IND approximation (Section 6.8) by its definition: Sigma with every
    entry between different diagonal blocks of `block` consecutive locations
    set to zero, then Eq. 1 by Algorithm 2 (LAPACK steps) on that matrix."""
    import scipy.linalg as sla

    S = cov_matrix(locs, theta)
    n = S.shape[0]
    blk = np.arange(n) // int(block)
    S[blk[:, None] != blk[None, :]] = 0.0
    try:
        L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(-1) from exc
    y = sla.solve_triangular(L, _f64(z), lower=True, check_finite=False)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    quad = float(y @ y)
    return {"loglik": -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2.0 * math.pi),
            "logdet": logdet, "quad": quad}


def simulate_z(locs, theta, e) -> np.ndarray:
    """Algorithm 1: Sigma = L L^T (dpotrf), Z = L e (dtrmm)."""
    import scipy.linalg as sla

    S = cov_matrix(locs, theta)
    L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    return L @ _f64(e)


def simulate_loglik(locs, theta, e) -> dict:
    """Algorithm 1 followed by Algorithm 2 at the same theta, sharing the one
    factorisation both take of Sigma(theta): L = dpotrf(Sigma), Z = L e
    (Algorithm 1), then y = L^-1 Z, log|Sigma| = 2 sum log L_ii, Z^T Sigma^-1 Z
    = y^T y and Eq. 1 (Algorithm 2).  Returns l, logdet, quad and z; the same
    numbers as simulate_z followed by loglik_lapack, for one Cholesky instead
    of two at large n."""
    import scipy.linalg as sla

    S = cov_matrix(locs, theta)
    n = S.shape[0]
    try:
        L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(-1) from exc
    del S
    z = L @ _f64(e)
    y = sla.solve_triangular(L, z, lower=True, check_finite=False)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    quad = float(y @ y)
    return {"loglik": -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2.0 * math.pi),
            "logdet": logdet, "quad": quad, "z": z}


def predict(locs_obs, z_obs, locs_new, theta) -> np.ndarray:
    """Eq. 5 via Algorithm 3: Z1 = Sigma_12 Sigma_22^{-1} Z2."""
    import scipy.linalg as sla

    S22 = cov_matrix(locs_obs, theta)
    S12 = cov_cross(locs_new, locs_obs, theta)
    c = sla.cho_factor(S22, lower=True, check_finite=False)
    x = sla.cho_solve(c, _f64(z_obs), check_finite=False)
    return S12 @ x


# ----------------------------------------------------------------------------
# Brute force (long double)
# ----------------------------------------------------------------------------

def brute_logdet(S) -> tuple:
    """(sign, log|det S|) by LU with partial pivoting in long double."""
    lib = _load()
    S = _f64(S)
    out = ctypes.c_longdouble(0.0)
    sign = lib.ora_brute_logdet(S.shape[0], _p(S), ctypes.byref(out))
    return int(sign), float(out.value)


def brute_quad(S, z) -> float:
    """Z^T S^{-1} Z with a Gauss-Jordan inverse in long double."""
    lib = _load()
    S = _f64(S)
    out = ctypes.c_longdouble(0.0)
    rc = lib.ora_brute_quad(S.shape[0], _p(S), _p(_f64(z)), ctypes.byref(out))
    if rc != 0:
        raise ZeroDivisionError("singular matrix")
    return float(out.value)


def tiles_lower(M, tile: int) -> list:
    """Reference view of a dense n x n matrix as padded lower tiles.

    Tile (i, j), i >= j, of a T x T tiling (T = ceil(n / tile)) is returned in
    row-major order; rows and columns beyond n are zero except the padded
    diagonal, which is one.  This is how the library is specified to lay out
    Sigma and L, so tests can compare tile by tile."""
    M = _f64(M)
    n = M.shape[0]
    T = -(-n // tile)
    P = np.zeros((T * tile, T * tile))
    P[:n, :n] = M
    for k in range(n, T * tile):
        P[k, k] = 1.0
    out = []
    for i in range(T):
        for j in range(i + 1):
            out.append(P[i * tile:(i + 1) * tile, j * tile:(j + 1) * tile].copy())
    return out
