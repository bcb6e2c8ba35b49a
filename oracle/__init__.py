"""CPU oracle for Monte Carlo SPECT system matrices and ML-EM.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product library never imports it.  It shares no
code with the CUDA path (``mc_oracle.c`` is its own FP64 transport; the
reconstruction below is plain NumPy/SciPy in float64).

Transport (paper Sec. 2, Sec. 5.1): ``run`` follows photon histories and
returns tally events; ``system_counts`` turns events into the count matrix C
whose columns, divided by the histories started in each voxel, estimate
T_ij of Eq. (IMC).  ``run_fd`` is the forced-detection variant (the paper's
variance-reduction section): weighted events, summed by ``system_weights``.

Reconstruction (paper Sec. 5.1, Eq. (MLEM)):
    S_i^{k+1} = S_i^k / (sum_j T_ij) * sum_m P_m T_im / (sum_l S_l^k T_lm)
written with A[m, i] = T_im (rows = detector bins, columns = voxels):
    x <- x / s * A^T (y / (A x)),   s = A^T 1.
Readings where the equation is silent: voxels with s_v = 0 stay 0; a bin
with (A x)_j = 0 contributes 0 to the back-projection; the start image is
uniform, sum(y) / sum(s) on the support.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "mc_oracle.c")

FATE_ABSORBED, FATE_BELOW_WINDOW, FATE_ESCAPE, FATE_CAP = 0, 1, 2, 3
FATE_NAMES = ("absorbed", "below_window", "escape", "cap")
MAX_REC_EVENTS = 4

RECORD_DTYPE = np.dtype([
    ("fate", np.uint8), ("n_events", np.uint8), ("pad", np.uint16),
    ("n_virtual", np.uint32), ("n_real", np.uint32), ("n_compton", np.uint32),
    ("n_draws", np.uint32), ("pad2", np.uint32), ("e_final_kev", np.float64),
    ("event_row", np.int32, (MAX_REC_EVENTS,)),
])


def build(force: bool = False) -> str:
    """Compile mc_oracle.c into _build/liboracle.so with gcc (FP64, no
    fused multiply-add, so results match across hosts)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None
_lock = threading.Lock()


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("voxel_mm", ctypes.c_double),
        ("material", ctypes.c_void_p),
        ("n_materials", ctypes.c_int32),
        ("rho", ctypes.c_void_p), ("z_over_a", ctypes.c_void_p), ("z_eff", ctypes.c_void_p),
        ("n_views", ctypes.c_int32),
        ("start_deg", ctypes.c_double), ("arc_deg", ctypes.c_double),
        ("n_bins_u", ctypes.c_int32), ("n_bins_v", ctypes.c_int32),
        ("bin_mm", ctypes.c_double), ("radius_mm", ctypes.c_double),
        ("hole_len_mm", ctypes.c_double), ("hole_diam_mm", ctypes.c_double),
        ("fwhm_mm", ctypes.c_double), ("e0_kev", ctypes.c_double),
        ("window_frac", ctypes.c_double), ("photo_k", ctypes.c_double),
        ("primary_only", ctypes.c_int32),
        ("forced_detection", ctypes.c_int32),
        ("forced_direction", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_sigma_kn_cm2.argtypes = [dbl]
            L.orc_sigma_kn_cm2.restype = dbl
            L.orc_mu_total.argtypes = [P, ctypes.c_int, dbl]
            L.orc_mu_total.restype = dbl
            L.orc_majorant.argtypes = [P]
            L.orc_majorant.restype = dbl
            L.orc_rotate.argtypes = [vp, dbl, dbl]
            L.orc_trace.argtypes = [P, u64, u64, u64, vp]
            L.orc_trace.restype = ctypes.c_int
            L.orc_run.argtypes = [P, u64, u64, u64, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                  ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)), ctypes.POINTER(ctypes.c_int64), vp]
            L.orc_run.restype = ctypes.c_int
            L.orc_run_w.argtypes = [P, u64, u64, u64, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                    ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                    ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)), ctypes.POINTER(ctypes.c_int64), vp]
            L.orc_run_w.restype = ctypes.c_int
            L.orc_direction_band.argtypes = [P]
            L.orc_direction_band.restype = dbl
            L.orc_kn_pdf_sr.argtypes = [dbl, dbl]
            L.orc_kn_pdf_sr.restype = dbl
            L.orc_transmission.argtypes = [P, vp, vp, dbl]
            L.orc_transmission.restype = dbl
            L.orc_fd_point.argtypes = [P, u64, u64, ctypes.c_uint32, vp, vp, dbl, dbl, ctypes.c_int, vp, vp, i32]
            L.orc_fd_point.restype = ctypes.c_int
            L.orc_free.argtypes = [vp]
            L.orc_beam.argtypes = [P, u64, u64, vp, vp, dbl]
            L.orc_beam.restype = u64
            L.orc_kn_sample.argtypes = [dbl, u64, u64, vp, vp]
            L.orc_kn_sample.restype = u64
            L.orc_uniforms.argtypes = [u64, u64, u64, vp]
            L.orc_detect.argtypes = [P, u64, u64, vp, vp, vp, i32]
            L.orc_detect.restype = ctypes.c_int
            _lib = L
    return _lib


class Problem:
    """A phantom + geometry pair marshalled for the C oracle.  Keeps the
    NumPy buffers alive for as long as the struct is in use."""

    def __init__(self, phantom, geometry, primary_only: bool = False, forced_detection: bool = False,
                 forced_direction: bool = False):
        if forced_direction and not primary_only:
            raise ValueError("forced direction is exact for unscattered photons only: use primary_only=True")
        self.material = np.ascontiguousarray(phantom.material, dtype=np.uint8)
        self.rho = np.ascontiguousarray(phantom.rho, dtype=np.float64)
        self.zoa = np.ascontiguousarray(phantom.z_over_a, dtype=np.float64)
        self.zeff = np.ascontiguousarray(phantom.z_eff, dtype=np.float64)
        nz, ny, nx = self.material.shape
        g = geometry
        self.n_voxels = nx * ny * nz
        self.n_rows = g.n_views * g.n_bins_u * g.n_bins_v
        self.s = _Problem(nx, ny, nz, float(phantom.voxel_mm), self.material.ctypes.data, len(self.rho),
                          self.rho.ctypes.data, self.zoa.ctypes.data, self.zeff.ctypes.data,
                          g.n_views, float(g.start_deg), float(g.arc_deg), g.n_bins_u, g.n_bins_v,
                          float(g.bin_mm), float(g.radius_mm), float(g.hole_len_mm), float(g.hole_diam_mm),
                          float(g.fwhm_mm), float(g.e0_kev), float(g.window_frac), float(g.photo_k),
                          int(bool(primary_only)), int(bool(forced_detection)), int(bool(forced_direction)))
        self.forced_detection = bool(forced_detection)
        self.forced_direction = bool(forced_direction)

    @property
    def ref(self):
        return ctypes.byref(self.s)


# ---------------------------------------------------------------------------
# transport
# ---------------------------------------------------------------------------
def philox4x32_10(counter, key):
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def uniforms(seed: int, history: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.float64)
    lib().orc_uniforms(seed, history, n, out.ctypes.data)
    return out


def sigma_kn_cm2(e_kev: float) -> float:
    return lib().orc_sigma_kn_cm2(float(e_kev))


def mu_total(prob: Problem, m: int, e_kev: float) -> float:
    """Linear attenuation of material m, 1/mm."""
    return lib().orc_mu_total(prob.ref, int(m), float(e_kev))


def majorant(prob: Problem) -> float:
    return lib().orc_majorant(prob.ref)


def rotate(d, mu: float, phi: float) -> np.ndarray:
    v = np.array(d, dtype=np.float64)
    lib().orc_rotate(v.ctypes.data, float(mu), float(phi))
    return v


def trace(prob: Problem, seed: int, first: int, count: int) -> np.ndarray:
    """Per-history records (fate, collision counts, final energy, events)."""
    out = np.zeros(count, RECORD_DTYPE)
    lib().orc_trace(prob.ref, seed, first, count, out.ctypes.data)
    return out


def run(prob: Problem, seed: int, first: int, count: int, threads: int | None = None):
    """Run histories [first, first+count).  Returns (rows int32, cols int64,
    fates[4]) with events in history order."""
    if threads is None:
        threads = os.cpu_count() or 1
    L = lib()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cp = ctypes.POINTER(ctypes.c_int64)()
    n = ctypes.c_int64(0)
    fates = np.zeros(4, np.uint64)
    rc = L.orc_run(prob.ref, seed, first, count, int(threads), ctypes.byref(rp), ctypes.byref(cp),
                   ctypes.byref(n), fates.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle transport ran out of memory")
    ne = n.value
    rows = np.ctypeslib.as_array(rp, shape=(max(ne, 1),))[:ne].copy()
    cols = np.ctypeslib.as_array(cp, shape=(max(ne, 1),))[:ne].copy()
    L.orc_free(ctypes.cast(rp, ctypes.c_void_p))
    L.orc_free(ctypes.cast(cp, ctypes.c_void_p))
    return rows, cols, fates


def run_fd(prob: Problem, seed: int, first: int, count: int, threads: int | None = None):
    """Weighted transport (Problem(..., forced_detection=True) or
    forced_direction=True): histories [first, first+count).  Returns
    (rows int32, cols int64, q int64, fates[4]), q the fixed-point weights
    w * 2^48 rounded to the nearest integer."""
    if not (prob.forced_detection or prob.forced_direction):
        raise ValueError("run_fd needs a Problem with forced_detection or forced_direction")
    if threads is None:
        threads = os.cpu_count() or 1
    L = lib()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cp = ctypes.POINTER(ctypes.c_int64)()
    qp = ctypes.POINTER(ctypes.c_int64)()
    n = ctypes.c_int64(0)
    fates = np.zeros(4, np.uint64)
    rc = L.orc_run_w(prob.ref, seed, first, count, int(threads), ctypes.byref(rp), ctypes.byref(cp),
                     ctypes.byref(qp), ctypes.byref(n), fates.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle transport ran out of memory")
    ne = n.value
    rows = np.ctypeslib.as_array(rp, shape=(max(ne, 1),))[:ne].copy()
    cols = np.ctypeslib.as_array(cp, shape=(max(ne, 1),))[:ne].copy()
    q = np.ctypeslib.as_array(qp, shape=(max(ne, 1),))[:ne].copy()
    for ptr in (rp, cp, qp):
        L.orc_free(ctypes.cast(ptr, ctypes.c_void_p))
    return rows, cols, q, fates


FD_SCALE = 2.0 ** 48


def direction_band(prob: Problem) -> float:
    """Half-width in cos(theta) of the forced emission band, sin(psi_max)."""
    return lib().orc_direction_band(prob.ref)


def kn_pdf_sr(e_kev: float, mu: float) -> float:
    """Klein-Nishina angular density of the scattered direction, per sr."""
    return lib().orc_kn_pdf_sr(float(e_kev), float(mu))


def transmission(prob: Problem, p, d, e_kev: float) -> float:
    """exp(-line integral of mu(E)) from p along d to the grid boundary."""
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    return lib().orc_transmission(prob.ref, pp.ctypes.data, dd.ctypes.data, float(e_kev))


def fd_point(prob: Problem, seed: int, history: int, n: int, p, d_in, e_kev: float, p_keep: float,
             emission: bool, max_rows: int = 4096):
    """Forced copies of one interaction: (rows, q) over the views."""
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d_in, dtype=np.float64)
    rows = np.zeros(max_rows, np.int32)
    qs = np.zeros(max_rows, np.int64)
    k = lib().orc_fd_point(prob.ref, seed, history, int(n), pp.ctypes.data, dd.ctypes.data, float(e_kev),
                           float(p_keep), int(bool(emission)), rows.ctypes.data, qs.ctypes.data, max_rows)
    return rows[:min(k, max_rows)], qs[:min(k, max_rows)]


def beam(prob: Problem, seed: int, n: int, p0, d, e_kev: float) -> int:
    p = np.ascontiguousarray(p0, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    return int(lib().orc_beam(prob.ref, seed, n, p.ctypes.data, dd.ctypes.data, float(e_kev)))


def kn_sample(e_kev: float, seed: int, n: int):
    c = np.zeros(n, np.float64)
    e = np.zeros(n, np.float64)
    capped = lib().orc_kn_sample(float(e_kev), seed, n, c.ctypes.data, e.ctypes.data)
    return c, e, int(capped)


def detect(prob: Problem, seed: int, history: int, p, d, max_rows: int = 8):
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    rows = np.zeros(max_rows, np.int32)
    n = lib().orc_detect(prob.ref, seed, history, pp.ctypes.data, dd.ctypes.data, rows.ctypes.data, max_rows)
    return rows[:min(n, max_rows)], n


# ---------------------------------------------------------------------------
# system matrix (paper Eq. (IMC): T_ij = P(detected in j | emitted in i))
# ---------------------------------------------------------------------------
def histories_per_voxel(n_voxels: int, first: int, count: int) -> np.ndarray:
    """n_v = number of histories h in [first, first+count) with h mod N = v
    (history h starts in voxel h mod N)."""
    v = np.arange(n_voxels, dtype=np.int64)
    lo = first
    hi = first + count
    # count of h in [lo, hi) with h = v (mod N) = ceil((hi - v)/N) - ceil((lo - v)/N)
    return (-((v - hi) // n_voxels)) - (-((v - lo) // n_voxels))


def system_counts(rows, cols, n_rows: int, n_voxels: int) -> sp.csc_matrix:
    """Count matrix C[j, v] = number of events (j, v), as CSC int64 with
    sorted row indices."""
    key = np.asarray(cols, np.int64) * n_rows + np.asarray(rows, np.int64)
    uk, cnt = np.unique(key, return_counts=True)
    c = uk // n_rows
    r = uk % n_rows
    m = sp.csc_matrix((cnt.astype(np.int64), (r, c)), shape=(n_rows, n_voxels))
    m.sort_indices()
    return m


def system_weights(rows, cols, q, n_rows: int, n_voxels: int) -> sp.csc_matrix:
    """Weighted tally W[j, v] = sum of the fixed-point weights q of the events
    (j, v), summed as exact integers, returned as float64 (q * 2^-48) CSC
    with sorted row indices (every sum is below 2^53 units, so exact)."""
    key = np.asarray(cols, np.int64) * n_rows + np.asarray(rows, np.int64)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    qs = np.asarray(q, np.int64)[order]
    if len(ks) == 0:
        return sp.csc_matrix((n_rows, n_voxels), dtype=np.float64)
    heads = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    uk = ks[heads]
    sums = np.add.reduceat(qs, heads)
    m = sp.csc_matrix((sums.astype(np.float64) / FD_SCALE, (uk % n_rows, uk // n_rows)), shape=(n_rows, n_voxels))
    m.sort_indices()
    return m


def build_system_fd(prob: Problem, seed: int, n_histories: int, first: int = 0, threads=None):
    """Forced-detection transport + tally: (A float64 CSR, W float64 CSC, n_v, fates)."""
    rows, cols, q, fates = run_fd(prob, seed, first, n_histories, threads)
    w = system_weights(rows, cols, q, prob.n_rows, prob.n_voxels)
    n_v = histories_per_voxel(prob.n_voxels, first, n_histories)
    return system_matrix(w, n_v), w, n_v, fates


def system_matrix(counts: sp.spmatrix, n_v: np.ndarray) -> sp.csr_matrix:
    """A = C diag(1/n_v) in float64 (columns with n_v = 0 are empty)."""
    inv = np.where(n_v > 0, 1.0 / np.maximum(n_v, 1), 0.0)
    a = sp.csr_matrix(counts, dtype=np.float64) @ sp.diags(inv)
    a = sp.csr_matrix(a)
    a.sort_indices()
    return a


def build_system(prob: Problem, seed: int, n_histories: int, first: int = 0, threads=None):
    """Transport + tally: returns (A float64 CSR, C int64 CSC, n_v, fates)."""
    rows, cols, fates = run(prob, seed, first, n_histories, threads)
    c = system_counts(rows, cols, prob.n_rows, prob.n_voxels)
    n_v = histories_per_voxel(prob.n_voxels, first, n_histories)
    return system_matrix(c, n_v), c, n_v, fates


# ---------------------------------------------------------------------------
# ML-EM (paper Eq. (MLEM)), float64
# ---------------------------------------------------------------------------
def sensitivity(a: sp.spmatrix) -> np.ndarray:
    """s_v = sum_j A[j, v] (the normaliser of Eq. (MLEM))."""
    return np.asarray(a.sum(axis=0), dtype=np.float64).ravel()


def mlem_init(a: sp.spmatrix, y: np.ndarray) -> np.ndarray:
    s = sensitivity(a)
    tot = s.sum()
    x = np.zeros(a.shape[1], np.float64)
    if tot > 0:
        x[s > 0] = float(np.sum(np.asarray(y, np.float64))) / tot
    return x


def reached_bins(a: sp.spmatrix) -> np.ndarray:
    """Bins whose row of A holds an entry: the bins the model can reach."""
    return np.diff(sp.csr_matrix(a).indptr) > 0


def loglik(a: sp.spmatrix, x: np.ndarray, y: np.ndarray) -> float:
    """Poisson log-likelihood without the constant: sum_j y_j ln q_j - q_j,
    q = A x; bins with y_j = 0 contribute -q_j only.  A bin whose row of A is
    empty is left out of the y_j ln q_j sum: q_j = 0 for every image, so the
    term carries no information about x (it would be -inf whatever x is),
    and ML-EM ignores the bin the same way (r_j = 0 where (A x)_j = 0)."""
    q = a @ np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    pos = (y > 0) & reached_bins(a)
    with np.errstate(divide="ignore"):
        return float(np.sum(y[pos] * np.log(q[pos])) - np.sum(q))


def mlem_step(a: sp.spmatrix, y: np.ndarray, x: np.ndarray, s: np.ndarray | None = None) -> np.ndarray:
    if s is None:
        s = sensitivity(a)
    q = a @ x
    r = np.zeros_like(q)
    np.divide(np.asarray(y, np.float64), q, out=r, where=q > 0)
    b = a.T @ r
    out = np.zeros_like(x)
    np.divide(x * b, s, out=out, where=s > 0)
    return out


def mlem(a: sp.spmatrix, y: np.ndarray, x0: np.ndarray, n_iter: int, with_loglik: bool = False):
    """n_iter ML-EM updates from x0.  With with_loglik, also returns
    [L(x^0), ..., L(x^{n_iter-1})]."""
    a = sp.csr_matrix(a, dtype=np.float64)
    y = np.asarray(y, np.float64)
    x = np.asarray(x0, np.float64).copy()
    s = sensitivity(a)
    ll = []
    for _ in range(n_iter):
        if with_loglik:
            ll.append(loglik(a, x, y))
        x = mlem_step(a, y, x, s)
    return (x, ll) if with_loglik else x


# ---------------------------------------------------------------------------
# ordered subsets, dual matrix, additive term (paper Sec. 5.3-5.4:
# OSEM; Eq. (DMOS); Eq. (Sohlberg OSEM))
# ---------------------------------------------------------------------------
def subset_rows(n_rows: int, rows_per_view: int, n_subsets: int, subset: int) -> np.ndarray:
    """Rows of views subset, subset + n_subsets, ... (rows are view-major)."""
    views = np.arange(subset, n_rows // rows_per_view, n_subsets, dtype=np.int64)
    return (views[:, None] * rows_per_view + np.arange(rows_per_view, dtype=np.int64)[None, :]).ravel()


def osem(a_fwd: sp.spmatrix, a_back: sp.spmatrix, subsets, y: np.ndarray, x0: np.ndarray, n_iter: int,
         add: np.ndarray | None = None) -> np.ndarray:
    """n_iter sweeps over the row subsets: for each subset S,
        q = C_S x,  r = y_S / (q + add_S)  (0 where not positive),
        x <- x / (B_S^T 1) * B_S^T r      (x kept where B_S^T 1 = 0: the
                                           voxel is outside the subset's view),
    with C = a_fwd (reprojection) and B = a_back (back-projection)."""
    c = sp.csr_matrix(a_fwd, dtype=np.float64)
    b = sp.csr_matrix(a_back, dtype=np.float64)
    y = np.asarray(y, np.float64)
    ad = np.zeros_like(y) if add is None else np.asarray(add, np.float64)
    x = np.asarray(x0, np.float64).copy()
    parts = [(c[rows], b[rows], rows) for rows in subsets]
    for _ in range(n_iter):
        for cs, bs, rows in parts:
            den = cs @ x + ad[rows]
            r = np.zeros_like(den)
            np.divide(y[rows], den, out=r, where=den > 0)
            sb = np.asarray(bs.sum(axis=0), dtype=np.float64).ravel()
            t = bs.T @ r
            out = x.copy()      # a voxel the subset does not see keeps its value
            np.divide(x * t, sb, out=out, where=sb > 0)
            x = out
    return x


# ---------------------------------------------------------------------------
# penalised Poisson likelihood (Sec. 5.1 likelihood + quadratic smoothness)
# ---------------------------------------------------------------------------
def prior_quadratic(x: np.ndarray, shape, beta: float):
    """R(x) = beta/2 * sum over 6-neighbour voxel pairs (x_v - x_w)^2 and its
    gradient, for an image of shape (nz, ny, nx), x fastest."""
    img = np.asarray(x, np.float64).reshape(shape)
    val = 0.0
    grad = np.zeros_like(img)
    for ax in range(3):
        d = np.diff(img, axis=ax)            # x_{v+1} - x_v along the axis
        val += float(np.sum(d * d))
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        grad[tuple(lo)] -= d                 # v gets (x_v - x_{v+1})
        grad[tuple(hi)] += d                 # v+1 gets (x_{v+1} - x_v)
    return 0.5 * beta * val, beta * grad.ravel()


def penalised_objective(a: sp.spmatrix, y: np.ndarray, x: np.ndarray, shape, beta: float) -> float:
    """sum_j (q_j - y_j ln q_j) + R(x), q = A x (negative log-likelihood up to
    a constant, plus the prior); bins with an empty row of A are left out of
    the y_j ln q_j sum, as in ``loglik``."""
    q = a @ np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    pos = (y > 0) & reached_bins(a)
    with np.errstate(divide="ignore"):
        return float(np.sum(q) - np.sum(y[pos] * np.log(q[pos])) + prior_quadratic(x, shape, beta)[0])


def penalised_gradient(a: sp.spmatrix, y: np.ndarray, x: np.ndarray, shape, beta: float) -> np.ndarray:
    q = a @ np.asarray(x, np.float64)
    r = np.zeros_like(q)
    np.divide(np.asarray(y, np.float64), q, out=r, where=q > 0)
    return sensitivity(a) - a.T @ r + prior_quadratic(x, shape, beta)[1]
