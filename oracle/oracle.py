"""Python entry to the FP64 CPU oracle (``kp_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The product path never imports this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  It shares no code with the CUDA library.

Arrays are numpy ``float64`` vectors of length N = H*W in the paper's
y-fastest order (index ``i*H + j``, i = x column, j = y row; Sec. 2.3,
Eq. 14-15).  A channel held as a numpy array of shape ``(W, H)`` in C order
has exactly this layout.

Parity notes: every function states which passage of arXiv 2511.17634 it
follows.  The stencil, right-hand side and CSR assembly are pinned by the
consistency test against the continuous PDE (Eq. 5, linearised as in Sec. 2.3)
on quadratic fields, where the central differences are exact; GMRES and the
projection are pinned by dense LU, the discrete-sine closed form, the Arnoldi
identities and the FOM residual formula; BiCGSTAB by dense solves, finite
termination, and its key vectors spanning the Arnoldi spaces; the explicit
A_proj projection by its basis invariance against the Hessenberg one
(tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkp_oracle.so")

_d = ctypes.c_double
_i = ctypes.c_int
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)

NOT_CONVERGED = 1


def build(force: bool = False) -> str:
    """Compile kp_oracle.c into a shared library with gcc (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_coeffs.argtypes = [_i, _i, _d, _d, _d, _pd, _pd, _pd, _pd]
        L.orc_rhs.argtypes = [_i, _i, _d, _d, _pd, _pd, _pd, _pd]
        L.orc_apply.argtypes = [_i, _i, _pd, _pd, _pd]
        L.orc_csr.argtypes = [_i, _i, _pd, _pi, _pi, _pd]
        L.orc_csr.restype = _i
        L.orc_csr_matvec.argtypes = [_i, _pi, _pi, _pd, _pd, _pd]
        L.orc_gmres.argtypes = [_i, _i, _pd, _pd, _pd, _d, _i, _i, _pi, _pd, _pd, _i,
                                _pd, _pd, _pi, _pi, _i]
        L.orc_gmres.restype = _i
        L.orc_project.argtypes = [_i, _i, _i, _i, _pd, _pd, _pd, _pd, _pd]
        L.orc_project.restype = _i
        L.orc_dense_lu_solve.argtypes = [_i, _pd, _pd, _pd]
        L.orc_dense_lu_solve.restype = _i
        L.orc_march_step.argtypes = [_i, _i, _d, _d, _d, _i, _pd, _i, _pd, _pi, _i, _d, _i,
                                     _i, _d, _i, _i, _pi, _pi, _pd, _pi, _pd, _i, _i, _pi, _i, _pd]
        L.orc_accumulate.argtypes = [_i, _i, _pd, _i, _pd, _i, _pd, _i, _pd, _pd]
        L.orc_accumulate.restype = _i
        L.orc_bicgstab.argtypes = [_i, _i, _pd, _pd, _pd, _d, _i, _pi, _pd, _i, _pd, _pi]
        L.orc_bicgstab.restype = _i
        L.orc_project_dense.argtypes = [_i, _i, _pd, _pd, _pd, _pd, _pd]
        L.orc_project_dense.restype = _i
        L.orc_score.argtypes = [_i, _i, _d, _pd, _pd, _pd]
        L.orc_project_galerkin.argtypes = [_i, _i, _pd, _i, _pd, _pd, _pd, _pd]
        L.orc_project_galerkin.restype = _i
        L.orc_embed_step.argtypes = [_i, _d, _d, _pd, _pd, _pd, _pd]
        L.orc_set_threads.argtypes = [_i]
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the oracle's OpenMP loops over independent systems (no
    effect when it was built without OpenMP)."""
    lib().orc_set_threads(int(n))


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(_pd)
    assert a.dtype == np.int32
    return a.ctypes.data_as(_pi)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def coeffs(H, W, g2, dt, h, mt, fx=None, fy=None):
    """Stencil coefficients (Sec. 2.3, listing after Eq. 11): array (N, 5) of
    [diag, east, west, north, south] per grid point."""
    mt, fx, fy = _f64(mt), _f64(fx), _f64(fy)
    C = np.zeros(5 * H * W)
    lib().orc_coeffs(H, W, g2, dt, h, _p(mt), _p(fx), _p(fy), _p(C))
    return C.reshape(H * W, 5)


def rhs(H, W, dt, h, mprev, fx=None, fy=None):
    """b = m^{n-1}/dt - Div_h f (Sec. 2.3, last line of the listing)."""
    mprev, fx, fy = _f64(mprev), _f64(fx), _f64(fy)
    b = np.zeros(H * W)
    lib().orc_rhs(H, W, dt, h, _p(mprev), _p(fx), _p(fy), _p(b))
    return b


def apply(H, W, C, x):
    """y = A x from the stencil coefficients (Eq. 11)."""
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(-1)
    x = _f64(x)
    y = np.zeros(H * W)
    lib().orc_apply(H, W, _p(C), _p(x), _p(y))
    return y


def csr(H, W, C):
    """Explicit CSR matrix assembled from the block form (Eq. 12-15):
    returns (rowptr, col, val)."""
    N = H * W
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(-1)
    rowptr = np.zeros(N + 1, dtype=np.int32)
    col = np.zeros(5 * N, dtype=np.int32)
    val = np.zeros(5 * N)
    nnz = lib().orc_csr(H, W, _p(C), _p(rowptr), _p(col), _p(val))
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


def csr_dense(H, W, C):
    """Dense N x N copy of the CSR matrix (tiny grids only)."""
    rowptr, col, val = csr(H, W, C)
    N = H * W
    A = np.zeros((N, N))
    for r in range(N):
        for k in range(rowptr[r], rowptr[r + 1]):
            A[r, col[k]] = val[k]
    return A


def csr_matvec(rowptr, col, val, x):
    x = _f64(x)
    y = np.zeros(len(rowptr) - 1)
    lib().orc_csr_matvec(len(rowptr) - 1, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


@dataclass
class GmresResult:
    x: np.ndarray
    status: int
    iters: int
    rel_res: float
    hist: np.ndarray
    V: np.ndarray | None = None      # (a'+has_next, N): rows are v_1, v_2, ...
    Hbar: np.ndarray | None = None   # (a'+1, a') unrotated Hessenberg
    a: int = 0
    has_next: int = 0


def gmres(H, W, C, b, x0=None, tol=1e-10, m=30, maxit=1000, capture=0, fixed=False):
    """Restarted GMRES(m), MGS Arnoldi run twice + Givens (Saad 2003, Alg. 6.9); with
    ``capture=a`` keeps the first cycle's basis and Hessenberg (Sec. 3,
    Phase 1).  ``fixed=True`` gives the basis the fixed dimension min(a, m) of
    Sec. 3 (Sec. 5.2: a = 20): the first cycle keeps taking Arnoldi steps after
    the residual test is met, until a steps, an exact breakdown or maxit."""
    N = H * W
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(-1)
    b = _f64(b)
    x = np.zeros(N) if x0 is None else _f64(x0).copy()
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    hist = np.full(maxit + 1, np.nan)
    capV = capH = None
    used = np.zeros(1, dtype=np.int32)
    nxt = np.zeros(1, dtype=np.int32)
    if capture > 0:
        capV = np.zeros((capture + 1) * N)
        capH = np.zeros((capture + 1) * capture)
    st = lib().orc_gmres(H, W, _p(C), _p(b), _p(x), tol, m, maxit, _p(it), _p(rr), _p(hist),
                         capture, _p(capV), _p(capH), _p(used), _p(nxt), int(bool(fixed)))
    res = GmresResult(x=x, status=st, iters=int(it[0]), rel_res=float(rr[0]),
                      hist=hist[~np.isnan(hist)])
    if capture > 0:
        a = int(used[0])
        res.a, res.has_next = a, int(nxt[0])
        res.V = capV.reshape(capture + 1, N)[: a + res.has_next].copy()
        res.Hbar = capH.reshape(capture, capture + 1).T[: a + 1, :a].copy()
    return res


def project(V, Hbar, a, has_next, r, xinit=None):
    """Sec. 3, Phase 2: x0 = xinit + V_a H_a^{-1} V_a^T r (least squares on
    Hbar if H_a is numerically singular).  Returns (x0, used_lsq)."""
    N = V.shape[1]
    lda = a + 1
    Vc = np.zeros((a + 1) * N)
    Vc[: V.shape[0] * N] = V.reshape(-1)
    Hc = np.zeros((a + 1) * max(a, 1))
    Hc.reshape(max(a, 1), a + 1)[:a, : Hbar.shape[0]] = Hbar.T
    r = _f64(r)
    xi = _f64(xinit)
    x0 = np.zeros(N)
    lsq = lib().orc_project(N, a, lda, has_next, _p(Vc), _p(Hc), _p(r), _p(xi), _p(x0))
    return x0, bool(lsq)


@dataclass
class BicgResult:
    x: np.ndarray
    status: int
    iters: int
    rel_res: float
    V: np.ndarray      # (a', N): the kept key vectors, orthonormal rows


def bicgstab(H, W, C, b, x0=None, tol=1e-10, maxit=1000, capture=0):
    """BiCGSTAB (van der Vorst 1992; Sec. 3, Phase 1 as printed) with true-residual
    restarts; with ``capture=a`` keeps up to a orthonormalised key vectors
    r_0, s_1, r_1, s_2, ... of the first sweep."""
    N = H * W
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(-1)
    b = _f64(b)
    x = np.zeros(N) if x0 is None else _f64(x0).copy()
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    used = np.zeros(1, dtype=np.int32)
    capV = np.zeros(max(capture, 1) * N)
    st = lib().orc_bicgstab(H, W, _p(C), _p(b), _p(x), tol, maxit, _p(it), _p(rr), capture,
                            _p(capV) if capture > 0 else None, _p(used))
    return BicgResult(x=x, status=st, iters=int(it[0]), rel_res=float(rr[0]),
                      V=capV.reshape(-1, N)[: int(used[0])].copy())


def project_dense(V, Aproj, r, xinit=None):
    """Sec. 3, Phase 2 with an explicit A_proj (a x a): x0 = xinit + V_a
    A_proj^{-1} V_a^T r.  V: (a, N) rows.  Returns (x0, singular)."""
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
    a, N = V.shape
    A = np.ascontiguousarray(np.asarray(Aproj, dtype=np.float64).reshape(a, a))
    x0 = np.zeros(N)
    rc = lib().orc_project_dense(N, a, _p(V.reshape(-1)), _p(A.reshape(-1)), _p(_f64(r)),
                                 _p(_f64(xinit)), _p(x0))
    return x0, bool(rc)


def accumulate(H, W, C, Vown, Vprev, cap_a):
    """Seed cycling (Sec. 5.2): the new seed's basis rows Vown first, then the
    previous accumulated rows Vprev, orthonormalised, capped at cap_a; returns
    (V rows, A_proj = V A_seed V^T) with C the new seed's coefficients."""
    N = H * W
    Vo = np.ascontiguousarray(np.asarray(Vown, dtype=np.float64).reshape(-1, N))
    Vp = np.ascontiguousarray(np.asarray(Vprev, dtype=np.float64).reshape(-1, N))
    V = np.zeros(max(cap_a, 1) * N)
    A = np.zeros(max(cap_a, 1) ** 2)
    u = lib().orc_accumulate(H, W, _p(_f64(C)), Vo.shape[0], _p(Vo.reshape(-1)), Vp.shape[0],
                             _p(Vp.reshape(-1)), cap_a, _p(V), _p(A))
    return V.reshape(-1, N)[:u].copy(), A[: u * u].reshape(u, u).copy()


def dense_lu_solve(A, b):
    """Dense LU with partial pivoting (tiny systems)."""
    n = A.shape[0]
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    b = _f64(b).copy()
    x = np.zeros(n)
    rc = lib().orc_dense_lu_solve(n, _p(A.reshape(-1)), _p(b), _p(x))
    if rc != 0:
        raise ArithmeticError("singular matrix")
    return x


MODE_PROJECTED, MODE_PLAIN, MODE_WARM, MODE_GALERKIN = 0, 1, 2, 3
MODE_GUESS_PROJECTED, MODE_GUESS = 4, 5   # a given initial guess, with / without projection


def project_galerkin(H, W, C, V, a, r, xinit=None):
    """Sec. 3, Phase 2 with the target's own operator: x0 = xinit + V_a G^{-1}
    V_a^T r, G = V_a^T A_i V_a (C: the target's coefficients, as from coeffs).
    Returns (x0, singular)."""
    N = H * W
    Vc = np.ascontiguousarray(np.asarray(V, dtype=np.float64)[:a].reshape(-1))
    x0 = np.zeros(N)
    rc = lib().orc_project_galerkin(H, W, _p(_f64(C)), a, _p(Vc), _p(_f64(r)), _p(_f64(xinit)),
                                    _p(x0))
    return x0, bool(rc)


@dataclass
class StepStats:
    seed_iters: np.ndarray
    tgt_iters: np.ndarray
    tgt_res: np.ndarray
    tgt_status: np.ndarray
    tgt_x0res: np.ndarray


SEED_GMRES, SEED_BICGSTAB = 0, 1


def march_step(H, W, dt, h, g2, mseed, mtgt, target_seed, mode=MODE_PROJECTED,
               tol_seed=1e-10, m_seed=40, a=40, tol_ref=1e-8, m_ref=40, maxit=1000, picard=1,
               seed_solver=SEED_GMRES, seed_prev=None, fixed_a=False, xinit=None):
    """One timestep of Sec. 2.3 + Sec. 3 for seeds and targets of one grid
    size (f = 0), with `picard` lagged-linearisation iterations; the seeds are
    solved by GMRES (Arnoldi basis) or BiCGSTAB (Sec. 3, Phase 1 as printed:
    its key vectors, A_proj = V^T A_seed V); ``seed_prev`` (seed cycling, Sec.
    5.2) links each seed to its predecessor (-1: none), whose accumulated basis
    it extends (``accumulate``).  ``mseed`` (nseed, N) and ``mtgt`` (ntgt, N)
    are updated in place from m^{n-1} to m^n.  ``fixed_a=True``: every seed
    basis has the fixed dimension min(a, m_seed) of Sec. 3 (see ``gmres``).
    ``xinit`` (ntgt, N): the targets' initial guesses for modes
    MODE_GUESS_PROJECTED (x0 = xinit + V_a H_a^{-1} V_a^T (b - A xinit), Sec. 3
    Phase 2 in residual form, unless the warm start m^{n-1} leaves a smaller
    residual than xinit: then x0 = m^{n-1}) and MODE_GUESS (x0 = xinit)."""
    assert mseed.dtype == np.float64 and mseed.flags["C_CONTIGUOUS"]
    assert mtgt.dtype == np.float64 and mtgt.flags["C_CONTIGUOUS"]
    ns, nt = mseed.shape[0], mtgt.shape[0]
    ts = np.ascontiguousarray(target_seed, dtype=np.int32)
    if mode in (MODE_GUESS_PROJECTED, MODE_GUESS):
        assert xinit is not None and xinit.shape == mtgt.shape
    xi = None if xinit is None else np.ascontiguousarray(xinit, dtype=np.float64)
    st = StepStats(np.zeros(ns, np.int32), np.zeros(nt, np.int32), np.zeros(nt),
                   np.zeros(nt, np.int32), np.zeros(nt))
    lib().orc_march_step(H, W, dt, h, g2, ns, _p(mseed), nt, _p(mtgt), _p(ts), mode,
                         tol_seed, m_seed, a, tol_ref, m_ref, maxit, _p(st.seed_iters),
                         _p(st.tgt_iters), _p(st.tgt_res), _p(st.tgt_status), _p(st.tgt_x0res),
                         int(picard), int(seed_solver),
                         _p(np.ascontiguousarray(seed_prev, dtype=np.int32))
                         if seed_prev is not None else None, int(bool(fixed_a)), _p(xi))
    return st


def march(H, W, T, g2, seeds, targets, target_seed, steps=None, **kw):
    """Time march n = 1..steps (default T) with dt = 1/T, h = 1/H (Sec. 2.3),
    from m^0 = the images.  Returns (m_seed^n, m_target^n, list of StepStats)."""
    dt, h = 1.0 / T, 1.0 / H
    ms = np.array(seeds, dtype=np.float64).reshape(len(seeds), -1).copy()
    mt = np.array(targets, dtype=np.float64).reshape(len(targets), -1).copy()
    stats = []
    for n in range(steps if steps is not None else T):
        stats.append(march_step(H, W, dt, h, float(g2[n]), ms, mt, target_seed, **kw))
    return ms, mt, stats


def score(H, W, h, m):
    """Central-difference score (sx, sy) of one solved channel (end of Sec. 2.3,
    divided by 2h), zero padding outside the grid."""
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(-1))
    sx = np.zeros(H * W)
    sy = np.zeros(H * W)
    lib().orc_score(H, W, h, _p(m), _p(sx), _p(sy))
    return sx, sy


def embed_step(dt, g2prev, sx, sy, ex, ey):
    """x^n = x^{n-1} + dt * (-(g^{n-1})^2 / 2) grad m^{n-1} (Sec. 4.1, f = 0), in place."""
    lib().orc_embed_step(len(ex), dt, g2prev, _p(sx), _p(sy), _p(ex), _p(ey))


def march_scores(H, W, T, g2, seeds, targets, target_seed, steps=None, **kw):
    """The march of `march` plus, for every target and timestep n, the score
    of m^n and the probability-flow embedding x^n (x^0 = 0), which advances
    with grad m^{n-1} and (g^{n-1})^2 (taken as (g^1)^2 for n = 1).
    Returns (m_seed, m_target, scores [steps][ntgt][2][N], embedding [ntgt][2][N])."""
    dt, h = 1.0 / T, 1.0 / H
    ms = np.array(seeds, dtype=np.float64).reshape(len(seeds), -1).copy()
    mt = np.array(targets, dtype=np.float64).reshape(len(targets), -1).copy()
    nt, N = mt.shape
    emb = np.zeros((nt, 2, N))
    scores = []
    for n in range(steps if steps is not None else T):
        g2prev = float(g2[max(n - 1, 0)])
        for k in range(nt):
            sx, sy = score(H, W, h, mt[k])
            embed_step(dt, g2prev, sx, sy, emb[k, 0], emb[k, 1])
        march_step(H, W, dt, h, float(g2[n]), ms, mt, target_seed, **kw)
        scores.append(np.stack([np.stack(score(H, W, h, mt[k])) for k in range(nt)]))
    return ms, mt, np.stack(scores), emb


def march_learned(H, W, T, g2, seeds, targets, target_seed, params, channels, steps=None,
                  project=True, operand_round=None, tol_seed=1e-10, m_seed=40, a=40,
                  fixed_a=False, maxit=1000, n0=0, **kw):
    """The march with the learned initial guess (``cnn_oracle.learned_guess``):
    at every timestep the seeds are solved first (the same GMRES solve the
    march step repeats), the network maps [m_i^{n-1}, m_seed^n, time planes]
    to x_init = m_i^{n-1} + s_n * net, and the targets start from x_init
    projected in residual form onto the seed basis (``project``; Sec. 3,
    Phase 2 applied to b - A x_init) -- or from the warm start m_i^{n-1}
    when that leaves a smaller residual than x_init -- or from x_init
    itself, then GMRES.
    The states are those of timestep n0 (the march runs n0+1 .. n0+steps).
    Returns (m_seed, m_target, list of StepStats)."""
    from . import cnn_oracle as R
    dt, h = 1.0 / T, 1.0 / H
    ms = np.array(seeds, dtype=np.float64).reshape(len(seeds), -1).copy()
    mt = np.array(targets, dtype=np.float64).reshape(len(targets), -1).copy()
    ts = np.asarray(target_seed, dtype=np.int64)
    stats = []
    for n in range(n0, n0 + (steps if steps is not None else T - n0)):
        g2n = float(g2[n])
        snew = np.empty_like(ms)
        for s in range(len(ms)):
            C = coeffs(H, W, g2n, dt, h, ms[s])
            snew[s] = gmres(H, W, C, rhs(H, W, dt, h, ms[s]), tol=tol_seed, m=m_seed, maxit=maxit,
                            capture=a, fixed=fixed_a).x
        xin = R.learned_guess(params, channels, mt, snew[ts], n + 1, T, g2n, H, W, operand_round)
        stats.append(march_step(H, W, dt, h, g2n, ms, mt, target_seed,
                                mode=MODE_GUESS_PROJECTED if project else MODE_GUESS,
                                tol_seed=tol_seed, m_seed=m_seed, a=a, maxit=maxit,
                                fixed_a=fixed_a, xinit=xin, **kw))
        assert np.array_equal(ms, snew)
    return ms, mt, stats
