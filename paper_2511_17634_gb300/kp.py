"""Thin Python binding of the C ABI in ``include/kp.h`` (argument marshalling
only; every step of the solver runs in the CUDA library ``libkp.so``).

Vectors are CUDA ``torch.float64`` tensors.  A batch of systems of one grid
size is a 2-D tensor ``(nsys, N)``; a list of 1-D tensors also works.  The
library must have been built (``paper_2511_17634_gb300.build``); importing
this module without it raises ``ImportError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkp.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NO_BASIS, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
ERR_TOO_LARGE = -7
PREC_FP64, PREC_MIXED = 0, 1


class KPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"kp status {status}: {msg}")
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("max_seeds", ctypes.c_int), ("max_a", ctypes.c_int), ("max_n", ctypes.c_int),
                ("precision", ctypes.c_int), ("smem_vectors", ctypes.c_int),
                ("reorth", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("cluster_size", ctypes.c_int),
                ("fixed_a", ctypes.c_int), ("inner_digits", ctypes.c_int),
                ("cluster_blocks_per_sm", ctypes.c_int)]


# kp_op: int H, W; double dt, g2, h; const double *mtilde, *fx, *fy
OP_DTYPE = np.dtype({"names": ["H", "W", "dt", "g2", "h", "mt", "fx", "fy"],
                     "formats": [np.int32, np.int32, np.float64, np.float64, np.float64,
                                 np.uint64, np.uint64, np.uint64],
                     "offsets": [0, 4, 8, 16, 24, 32, 40, 48], "itemsize": 56})

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2511_17634_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.kp_options_default.argtypes = [ctypes.POINTER(_Options)]
        L.kp_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Options), vp]
        L.kp_destroy.argtypes = [vp]
        L.kp_set_stream.argtypes = [vp, vp]
        L.kp_last_error.argtypes = [vp]
        L.kp_last_error.restype = ctypes.c_char_p
        L.kp_version.restype = ctypes.c_char_p
        L.kp_apply.argtypes = [vp, i, vp, vp, vp]
        L.kp_rhs.argtypes = [vp, i, vp, vp, vp]
        L.kp_seed_solve.argtypes = [vp, i, vp, vp, vp, d, i, i, vp]
        L.kp_refine.argtypes = [vp, i, vp, vp, vp, d, i, i, vp]
        L.kp_store_basis.argtypes = [vp, i, i, i]
        L.kp_project_targets.argtypes = [vp, i, i, i, vp, vp, vp]
        L.kp_project_targets_multi.argtypes = [vp, i, i, vp, vp, vp, vp]
        L.kp_basis_get.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), vp, vp]
        L.kp_project_gemm_bf16.argtypes = [vp, i, i, i, vp, i, vp, i, vp, i]
        L.kp_residual.argtypes = [vp, i, vp, vp, vp, vp]
        L.kp_measure_alu_peaks.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
        f32 = ctypes.c_float
        L.kp_cnn_create.argtypes = [vp, i, i, i, i, vp, ctypes.POINTER(vp)]
        L.kp_cnn_destroy.argtypes = [vp]
        L.kp_cnn_num_params.argtypes = [vp]
        L.kp_cnn_set_params.argtypes = [vp, vp]
        L.kp_cnn_get_params.argtypes = [vp, vp]
        L.kp_cnn_forward.argtypes = [vp, i, vp, vp]
        L.kp_cnn_gradients.argtypes = [vp, i, vp, vp, vp, vp]
        L.kp_cnn_train_step.argtypes = [vp, i, vp, vp, f32, f32, f32, f32, i, vp]
        L.kp_cnn_pack_inputs.argtypes = [vp, i, vp, vp, i, i, d, vp, vp]
        L.kp_cnn_add_guess.argtypes = [vp, i, vp, vp, vp, d, vp]
        L.kp_cnn_pack_target.argtypes = [vp, i, vp, vp, vp, d, vp]
        L.kp_cnn_set_inference_batch.argtypes = [vp, i]
        for f in ("kp_create", "kp_destroy", "kp_set_stream", "kp_apply", "kp_rhs", "kp_seed_solve",
                  "kp_refine", "kp_store_basis", "kp_project_targets", "kp_project_targets_multi",
                  "kp_basis_get", "kp_project_gemm_bf16", "kp_residual", "kp_measure_alu_peaks", "kp_cnn_create",
                  "kp_cnn_destroy", "kp_cnn_num_params", "kp_cnn_set_params", "kp_cnn_get_params",
                  "kp_cnn_forward", "kp_cnn_gradients", "kp_cnn_train_step", "kp_cnn_pack_inputs",
                  "kp_cnn_add_guess", "kp_cnn_pack_target", "kp_cnn_set_inference_batch"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


def version() -> str:
    return lib().kp_version().decode()


def ptrs(vs):
    """Host array of device pointers for a 2-D tensor (rows), a list of tensors,
    or an array of pointers made by an earlier call (returned unchanged)."""
    import torch
    if isinstance(vs, np.ndarray):
        assert vs.dtype == np.uint64 and vs.ndim == 1
        return np.ascontiguousarray(vs)
    if isinstance(vs, torch.Tensor):
        assert vs.is_cuda and vs.dtype == torch.float64 and vs.dim() == 2 and vs.stride(1) == 1
        base = vs.data_ptr()
        arr = (np.arange(vs.shape[0], dtype=np.uint64) * np.uint64(vs.stride(0) * 8)
               + np.uint64(base))
    else:
        for v in vs:
            assert v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()
        arr = np.array([v.data_ptr() for v in vs], dtype=np.uint64)
    return np.ascontiguousarray(arr)


class Ops:
    """Host array of kp_op descriptors plus references to the tensors they
    point to (so that those stay alive while the descriptors are in use)."""

    def __init__(self, arr, refs):
        self.arr = arr
        self.refs = refs

    def __len__(self):
        return len(self.arr)

    @staticmethod
    def concat(parts):
        return Ops(np.concatenate([p.arr for p in parts]), tuple(r for p in parts for r in p.refs))


def make_ops(H, W, dt, g2, h, mtilde, fx=None, fy=None):
    """kp_op descriptors for systems of one grid size; dt, g2, h may be
    per-system arrays."""
    mt = ptrs(mtilde)
    n = len(mt)
    ops = np.zeros(n, dtype=OP_DTYPE)
    ops["H"], ops["W"] = H, W
    ops["dt"], ops["g2"], ops["h"] = dt, g2, h
    ops["mt"] = mt
    ops["fx"] = ptrs(fx) if fx is not None else 0
    ops["fy"] = ptrs(fy) if fy is not None else 0
    return Ops(ops, (mtilde, fx, fy))


def info_tensor(nsys, device="cuda"):
    import torch
    return torch.zeros((nsys, 2), dtype=torch.float64, device=device)


def decode_info(info):
    """(iters, status, rel_res) numpy arrays from an info tensor."""
    a = info.detach().cpu().numpy()
    i32 = a.view(np.int32).reshape(a.shape[0], 4)
    return i32[:, 0].copy(), i32[:, 1].copy(), a[:, 1].copy()


class Context:
    """A kp_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, max_seeds=64, max_a=40, max_n=4096, precision=PREC_FP64, smem_vectors=0,
                 reorth=0, stream=None, block_threads=0, blocks_per_sm=0, cluster_size=0,
                 fixed_a=False, inner_digits=0, cluster_blocks_per_sm=0):
        import torch
        L = lib()
        o = _Options()
        L.kp_options_default(ctypes.byref(o))
        o.max_seeds, o.max_a, o.max_n = max_seeds, max_a, max_n
        o.precision, o.smem_vectors, o.reorth = precision, smem_vectors, reorth
        o.block_threads = block_threads
        o.blocks_per_sm = blocks_per_sm
        o.cluster_size = cluster_size
        o.fixed_a = int(bool(fixed_a))
        o.inner_digits = int(inner_digits)
        o.cluster_blocks_per_sm = int(cluster_blocks_per_sm)
        self._h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        st = L.kp_create(ctypes.byref(self._h), ctypes.byref(o), ctypes.c_void_p(s.cuda_stream))
        if st != OK:
            raise KPError(st, "kp_create failed")

    def close(self):
        if self._h:
            lib().kp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise KPError(st, lib().kp_last_error(self._h).decode())

    @staticmethod
    def _arr(a):
        if isinstance(a, Ops):
            a = a.arr
        return a.ctypes.data_as(ctypes.c_void_p)

    def apply(self, ops, x, y):
        self._check(lib().kp_apply(self._h, len(ops), self._arr(ops), self._arr(ptrs(x)),
                                   self._arr(ptrs(y))))

    def rhs(self, ops, mprev, b):
        self._check(lib().kp_rhs(self._h, len(ops), self._arr(ops), self._arr(ptrs(mprev)),
                                 self._arr(ptrs(b))))

    def seed_solve(self, ops, b, x, tol=1e-10, m=40, maxit=1000, info=None):
        if info is None:
            info = info_tensor(len(ops))
        self._check(lib().kp_seed_solve(self._h, len(ops), self._arr(ops), self._arr(ptrs(b)),
                                        self._arr(ptrs(x)), tol, m, maxit,
                                        ctypes.c_void_p(info.data_ptr())))
        return info

    def refine(self, ops, b, x, tol=1e-8, m=40, maxit=1000, info=None):
        if info is None:
            info = info_tensor(len(ops))
        self._check(lib().kp_refine(self._h, len(ops), self._arr(ops), self._arr(ptrs(b)),
                                    self._arr(ptrs(x)), tol, m, maxit,
                                    ctypes.c_void_p(info.data_ptr())))
        return info

    def store_basis(self, seed_id, timestep, sys):
        self._check(lib().kp_store_basis(self._h, seed_id, timestep, sys))

    def project_targets(self, seed_id, timestep, ops, r, x):
        self._check(lib().kp_project_targets(self._h, seed_id, timestep, len(ops), self._arr(ops),
                                             self._arr(ptrs(r)), self._arr(ptrs(x))))

    def project_targets_multi(self, timestep, seed_ids, ops, r, x):
        ids = np.ascontiguousarray(seed_ids, dtype=np.int32)
        self._check(lib().kp_project_targets_multi(self._h, timestep, len(ops), self._arr(ids),
                                                   self._arr(ops), self._arr(ptrs(r)),
                                                   self._arr(ptrs(x))))

    def measure_alu_peaks(self):
        """(FP64, FP32) FMA throughput of this GPU in TFLOP/s, measured."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(lib().kp_measure_alu_peaks(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def residual(self, ops, b, x, r):
        """r = b - A x (FP64)."""
        self._check(lib().kp_residual(self._h, len(ops), self._arr(ops), self._arr(ptrs(b)),
                                      self._arr(ptrs(x)), self._arr(ptrs(r))))

    def project_gemm_bf16(self, B, V, C, K=None):
        """C[t][i] = sum_k B[t][k] V[i][k] on the tensor cores (BF16 in, FP32 out)."""
        import torch
        assert B.dtype == torch.bfloat16 and V.dtype == torch.bfloat16 and C.dtype == torch.float32
        K = B.shape[1] if K is None else K
        self._check(lib().kp_project_gemm_bf16(self._h, B.shape[0], V.shape[0], K,
                                               ctypes.c_void_p(B.data_ptr()), B.stride(0),
                                               ctypes.c_void_p(V.data_ptr()), V.stride(0),
                                               ctypes.c_void_p(C.data_ptr()), C.stride(0)))

    def basis_get(self, seed_id, timestep, N):
        """(a, has_next, V (a+has_next, N) tensor, Hbar (a+1, a) numpy)."""
        import torch
        a = ctypes.c_int()
        hn = ctypes.c_int()
        self._check(lib().kp_basis_get(self._h, seed_id, timestep, ctypes.byref(a),
                                       ctypes.byref(hn), None, None))
        V = torch.zeros((a.value + hn.value, N), dtype=torch.float64, device="cuda")
        Hb = np.zeros((a.value + 1) * max(a.value, 1))
        self._check(lib().kp_basis_get(self._h, seed_id, timestep, None, None,
                                       ctypes.c_void_p(V.data_ptr()) if V.numel() else None,
                                       self._arr(Hb)))
        Hbar = Hb[: (a.value + 1) * a.value].reshape(a.value, a.value + 1).T.copy()
        return a.value, hn.value, V, Hbar


# ---------------------------------------------------------------- time march
MARCH_PROJECTED, MARCH_PLAIN, MARCH_WARM, MARCH_GALERKIN = 0, 1, 2, 3
MARCH_LEARNED, MARCH_LEARNED_ONLY = 4, 5
SEED_GMRES, SEED_BICGSTAB = 0, 1


class _Group(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("nseed", ctypes.c_int),
                ("ntgt", ctypes.c_int), ("m_seed", ctypes.c_void_p), ("m_tgt", ctypes.c_void_p),
                ("tgt_seed", ctypes.c_void_p), ("seed_prev", ctypes.c_void_p)]


class _MarchOpts(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("g2", ctypes.c_void_p), ("mode", ctypes.c_int),
                ("tol_seed", ctypes.c_double), ("tol", ctypes.c_double), ("m_seed", ctypes.c_int),
                ("m", ctypes.c_int), ("maxit", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("window", ctypes.c_int), ("target_blocks", ctypes.c_int),
                ("score", ctypes.c_void_p), ("embed", ctypes.c_void_p), ("picard", ctypes.c_int),
                ("seed_solver", ctypes.c_int), ("wait_probe", ctypes.c_int), ("maxit_seed", ctypes.c_int),
                ("cnn", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("seed_iters", "tgt_iters", "tgt_iters_max",
                                                "not_converged", "max_rel_res", "refine_flops",
                                                "seed_flops", "proj_flops", "refine_flops32")]


class MarchTiming(ctypes.Structure):
    _fields_ = [("seed_ms", ctypes.c_float), ("store_ms", ctypes.c_float),
                ("proj_ms", ctypes.c_float), ("refine_ms", ctypes.c_float),
                ("step_ms", ctypes.c_float), ("launches", ctypes.c_int)]


def _march_lib():
    L = lib()
    if not hasattr(L, "_march_ready"):
        vp = ctypes.c_void_p
        L.kp_march_create.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(_MarchOpts),
                                      ctypes.POINTER(vp)]
        L.kp_march_run.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.kp_march_destroy.argtypes = [vp]
        for f in ("kp_march_create", "kp_march_run", "kp_march_destroy"):
            getattr(L, f).restype = ctypes.c_int
        L._march_ready = True
    return L


class March:
    """Time march over groups of (seed, target) channel planes of one grid size
    each.  groups: list of (seeds (ns, N) tensor, targets (nt, N) tensor,
    target_seed int array, H, W[, seed_prev int array]); seed_prev links each
    seed to the one whose basis it extends (seed cycling, -1: none).  The
    tensors are updated in place by run()."""

    def __init__(self, ctx, groups, T, g2, mode=MARCH_PROJECTED, tol_seed=1e-10, tol=1e-8,
                 m_seed=40, m=40, maxit=1000, use_graph=True, window=0, target_blocks=0,
                 score=None, embed=None, picard=1, seed_solver=0, wait_probe=False, cnn=None,
                 maxit_seed=0):
        L = _march_lib()
        self.ctx = ctx
        self._keep = []
        arr = (_Group * len(groups))()
        for k, grp in enumerate(groups):
            s, t, ts, H, W = grp[:5]
            sp = grp[5] if len(grp) > 5 else None
            ts = np.ascontiguousarray(ts, dtype=np.int32)
            self._keep += [s, t, ts]
            if sp is not None:
                sp = np.ascontiguousarray(sp, dtype=np.int32)
                self._keep.append(sp)
                arr[k].seed_prev = sp.ctypes.data
            arr[k].H, arr[k].W = H, W
            arr[k].nseed, arr[k].ntgt = s.shape[0], t.shape[0]
            arr[k].m_seed = s.data_ptr() if s.numel() else None
            arr[k].m_tgt = t.data_ptr() if t.numel() else None
            arr[k].tgt_seed = ts.ctypes.data if len(ts) else None
        g2 = np.ascontiguousarray(g2, dtype=np.float64)
        self._keep.append(g2)
        # optional score output [T][targets][2][H*W] and embedding state
        # [targets][2][H*W] (CUDA float64, groups in order)
        for a in (score, embed):
            if a is not None:
                import torch
                assert a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                self._keep.append(a)
        o = _MarchOpts(T, g2.ctypes.data, mode, tol_seed, tol, m_seed, m, maxit, int(use_graph),
                       int(window), int(target_blocks),
                       score.data_ptr() if score is not None else None,
                       embed.data_ptr() if embed is not None else None, int(picard),
                       int(seed_solver), int(wait_probe), int(maxit_seed),
                       cnn._h if cnn is not None else None)
        if cnn is not None:
            self._keep.append(cnn)
        self.T = T
        self._h = ctypes.c_void_p()
        ctx._check(L.kp_march_create(ctx._h, len(groups), ctypes.cast(arr, ctypes.c_void_p),
                                     ctypes.byref(o), ctypes.byref(self._h)))

    def run(self, n0, steps, stats=False, timing=False):
        """Timesteps n0+1..n0+steps.  Returns (stats list or None, timing or None)."""
        L = _march_lib()
        st = (StepStats * steps)() if stats else None
        tm = MarchTiming() if timing else None
        self.ctx._check(L.kp_march_run(self._h, n0, steps,
                                       ctypes.cast(st, ctypes.c_void_p) if st is not None else None,
                                       ctypes.byref(tm) if tm is not None else None))
        return st, tm

    def close(self):
        if self._h:
            _march_lib().kp_march_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CNN:
    """The learned-initial-guess network on the GPU (kp_cnn_*)."""

    def __init__(self, ctx, H, W, channels=(6, 32, 32, 32, 1), max_batch=16):
        L = lib()
        self.ctx = ctx
        ch = (ctypes.c_int * len(channels))(*channels)
        self._h = ctypes.c_void_p()
        ctx._check(L.kp_cnn_create(ctx._h, H, W, max_batch, len(channels) - 1,
                                   ctypes.cast(ch, ctypes.c_void_p), ctypes.byref(self._h)))
        self.H, self.W, self.channels, self.max_batch = H, W, tuple(channels), max_batch
        self.nparams = L.kp_cnn_num_params(self._h)
        self.inference_batch = max_batch

    def close(self):
        if self._h:
            lib().kp_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        self.ctx._check(lib().kp_cnn_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        self.ctx._check(lib().kp_cnn_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def set_inference_batch(self, B):
        """Size the inference buffers (forward and the learned march) for B images."""
        self.ctx._check(lib().kp_cnn_set_inference_batch(self._h, int(B)))
        self.inference_batch = int(B)

    def forward(self, x, out):
        """x: CUDA float32 [B][c0][H*W]; out: CUDA float32 [B][cL][H*W]."""
        self.ctx._check(lib().kp_cnn_forward(self._h, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr())))

    def gradients(self, x, target, grads=None):
        loss = ctypes.c_double()
        self.ctx._check(lib().kp_cnn_gradients(
            self._h, x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
            ctypes.c_void_p(grads.data_ptr()) if grads is not None else None, ctypes.byref(loss)))
        return loss.value

    def pack_inputs(self, mprev, seed, n, T, g2n, out, rho):
        """out [B][10][H*W] float32 from FP64 lagged-field and seed-state planes
        (rows or lists) at timestep n of T with (g^n)^2 = g2n; rho (CUDA
        float64 [B]) receives each sample's step-residual rms."""
        pi, ps = ptrs(mprev), ptrs(seed)
        self.ctx._check(lib().kp_cnn_pack_inputs(self._h, len(pi), pi.ctypes.data_as(ctypes.c_void_p),
                                                 ps.ctypes.data_as(ctypes.c_void_p), int(n), int(T),
                                                 float(g2n), ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(rho.data_ptr())))

    def pack_target(self, a, b, out, scale=1.0, rho=None):
        """out [B][1][H*W] float32 = (a - b) * scale / rho_b (FP64 planes; rho
        CUDA float64 [B] or None)."""
        pa, pb = ptrs(a), ptrs(b)
        self.ctx._check(lib().kp_cnn_pack_target(self._h, len(pa), pa.ctypes.data_as(ctypes.c_void_p),
                                                 pb.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.c_void_p(rho.data_ptr()) if rho is not None else None,
                                                 float(scale), ctypes.c_void_p(out.data_ptr())))

    def add_guess(self, delta, base, x, scale=1.0, rho=None):
        """x = base + scale * rho_b * delta (FP64 planes; delta float32
        [B][1][H*W]; rho CUDA float64 [B] or None)."""
        pb, px = ptrs(base), ptrs(x)
        self.ctx._check(lib().kp_cnn_add_guess(self._h, len(pb), ctypes.c_void_p(delta.data_ptr()),
                                               pb.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.c_void_p(rho.data_ptr()) if rho is not None else None,
                                               float(scale), px.ctypes.data_as(ctypes.c_void_p)))

    def train_step(self, x, target, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        loss = ctypes.c_double()
        self.ctx._check(lib().kp_cnn_train_step(
            self._h, x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
            lr, beta1, beta2, eps, t, ctypes.byref(loss)))
        return loss.value
