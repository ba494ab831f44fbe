"""Python binding of the C ABI: the same calls as include/jkcals.h, taking NumPy
arrays (host) or torch tensors (host or CUDA).  It only marshals arguments;
every step of the computation runs in libjkcals.so.
"""
from __future__ import annotations

import ctypes as ct
from typing import List, Optional, Sequence

import numpy as np

from . import _lib as L

__all__ = ["JKCALS", "JKError", "from_workload", "left_out_csr", "multi_init"]

JKError = L.JKError


def _ptr(x) -> int:
    """Device or host address of a contiguous NumPy array / torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _dtype_code(x) -> int:
    name = str(x.dtype)
    if name.endswith("float64"):
        return L.DTYPE_F64
    if name.endswith("float32"):
        return L.DTYPE_F32
    raise TypeError(f"tensor dtype must be float32 or float64, got {x.dtype}")


def left_out_csr(left_out: Sequence[Sequence[int]]):
    ptr = np.zeros(len(left_out) + 1, dtype=np.int64)
    for g, D in enumerate(left_out):
        ptr[g + 1] = ptr[g] + len(D)
    idx = np.concatenate([np.asarray(D, dtype=np.int64) for D in left_out]) if ptr[-1] else np.zeros(1, np.int64)
    return ptr, np.ascontiguousarray(idx)


def multi_init(init_blocks: Sequence[Sequence[np.ndarray]]) -> List[np.ndarray]:
    """Concatenate per-block initial factors side by side (Alg. 3 initialisation)."""
    N = len(init_blocks[0])
    return [np.ascontiguousarray(np.concatenate([np.asarray(b[n], dtype=np.float64) for b in init_blocks], axis=1))
            for n in range(N)]


def init_from_model(U: Sequence[np.ndarray], K: int) -> List[np.ndarray]:
    """Initial multi-matrices of K jackknife submodels that all start from one fitted model U
    (I_n x R per mode, Alg. 2 and Alg. 3 initialisation).  The rows each submodel leaves out
    are zeroed by jkcals_create, so the model's factors are repeated unchanged."""
    return multi_init([list(U)] * int(K))


def _torch():
    import torch
    return torch


class JKCALS:
    """Handle of one jackknife problem (jkcals_create ... jkcals_destroy)."""

    def __init__(self, T, n_hat: int, ranks: Sequence[int], left_out: Sequence[Sequence[int]],
                 init: Sequence, *, precision: str = "fp64", normalise: bool = True,
                 use_graph: bool = True, splits: int = 0, max_device_bytes: int = 0,
                 kernel_timing: bool = False, update_mode: int = 0, autotune: bool = False, compact: bool = True,
                 batch_branches: bool = False, stream=None):
        lib = L.load()
        self._lib = lib
        self._h = ct.c_void_p()
        self.dims = tuple(int(d) for d in T.shape)
        self.N = len(self.dims)
        self.K = len(ranks)
        self.ranks = [int(r) for r in ranks]
        self.C = int(sum(self.ranks))
        self.n_hat = int(n_hat)
        self.precision = precision
        opt = L.Options()
        lib.jkcals_default_options(ct.byref(opt))
        opt.precision = L.PREC[precision]
        opt.normalise = int(bool(normalise))
        opt.use_graph = int(bool(use_graph))
        opt.splits = int(splits)
        opt.max_device_bytes = int(max_device_bytes)
        opt.kernel_timing = int(bool(kernel_timing))
        opt.update_mode = int(update_mode)
        opt.autotune = int(bool(autotune))
        opt.compact = int(bool(compact))
        opt.batch_branches = int(bool(batch_branches))
        dims = (ct.c_int64 * self.N)(*self.dims)
        rk = (ct.c_int32 * self.K)(*self.ranks)
        ptr, idx = left_out_csr(left_out)
        self._has_left_out = [bool(ptr[g + 1] > ptr[g]) for g in range(self.K)]
        self._keep = [T, ptr, idx, init]
        init_ptrs = (ct.c_void_p * self.N)(*[_ptr(u) for u in init])
        for n, u in enumerate(init):
            if tuple(u.shape) != (self.dims[n], self.C):
                raise ValueError(f"init[{n}] must be {self.dims[n]} x {self.C}")
            if "float64" not in str(u.dtype):
                raise TypeError("init factors must be float64")
        if stream is None and hasattr(T, "is_cuda") and T.is_cuda:
            stream = _torch().cuda.current_stream().cuda_stream
        st = L.check(lib.jkcals_create(ct.byref(self._h), self.N, dims, ct.c_void_p(_ptr(T)), _dtype_code(T),
                                       self.n_hat, self.K, rk,
                                       ptr.ctypes.data_as(L.I64P), idx.ctypes.data_as(L.I64P),
                                       init_ptrs, ct.byref(opt), ct.c_void_p(stream) if stream else None),
                     "jkcals_create")
        del st
        self._keep = None

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if self._h:
            self._lib.jkcals_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -------------------------------------------------------------------
    def _out(self, shape, device):
        if device is None or device == "cpu":
            return np.empty(shape, dtype=np.float64)
        torch = _torch()
        return torch.empty(shape, dtype=torch.float64, device=device)

    def mttkrp(self, mode: int, out=None, device=None):
        """Concurrent MTTKRP of Alg. 3 for the current factors: I_mode x C FP64."""
        if out is None:
            out = self._out((self.dims[mode], self.C), device)
        L.check(self._lib.jkcals_mttkrp(self._h, int(mode), ct.c_void_p(_ptr(out))), "jkcals_mttkrp")
        return out

    def als_sweep(self, nsweeps: int, losses=True, device=None, raise_not_spd: bool = False):
        """nsweeps JK-CALS sweeps; returns the nsweeps x K losses (or None)."""
        out = None
        if losses is True:
            out = self._out((nsweeps, self.K), device)
        elif losses is not None and losses is not False:
            out = losses
        st = self._lib.jkcals_als_sweep(self._h, int(nsweeps), ct.c_void_p(_ptr(out)) if out is not None else None)
        if st != L.ERR_NOT_SPD or raise_not_spd:
            L.check(st, "jkcals_als_sweep")
        return out

    def als_sweep_async(self, nsweeps: int, losses_dev=None):
        """Enqueue nsweeps sweeps without synchronising (losses_dev: CUDA tensor or None)."""
        L.check(self._lib.jkcals_als_sweep_async(self._h, int(nsweeps),
                                                 ct.c_void_p(_ptr(losses_dev)) if losses_dev is not None else None),
                "jkcals_als_sweep_async")
        return losses_dev

    def kernel_times(self):
        """Per-mode MTTKRP device time (ms) of the last completed sweep (kernel_timing=True)."""
        ms = (ct.c_double * self.N)()
        L.check(self._lib.jkcals_kernel_times(self._h, ms), "jkcals_kernel_times")
        return list(ms)

    def sweep_info(self):
        k = ct.c_int(0)
        sp = (ct.c_int * self.N)()
        L.check(self._lib.jkcals_sweep_info(self._h, ct.byref(k), sp), "jkcals_sweep_info")
        return k.value, list(sp)

    def mode_plan(self, mode: int):
        """How mode `mode`'s MTTKRP runs: kernel ('fp64', 'tensor-core' or 'two-step'),
        rows per CTA, pipeline stages and the fastest other mode of the operand layout."""
        k, bn, st, fm = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        L.check(self._lib.jkcals_mode_plan(self._h, int(mode), ct.byref(k), ct.byref(bn), ct.byref(st),
                                           ct.byref(fm)), "jkcals_mode_plan")
        return {"kernel": ("fp64", "tensor-core", "two-step")[k.value], "tile_rows": bn.value,
                "stages": st.value, "fastest_mode": fm.value}

    def run(self, max_sweeps: int, tol: float = 0.0):
        done = ct.c_int(0)
        fl = np.empty(self.K, dtype=np.float64)
        st = self._lib.jkcals_run(self._h, int(max_sweeps), float(tol), ct.byref(done), ct.c_void_p(fl.ctypes.data))
        if st != L.ERR_NOT_SPD:
            L.check(st, "jkcals_run")
        return done.value, fl

    def run_block_sweeps(self):
        """Sweeps each block ran in the latest run() (K ints): where a block converged
        (or met a non-positive pivot) and was frozen."""
        out = np.empty(self.K, dtype=np.int32)
        L.check(self._lib.jkcals_run_block_sweeps(self._h, out.ctypes.data_as(ct.POINTER(ct.c_int32))),
                "jkcals_run_block_sweeps")
        return out

    def get_factors_into(self, outs):
        return self.get_factors(outs=outs)

    def get_factors(self, device=None, outs=None):
        if outs is None:
            outs = [self._out((I, self.C), device) for I in self.dims]
        arr = (ct.c_void_p * self.N)(*[_ptr(o) for o in outs])
        L.check(self._lib.jkcals_get_factors(self._h, arr), "jkcals_get_factors")
        return outs

    def set_factors(self, U):
        arr = (ct.c_void_p * self.N)(*[_ptr(u) for u in U])
        L.check(self._lib.jkcals_set_factors(self._h, arr), "jkcals_set_factors")

    def jackknife_se(self, ref_block: Optional[int] = None, ref=None):
        """Alg. 2 post-processing on the device: the submodels (blocks with left-out rows)
        adjusted to a reference model, and the jackknife standard errors.  The reference is
        block ``ref_block``'s factors or the factor list ``ref`` (I_n x R each).  Returns
        (S, perm, aligned): S[n] is I_n x R (None for the sampled mode), perm is G x R
        (reference column s <- submodel column perm[g, s]), aligned[n] is G x I_n x R."""
        sub = [g for g in range(self.K) if self._has_left_out[g]]
        if not sub:
            raise ValueError("no submodel has left-out rows")
        R = self.ranks[sub[0]]
        G = len(sub)
        S = [None if n == self.n_hat else np.empty((I, R)) for n, I in enumerate(self.dims)]
        perm = np.empty((G, R), dtype=np.int32)
        aligned = [np.empty((G, I, R)) for I in self.dims]
        refs = None
        if ref_block is None:
            if ref is None:
                raise ValueError("give ref_block or ref")
            refs = [np.ascontiguousarray(r, dtype=np.float64) for r in ref]
            refarr = (ct.c_void_p * self.N)(*[_ptr(r) for r in refs])
        else:
            refarr = None
        Sarr = (ct.c_void_p * self.N)(*[None if s is None else _ptr(s) for s in S])
        Aarr = (ct.c_void_p * self.N)(*[_ptr(a) for a in aligned])
        got = ct.c_int(0)
        L.check(self._lib.jkcals_jackknife_se(self._h, -1 if ref_block is None else int(ref_block), refarr, Sarr,
                                              ct.c_void_p(_ptr(perm)), Aarr, ct.byref(got)), "jkcals_jackknife_se")
        if got.value != G:
            raise RuntimeError(f"jkcals_jackknife_se counted {got.value} submodels, expected {G}")
        return S, perm, aligned

    def block_status(self):
        st = np.zeros(self.K, dtype=np.int32)
        L.check(self._lib.jkcals_get_block_status(self._h, st.ctypes.data_as(L.I32P)), "jkcals_get_block_status")
        return st

    def grad(self, U=None, G=None, device=None, want_grad: bool = True):
        """Summed jackknife loss and its gradient w.r.t. the multi-matrices."""
        Uarr = (ct.c_void_p * self.N)(*[_ptr(u) for u in U]) if U is not None else None
        if want_grad and G is None:
            G = [self._out((I, self.C), device) for I in self.dims]
        Garr = (ct.c_void_p * self.N)(*[_ptr(g) for g in G]) if G is not None else None
        loss = ct.c_double(0.0)
        L.check(self._lib.jkcals_grad(self._h, Uarr, Garr, ct.byref(loss)), "jkcals_grad")
        return loss.value, G

    def sync(self):
        L.check(self._lib.jkcals_sync(self._h), "jkcals_sync")

    def loss_history(self, nsweeps: int, device=None):
        """Losses of the last ``nsweeps`` sweeps of the latest sweep call (nsweeps x K)."""
        out = self._out((nsweeps, self.K), device)
        L.check(self._lib.jkcals_loss_history(self._h, int(nsweeps), ct.c_void_p(_ptr(out))),
                "jkcals_loss_history")
        return out

    def loss(self, U):
        """Differentiable summed jackknife loss f(U) = sum_g ||T_{-g} - [[U_{|g}]]||^2
        as a 0-dim FP64 CUDA tensor; U is the list of N multi-matrices (FP64 CUDA,
        I_n x C).  Its backward is the hand-written jkcals_grad (concurrent MTTKRP
        minus U times the Hadamard of Grams)."""
        return _loss_function().apply(self, *U)


class Batch:
    """Many independent problems advanced together: one CUDA graph per sweep of
    the whole batch, of grouped launches over all problems or of one branch per
    problem (jkcals_batch_create / _sweep / _sync / _destroy).  The handles stay
    owned by the caller and must outlive the batch."""

    def __init__(self, handles: Sequence[JKCALS], max_sweeps: int, stream=None):
        self._lib = L.load()
        self.handles = list(handles)
        self.max_sweeps = int(max_sweeps)
        self._b = ct.c_void_p()
        arr = (ct.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        L.check(self._lib.jkcals_batch_create(ct.byref(self._b), len(self.handles), arr, self.max_sweeps,
                                              ct.c_void_p(stream) if stream else None), "jkcals_batch_create")

    def sweep(self, nsweeps: int):
        L.check(self._lib.jkcals_batch_sweep(self._b, int(nsweeps)), "jkcals_batch_sweep")

    def sync(self):
        L.check(self._lib.jkcals_batch_sync(self._b), "jkcals_batch_sync")

    def close(self):
        if self._b:
            self._lib.jkcals_batch_destroy(self._b)
            self._b = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_LOSS_FN = None


def _loss_function():
    """torch.autograd.Function for JKCALS.loss, built on first use (torch is
    imported lazily).  forward: the loss only (one MTTKRP, of the last mode);
    backward: all N MTTKRPs through jkcals_grad, scaled by the incoming grad."""
    global _LOSS_FN
    if _LOSS_FN is not None:
        return _LOSS_FN
    torch = _torch()

    class JKLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, h, *U):
            U = [u.detach().contiguous() for u in U]
            for u in U:
                if u.dtype != torch.float64 or not u.is_cuda:
                    raise TypeError("JKCALS.loss takes FP64 CUDA tensors")
            torch.cuda.current_stream().synchronize()   # the library runs on its own stream
            f, _ = h.grad(U=U, want_grad=False)
            ctx.h = h
            ctx.save_for_backward(*U)
            return torch.tensor(f, dtype=torch.float64, device=U[0].device)

        @staticmethod
        def backward(ctx, gout):
            U = ctx.saved_tensors
            G = [torch.empty_like(u) for u in U]
            torch.cuda.current_stream().synchronize()
            ctx.h.grad(U=list(U), G=G)
            return (None, *[gout * g for g in G])

    _LOSS_FN = JKLoss
    return _LOSS_FN


def selftest_bounded_wait(limit_ms: float = 20.0):
    """jkcals_selftest_bounded_wait: runs the bounded-wait self-test on the current
    device; returns (status, error code recorded, ms until the second waiter left)."""
    lib = L.load()
    code = ct.c_int32(0)
    left = ct.c_double(0.0)
    st = lib.jkcals_selftest_bounded_wait(float(limit_ms), ct.byref(code), ct.byref(left))
    return int(st), int(code.value), float(left.value)


def plan_query(dims: Sequence[int], ranks: Sequence[int], precision: str = "fp64", splits: int = 0,
               num_sms: int = 152):
    """The per-mode plan jkcals_create would make (host only, no device): kernel ('fp64',
    'tensor-core' or 'two-step'), rows per CTA, pipeline stages and split-K factor."""
    lib = L.load()
    N, K = len(dims), len(ranks)
    opt = L.Options()
    lib.jkcals_default_options(ct.byref(opt))
    opt.precision = L.PREC[precision]
    opt.splits = int(splits)
    d = (ct.c_int64 * N)(*[int(x) for x in dims])
    rk = (ct.c_int32 * K)(*[int(r) for r in ranks])
    out = [(ct.c_int32 * N)() for _ in range(4)]
    L.check(lib.jkcals_plan_query(N, d, K, rk, ct.byref(opt), int(num_sms), *out), "jkcals_plan_query")
    kinds = ("fp64", "tensor-core", "two-step")
    return [{"kernel": kinds[out[0][n]], "tile_rows": out[1][n], "stages": out[2][n], "splits": out[3][n]}
            for n in range(N)]


def from_workload(w, precision: str = "fp64", device: Optional[str] = None, **kw) -> JKCALS:
    """Handle for a ``workloads.Workload`` (tensor in its dtype, init side by side)."""
    T = w.T.astype(np.float32) if w.dtype == "f32" else w.T
    T = np.ascontiguousarray(T)
    init = multi_init(w.init)
    if device is not None and device != "cpu":
        torch = _torch()
        T = torch.from_numpy(T).to(device)
        init = [torch.from_numpy(u).to(device) for u in init]
    return JKCALS(T, w.n_hat, w.ranks, w.left_out, init, precision=precision, **kw)


def _check_noalloc_args(Tn, U, mode: int, out):
    """Shapes, dtypes and devices of jkcals_mttkrp_f64_noalloc's arguments: the
    C ABI sees only pointers, so a mis-sized buffer would be read or written past
    its end.  Returns (dims, C).  Raises ValueError."""
    N = len(U)
    if not 2 <= N <= 8:
        raise ValueError("U must hold 2 to 8 factor matrices")
    if not 0 <= mode < N:
        raise ValueError("mode out of range")
    others = [k for k in range(N) if k != mode]
    tensors = [("Tn", Tn), ("out", out)] + [(f"U[{k}]", U[k]) for k in others]
    for name, t in tensors:
        if t is None:
            raise ValueError(f"{name} is missing")
        if t.dtype != _torch().float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if t.dim() != 2:
            raise ValueError(f"{name} must be a matrix")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous (row-major)")
    devs = {t.device for _, t in tensors}
    if len(devs) != 1:
        raise ValueError("Tn, out and the factor matrices must be on one device")
    C = int(U[others[0]].shape[1])
    dims = [0] * N
    dims[mode] = int(Tn.shape[0])
    for k in others:
        if int(U[k].shape[1]) != C:
            raise ValueError(f"U[{k}] has {U[k].shape[1]} columns, expected C = {C}")
        dims[k] = int(U[k].shape[0])
    J = 1
    for k in others:
        J *= dims[k]
    if tuple(Tn.shape) != (dims[mode], J):
        raise ValueError(f"Tn must be {dims[mode]} x {J} (the mode-{mode} unfolding), got {tuple(Tn.shape)}")
    if tuple(out.shape) != (dims[mode], C):
        raise ValueError(f"out must be {dims[mode]} x {C}, got {tuple(out.shape)}")
    if U[mode] is not None and tuple(U[mode].shape) != (dims[mode], C):
        raise ValueError(f"U[{mode}] must be {dims[mode]} x {C} or None")
    return dims, C


def mttkrp_f64_noalloc(Tn, U, mode: int, out, stream=None):
    """FP64 concurrent MTTKRP of one mode without any device allocation
    (jkcals_mttkrp_f64_noalloc): Tn is the I_mode x J unfolding, U the N factor
    matrices (I_k x C; U[mode] is not read and may be None), out the I_mode x C
    result; float64 CUDA tensors on one device, contiguous.  Enqueued on
    ``stream`` (default: torch's current stream), not synchronised."""
    dims, C = _check_noalloc_args(Tn, U, mode, out)
    lib = L.load()
    N = len(U)
    d = (ct.c_int64 * N)(*dims)
    ptrs = (ct.c_void_p * N)(*[(_ptr(u) if (k != mode and u is not None) else None) for k, u in enumerate(U)])
    if stream is None:   # host tensors reach the C ABI, which rejects them
        stream = _torch().cuda.current_stream(Tn.device).cuda_stream if Tn.is_cuda else 0
    L.check(lib.jkcals_mttkrp_f64_noalloc(N, d, int(mode), ct.c_void_p(_ptr(Tn)), ptrs, C,
                                          ct.c_void_p(_ptr(out)), ct.c_void_p(stream)),
            "jkcals_mttkrp_f64_noalloc")
    return out
