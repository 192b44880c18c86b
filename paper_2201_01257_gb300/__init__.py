"""GB300 (sm_103a) block-sparse tensor contractions after TAMM (arXiv:2201.01257).

Thin Python binding over the C ABI in ``include/tamm_gb300.h``: the functions
``tamm_*`` below have the same names and arguments as the C entry points and
only marshal arguments; every step of a contraction runs in the library's CUDA
kernels.  PyTorch provides device memory (tensor storage and the library's
scratch, through its caching allocator) and the CUDA stream.

There is no CPU path: if the CUDA library cannot be built or loaded, or no GPU
is present, calls raise instead of falling back.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading
import types

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

TAMM_OK, TAMM_EINVAL, TAMM_ENOMEM, TAMM_ECUDA, TAMM_EUNSUPPORTED, TAMM_ETIMEOUT, TAMM_ECHECK, TAMM_ELIMIT = range(8)
TAMM_SYM_DENSE, TAMM_SYM_SPIN, TAMM_SYM_SPIN_IRREP = 0, 1, 2
TAMM_PREC_F64, TAMM_PREC_OZAKI_BF16, TAMM_PREC_OZAKI_I8, TAMM_PREC_BF16X3 = 0, 1, 2, 3
KERNEL_CLASSES = ("add", "reduce", "gemm_f64", "slice", "gemm_ozaki", "split_reduce", "triples")
(TAMM_OPT_OZAKI_CHUNK_K, TAMM_OPT_OZAKI_PERSISTENT, TAMM_OPT_OZAKI_TILE_POLICY, TAMM_OPT_OZAKI_PANELS,
 TAMM_OPT_OZAKI_SPLIT_K, TAMM_OPT_WAIT_CYCLES, TAMM_OPT_TEST_WITHHOLD_COPY, TAMM_OPT_OZAKI_SHARED_SCALE,
 TAMM_OPT_OZAKI_FUSED_A) = range(9)
SYM = {"dense": TAMM_SYM_DENSE, "spin": TAMM_SYM_SPIN, "spin_irrep": TAMM_SYM_SPIN_IRREP}
PREC = {"f64": TAMM_PREC_F64, "ozaki_bf16": TAMM_PREC_OZAKI_BF16, "ozaki_i8": TAMM_PREC_OZAKI_I8,
        "bf16x3": TAMM_PREC_BF16X3}
STATUS_NAMES = {0: "TAMM_OK", 1: "TAMM_EINVAL", 2: "TAMM_ENOMEM", 3: "TAMM_ECUDA", 4: "TAMM_EUNSUPPORTED",
                5: "TAMM_ETIMEOUT", 6: "TAMM_ECHECK", 7: "TAMM_ELIMIT"}

# C prototypes: (name, restype, argtypes)
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_cp = ctypes.c_char_p
_i64p, _ip, _dp = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

PROTOTYPES = [
    ("tamm_ctx_create", _i, [_i, _vp, ALLOC_FN, FREE_FN, _vp, ctypes.POINTER(_vp)]),
    ("tamm_ctx_set_stream", _i, [_vp, _vp]),
    ("tamm_ctx_destroy", None, [_vp]),
    ("tamm_last_error", _cp, [_vp]),
    ("tamm_sync", _i, [_vp]),
    ("tamm_ctx_set_option", _i, [_vp, _i, _i64]),
    ("tamm_ctx_launch_count", _i, [_vp, _i64p]),
    ("tamm_ctx_profile", _i, [_vp, _i]),
    ("tamm_ctx_profile_read", _i, [_vp, _dp, _i64p]),
    ("tamm_space_create", _i, [_vp, _i, _i64p, _ip, _ip, _i, _i64p, _i64, ctypes.POINTER(_vp)]),
    ("tamm_space_info", _i, [_vp, _ip, _i64p]),
    ("tamm_space_tiles", _i, [_vp, _i64p, _i64p, _ip, _ip]),
    ("tamm_space_destroy", None, [_vp]),
    ("tamm_tensor_create", _i, [_vp, _i, ctypes.POINTER(_vp), _i, _i, ctypes.POINTER(_vp)]),
    ("tamm_tensor_create_permuted", _i, [_vp, _vp, _ip, ctypes.POINTER(_vp)]),
    ("tamm_tensor_info", _i, [_vp, _i64p, _i64p]),
    ("tamm_tensor_blocks", _i, [_vp, _i64p, _i64p]),
    ("tamm_tensor_bind", _i, [_vp, _vp]),
    ("tamm_tensor_allocate", _i, [_vp]),
    ("tamm_tensor_copy_from_host", _i, [_vp, _vp, _vp]),
    ("tamm_tensor_copy_to_host", _i, [_vp, _vp, _vp]),
    ("tamm_tensor_data", _vp, [_vp]),
    ("tamm_tensor_destroy", None, [_vp]),
    ("tamm_tensor_create_cholesky", _i, [_vp, _vp, _i64, ctypes.POINTER(_vp)]),
    ("tamm_cholesky_info", _i, [_vp, _ip, _dp, _i64p]),
    ("tamm_cholesky_form", _i, [_vp, _vp, _vp, _i, _i]),
    ("tamm_contract", _i, [_vp, _d, _vp, _cp, _d, _vp, _cp, _vp, _cp, _i, _i]),
    ("tamm_contract_flops", _i, [_vp, _vp, _cp, _vp, _cp, _vp, _cp, _dp]),
    ("tamm_add", _i, [_vp, _vp, _cp, _d, _vp, _i, ctypes.POINTER(_cp), _dp]),
    ("tamm_add_scaled", _i, [_vp, _vp, _cp, _d, _vp, _i, ctypes.POINTER(_cp), _dp, _vp]),
    ("tamm_contract_adjoint", _i, [_vp, _d, _vp, _cp, _vp, _cp, _vp, _cp, _vp, _vp, _d, _i, _i]),
    ("tamm_energy", _i, [_vp, _d, _vp, _cp, _vp, _cp, _dp]),
    ("tamm_energy_async", _i, [_vp, _d, _vp, _cp, _vp, _cp, _vp]),
    ("tamm_norm", _i, [_vp, _vp, _dp]),
    ("tamm_norm_async", _i, [_vp, _vp, _vp]),
    ("tamm_norm_noalloc", _i, [_vp, _i64, _vp, _vp]),
    ("tamm_triples_energy", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i64, _vp, _vp]),
    ("tamm_triples_info", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _i64p, _dp, _ip]),
    ("tamm_fp64_peak", _i, [_vp, _i, _dp]),
    ("tamm_autotune", _i, [_vp, _vp, _cp, _vp, _cp, _vp, _cp, _d, _ip, _ip, _ip, _ip, _ip, _dp, _dp]),
    ("tamm_group_begin", _i, [_vp]),
    ("tamm_group_end", _i, [_vp]),
    ("tamm_group_cancel", _i, [_vp]),
    ("tamm_graph_begin", _i, [_vp]),
    ("tamm_graph_end", _i, [_vp, ctypes.POINTER(_vp)]),
    ("tamm_graph_launch", _i, [_vp]),
    ("tamm_graph_info", _i, [_vp, _i64p]),
    ("tamm_graph_destroy", None, [_vp]),
    ("tamm_sched_create", _i, [_vp, ctypes.POINTER(_vp)]),
    ("tamm_sched_contract", _i, [_vp, _d, _vp, _cp, _d, _vp, _cp, _vp, _cp, _i, _i]),
    ("tamm_sched_add", _i, [_vp, _vp, _cp, _d, _vp, _i, ctypes.POINTER(_cp), _dp]),
    ("tamm_sched_energy", _i, [_vp, _d, _vp, _cp, _vp, _cp, _vp]),
    ("tamm_sched_levels", _i, [_vp, _ip, _ip, _ip]),
    ("tamm_sched_execute", _i, [_vp]),
    ("tamm_sched_destroy", None, [_vp]),
]


class TammError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load the CUDA library (building it in-tree first if sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library {_build.LIB} is missing; run paper_2201_01257_gb300/build.py")
            lib = ctypes.CDLL(_build.LIB)
            for name, res, args in PROTOTYPES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def __getattr__(name):
    # tamm_* entry points, same names as the C ABI
    if name.startswith("tamm_"):
        return getattr(load(), name)
    raise AttributeError(name)


def _i64arr(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a, t=ctypes.c_int64):
    return a.ctypes.data_as(ctypes.POINTER(t))


# --------------------------------------------------------------- objects

class Context:
    """A CUDA device + stream + the library's scratch/plan caches (tamm_ctx)."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True):
        self.lib = load()
        self.device = device
        if device < 0:
            # host-only context: spaces, block tables and flop counts; no device work
            h = ctypes.c_void_p()
            st = self.lib.tamm_ctx_create(-1, None, ctypes.cast(None, ALLOC_FN), ctypes.cast(None, FREE_FN), None,
                                          ctypes.byref(h))
            if st != TAMM_OK:
                raise TammError(st, "tamm_ctx_create failed")
            self.handle = h
            return
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: this library has no CPU execution path")
        torch.cuda.set_device(device)
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._callbacks = None
        alloc_cb = ctypes.cast(None, ALLOC_FN)
        free_cb = ctypes.cast(None, FREE_FN)
        if use_torch_allocator:
            dev = device

            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            alloc_cb, free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
            self._callbacks = (alloc_cb, free_cb)
        h = ctypes.c_void_p()
        st = self.lib.tamm_ctx_create(device, ctypes.c_void_p(self.torch_stream.cuda_stream), alloc_cb, free_cb,
                                      None, ctypes.byref(h))
        if st != TAMM_OK:
            raise TammError(st, "tamm_ctx_create failed")
        self.handle = h

    def check(self, st: int, what: str = "") -> None:
        if st != TAMM_OK:
            msg = self.lib.tamm_last_error(self.handle).decode()
            raise TammError(st, f"{what}: {msg}" if what else msg)

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.tamm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # construction --------------------------------------------------------
    def space(self, groups, tile: int = 0, tile_sizes=()) -> "Space":
        return Space(self, groups, tile, tile_sizes)

    def tensor(self, modes, n_upper: int, sym: str = "spin", allocate: bool = True) -> "Tensor":
        return Tensor(self, modes, n_upper, sym, allocate and self.device >= 0)

    def tensor_cholesky(self, X: "Tensor", slab_bytes: int = 0) -> "CholeskyTensor":
        """Lambda tensor V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L] (Eq. cc12) over X's
        (P, R, aux) modes, formed slab by slab inside the contractions that read it."""
        return CholeskyTensor(self, X, slab_bytes)

    def cholesky_form(self, V: "CholeskyTensor", out: "Tensor", precision="f64", slices: int = 0) -> None:
        """Form all of V into the stored tensor ``out`` (same spaces and block table)."""
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        self.check(self.lib.tamm_cholesky_form(self.handle, V.handle, out.handle, prec, slices), "tamm_cholesky_form")

    def tensor_permuted(self, like: "Tensor", perm, allocate: bool = True) -> "Tensor":
        """Tensor whose mode m is like's mode perm[m], storing the images of like's blocks."""
        return Tensor(self, [like.modes[p] for p in perm], 0, "dense", allocate and self.device >= 0,
                      like=like, perm=perm)

    # operations ----------------------------------------------------------
    def contract(self, alpha, C, lc, beta, A, la, B, lb, precision="f64", slices: int = 0) -> None:
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        self.check(self.lib.tamm_contract(self.handle, alpha, C.handle, lc.encode(), beta, A.handle, la.encode(),
                                          B.handle, lb.encode(), prec, slices), "tamm_contract")

    def contract_adjoint(self, alpha, dC, lc, A, la, B, lb, dA=None, dB=None, beta=0.0, precision="f64",
                         slices: int = 0) -> None:
        """dA(la) = beta dA + alpha dC(lc) B(lb), dB(lb) = beta dB + alpha A(la) dC(lc): the adjoint of
        C(lc) = alpha A(la) B(lb); dA / dB (either may be None) have A's / B's block tables."""
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        self.check(self.lib.tamm_contract_adjoint(self.handle, alpha, dC.handle, lc.encode(), A.handle, la.encode(),
                                                  B.handle, lb.encode(), dA.handle if dA is not None else None,
                                                  dB.handle if dB is not None else None, beta, prec, slices),
                   "tamm_contract_adjoint")

    def flops(self, C, lc, A, la, B, lb) -> float:
        f = ctypes.c_double()
        self.check(self.lib.tamm_contract_flops(self.handle, C.handle, lc.encode(), A.handle, la.encode(), B.handle,
                                                lb.encode(), ctypes.byref(f)), "tamm_contract_flops")
        return f.value

    def add(self, C, lc, beta, A, terms) -> None:
        """C(lc) = beta*C + sum alpha_t * A(la_t); ``terms`` is [(alpha, la), ...]."""
        n = len(terms)
        las = (ctypes.c_char_p * n)(*[t[1].encode() for t in terms])
        al = (ctypes.c_double * n)(*[float(t[0]) for t in terms])
        self.check(self.lib.tamm_add(self.handle, C.handle, lc.encode(), beta, A.handle, n, las, al), "tamm_add")

    def add_scaled(self, C, lc, beta, A, terms, scale_device_ptr: int) -> None:
        """As ``add`` with every alpha multiplied by the device double at ``scale_device_ptr``."""
        n = len(terms)
        las = (ctypes.c_char_p * n)(*[t[1].encode() for t in terms])
        al = (ctypes.c_double * n)(*[float(t[0]) for t in terms])
        self.check(self.lib.tamm_add_scaled(self.handle, C.handle, lc.encode(), beta, A.handle, n, las, al,
                                            ctypes.c_void_p(scale_device_ptr)), "tamm_add_scaled")

    def energy(self, alpha, A, la, B, lb) -> float:
        r = ctypes.c_double()
        self.check(self.lib.tamm_energy(self.handle, alpha, A.handle, la.encode(), B.handle, lb.encode(),
                                        ctypes.byref(r)), "tamm_energy")
        return r.value

    def energy_async(self, alpha, A, la, B, lb, out_device_ptr: int) -> None:
        self.check(self.lib.tamm_energy_async(self.handle, alpha, A.handle, la.encode(), B.handle, lb.encode(),
                                              ctypes.c_void_p(out_device_ptr)), "tamm_energy_async")

    def triples_energy(self, T2, T1, Vooov, Vvovv, Voovv, eps_occ_ptr: int, eps_virt_ptr: int, out_ptr: int,
                       precision="f64", slices: int = 0, workspace_bytes: int = 0, per_triple_ptr: int = 0) -> None:
        """E(T) (Sec. IV.B) into the device double at ``out_ptr``; orbital energies and the optional
        per-triple output (``per_triple_ptr``) are device pointers."""
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        self.check(self.lib.tamm_triples_energy(self.handle, T2.handle, T1.handle, Vooov.handle, Vvovv.handle,
                                                Voovv.handle, ctypes.c_void_p(eps_occ_ptr),
                                                ctypes.c_void_p(eps_virt_ptr), prec, slices, int(workspace_bytes),
                                                ctypes.c_void_p(out_ptr),
                                                ctypes.c_void_p(per_triple_ptr) if per_triple_ptr else None),
                   "tamm_triples_energy")

    def triples_info(self, T2, T1, Vooov, Vvovv, Voovv, workspace_bytes: int = 0) -> dict:
        n, f, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
        self.check(self.lib.tamm_triples_info(self.handle, T2.handle, T1.handle, Vooov.handle, Vvovv.handle,
                                              Voovv.handle, int(workspace_bytes), ctypes.byref(n), ctypes.byref(f),
                                              ctypes.byref(b)), "tamm_triples_info")
        return {"n_triples": n.value, "gemm_flops": f.value, "n_batches": b.value}

    def fp64_peak(self, kind: str = "dfma") -> float:
        """Measured FP64 TFLOP/s of this device: ``dfma`` (scalar FMA) or ``dmma`` (FP64 tensor-core MMA)."""
        r = ctypes.c_double()
        self.check(self.lib.tamm_fp64_peak(self.handle, {"dfma": 0, "dmma": 1}[kind], ctypes.byref(r)),
                   "tamm_fp64_peak")
        return r.value

    def norm(self, T) -> float:
        r = ctypes.c_double()
        self.check(self.lib.tamm_norm(self.handle, T.handle, ctypes.byref(r)), "tamm_norm")
        return r.value

    def sync(self) -> None:
        self.check(self.lib.tamm_sync(self.handle), "tamm_sync")

    def set_option(self, option: int, value: int) -> None:
        self.check(self.lib.tamm_ctx_set_option(self.handle, int(option), int(value)), "tamm_ctx_set_option")

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        self.check(self.lib.tamm_ctx_launch_count(self.handle, ctypes.byref(n)), "tamm_ctx_launch_count")
        return n.value

    def profile(self, enable: bool) -> None:
        self.check(self.lib.tamm_ctx_profile(self.handle, int(enable)), "tamm_ctx_profile")

    def profile_read(self) -> dict:
        """{kernel class: (total ms, launches)} recorded since the last read."""
        n = len(KERNEL_CLASSES)
        ms, cnt = (ctypes.c_double * n)(), (ctypes.c_int64 * n)()
        self.check(self.lib.tamm_ctx_profile_read(self.handle, ms, cnt), "tamm_ctx_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def autotune(self, C, lc, A, la, B, lb, target: float = 1e-10) -> dict:
        """Pick slices and chunk length for this split-precision contraction (used when slices = 0)."""
        s, ck, tp, pe, sh = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        err, ms = ctypes.c_double(), ctypes.c_double()
        self.check(self.lib.tamm_autotune(self.handle, C.handle, lc.encode(), A.handle, la.encode(), B.handle,
                                          lb.encode(), float(target), ctypes.byref(s), ctypes.byref(ck),
                                          ctypes.byref(tp), ctypes.byref(pe), ctypes.byref(sh), ctypes.byref(err),
                                          ctypes.byref(ms)),
                   "tamm_autotune")
        return {"slices": s.value, "chunk_k": ck.value, "tile_policy": tp.value, "persistent": pe.value,
                "shared_scale": int(sh.value == 1), "fused_a": int(sh.value == 2), "rel_err": err.value,
                "ms": ms.value}

    # grouped execution ---------------------------------------------------
    def group_begin(self) -> None:
        self.check(self.lib.tamm_group_begin(self.handle), "tamm_group_begin")

    def group_end(self) -> None:
        self.check(self.lib.tamm_group_end(self.handle), "tamm_group_end")

    @contextlib.contextmanager
    def group(self):
        """Split-precision contractions issued inside run as one grouped launch on exit."""
        self.group_begin()
        try:
            yield self
        except BaseException:
            self.lib.tamm_group_cancel(self.handle)  # drop what was recorded; the error propagates
            raise
        self.group_end()

    def graph_begin(self) -> None:
        self.check(self.lib.tamm_graph_begin(self.handle), "tamm_graph_begin")

    def graph_end(self) -> "Graph":
        h = ctypes.c_void_p()
        self.check(self.lib.tamm_graph_end(self.handle, ctypes.byref(h)), "tamm_graph_end")
        return Graph(self, h)

    @contextlib.contextmanager
    def capture(self):
        """Capture the library calls of the block into a Graph (``with ctx.capture() as g: ...; g.graph.launch()``)."""
        holder = types.SimpleNamespace(graph=None)
        self.graph_begin()
        try:
            yield holder
        finally:
            holder.graph = self.graph_end()

    def scheduler(self) -> "Scheduler":
        """Deferred execution by dependency level (tamm_sched_*)."""
        return Scheduler(self)

    def copy_from_host(self, T, host: np.ndarray) -> None:
        assert host.dtype == np.float64 and host.flags.c_contiguous and host.size >= T.n_elems
        self.check(self.lib.tamm_tensor_copy_from_host(self.handle, T.handle, ctypes.c_void_p(host.ctypes.data)),
                   "tamm_tensor_copy_from_host")

    def copy_to_host(self, T, host: np.ndarray) -> None:
        assert host.dtype == np.float64 and host.flags.c_contiguous and host.size >= T.n_elems
        self.check(self.lib.tamm_tensor_copy_to_host(self.handle, T.handle, ctypes.c_void_p(host.ctypes.data)),
                   "tamm_tensor_copy_to_host")


class Scheduler:
    """Recorded operations run level by level (tamm_sched); the recording methods return self."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self._keep = []  # tensors recorded here stay alive as long as the scheduler
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.tamm_sched_create(ctx.handle, ctypes.byref(h)), "tamm_sched_create")
        self.handle = h

    def contract(self, alpha, C, lc, beta, A, la, B, lb, precision="f64", slices: int = 0) -> "Scheduler":
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        self._keep += [C, A, B]
        self.ctx.check(self.ctx.lib.tamm_sched_contract(self.handle, alpha, C.handle, lc.encode(), beta, A.handle,
                                                        la.encode(), B.handle, lb.encode(), prec, slices),
                       "tamm_sched_contract")
        return self

    def add(self, C, lc, beta, A, terms) -> "Scheduler":
        n = len(terms)
        las = (ctypes.c_char_p * n)(*[t[1].encode() for t in terms])
        al = (ctypes.c_double * n)(*[float(t[0]) for t in terms])
        self._keep += [C, A]
        self.ctx.check(self.ctx.lib.tamm_sched_add(self.handle, C.handle, lc.encode(), beta, A.handle, n, las, al),
                       "tamm_sched_add")
        return self

    def energy_async(self, alpha, A, la, B, lb, out_device_ptr: int) -> "Scheduler":
        self._keep += [A, B]
        self.ctx.check(self.ctx.lib.tamm_sched_energy(self.handle, alpha, A.handle, la.encode(), B.handle,
                                                      lb.encode(), ctypes.c_void_p(out_device_ptr)),
                       "tamm_sched_energy")
        return self

    def levels(self) -> list:
        n, nl = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.tamm_sched_levels(self.handle, ctypes.byref(n), ctypes.byref(nl), None),
                       "tamm_sched_levels")
        lev = (ctypes.c_int * max(n.value, 1))()
        self.ctx.check(self.ctx.lib.tamm_sched_levels(self.handle, None, None, lev), "tamm_sched_levels")
        return [lev[i] for i in range(n.value)]

    def execute(self) -> None:
        self.ctx.check(self.ctx.lib.tamm_sched_execute(self.handle), "tamm_sched_execute")

    def __del__(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            self.ctx.lib.tamm_sched_destroy(self.handle)
            self.handle = None


class Graph:
    """A captured sequence of library calls (tamm_graph), replayed with one CUDA-graph launch."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def launch(self) -> None:
        self.ctx.check(self.ctx.lib.tamm_graph_launch(self.handle), "tamm_graph_launch")

    @property
    def kernel_launches(self) -> int:
        n = ctypes.c_int64()
        self.ctx.check(self.ctx.lib.tamm_graph_info(self.handle, ctypes.byref(n)), "tamm_graph_info")
        return n.value

    def destroy(self) -> None:
        if self.handle:
            self.ctx.lib.tamm_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Space:
    """Tiled index space of (size, spin, irrep) groups (tamm_space)."""

    def __init__(self, ctx: Context, groups, tile: int = 0, tile_sizes=()):
        self.ctx = ctx
        g = list(groups)
        gs = _i64arr([x[0] for x in g])
        sp = np.ascontiguousarray([int(x[1]) for x in g], dtype=np.int32)
        ir = np.ascontiguousarray([int(x[2]) if len(x) > 2 else 0 for x in g], dtype=np.int32)
        ts = _i64arr(tile_sizes if len(tile_sizes) else [0])
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.tamm_space_create(ctx.handle, len(g), _ptr(gs), _ptr(sp, ctypes.c_int),
                                            _ptr(ir, ctypes.c_int), len(tile_sizes), _ptr(ts), int(tile),
                                            ctypes.byref(h)), "tamm_space_create")
        self.handle = h
        nt, n = ctypes.c_int(), ctypes.c_int64()
        ctx.lib.tamm_space_info(h, ctypes.byref(nt), ctypes.byref(n))
        self.n_tiles, self.n = nt.value, n.value
        off, size = np.zeros(self.n_tiles, np.int64), np.zeros(self.n_tiles, np.int64)
        spin, irrep = np.zeros(self.n_tiles, np.int32), np.zeros(self.n_tiles, np.int32)
        ctx.lib.tamm_space_tiles(h, _ptr(off), _ptr(size), _ptr(spin, ctypes.c_int), _ptr(irrep, ctypes.c_int))
        self.tile_offset, self.tile_size, self.tile_spin, self.tile_irrep = off, size, spin, irrep

    def __del__(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            self.ctx.lib.tamm_space_destroy(self.handle)
            self.handle = None


class Tensor:
    """Block-sparse FP64 tensor (tamm_tensor) whose storage is a torch CUDA tensor."""

    def __init__(self, ctx: Context, modes, n_upper: int, sym: str = "spin", allocate: bool = True,
                 like: "Tensor" = None, perm=None):
        self.ctx = ctx
        self.modes = list(modes)
        self.nm = len(self.modes)
        h = ctypes.c_void_p()
        if like is not None:
            p = (ctypes.c_int * self.nm)(*[int(x) for x in perm])
            ctx.check(ctx.lib.tamm_tensor_create_permuted(ctx.handle, like.handle, p, ctypes.byref(h)),
                      "tamm_tensor_create_permuted")
        else:
            arr = (ctypes.c_void_p * self.nm)(*[m.handle for m in self.modes])
            ctx.check(ctx.lib.tamm_tensor_create(ctx.handle, self.nm, arr, n_upper, SYM[sym], ctypes.byref(h)),
                      "tamm_tensor_create")
        self.handle = h
        nb, ne = ctypes.c_int64(), ctypes.c_int64()
        ctx.lib.tamm_tensor_info(h, ctypes.byref(nb), ctypes.byref(ne))
        self.n_blocks, self.n_elems = nb.value, ne.value
        self.block_tiles = np.zeros((self.n_blocks, self.nm), np.int64)
        self.block_offsets = np.zeros(self.n_blocks, np.int64)
        if self.n_blocks:
            ctx.lib.tamm_tensor_blocks(h, _ptr(self.block_tiles), _ptr(self.block_offsets))
        self.data = None
        if allocate:
            import torch

            self.bind(torch.zeros(max(self.n_elems, 1), dtype=torch.float64, device=f"cuda:{ctx.device}"))

    def bind(self, t) -> None:
        import torch

        assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous() and t.numel() >= self.n_elems
        self.ctx.check(self.ctx.lib.tamm_tensor_bind(self.handle, ctypes.c_void_p(t.data_ptr())), "tamm_tensor_bind")
        self.data = t

    def block_lo_ext(self):
        lo = np.zeros((self.n_blocks, self.nm), np.int64)
        ext = np.zeros((self.n_blocks, self.nm), np.int64)
        for m in range(self.nm):
            lo[:, m] = self.modes[m].tile_offset[self.block_tiles[:, m]]
            ext[:, m] = self.modes[m].tile_size[self.block_tiles[:, m]]
        return lo, ext

    def upload(self, host: np.ndarray) -> None:
        import torch

        assert host.size == self.n_elems
        self.data[: self.n_elems].copy_(torch.from_numpy(np.ascontiguousarray(host, dtype=np.float64)))

    def download(self) -> np.ndarray:
        return self.data[: self.n_elems].cpu().numpy()

    def __del__(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            self.ctx.lib.tamm_tensor_destroy(self.handle)
            self.handle = None


class CholeskyTensor(Tensor):
    """Read-only lambda tensor formed from Cholesky vectors X (tamm_tensor_create_cholesky); it has a block
    table but no storage, and keeps X alive."""

    def __init__(self, ctx: Context, X: Tensor, slab_bytes: int = 0):
        self.ctx = ctx
        self.factor = X
        self.modes = [X.modes[0], X.modes[0], X.modes[1], X.modes[1]]
        self.nm = 4
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.tamm_tensor_create_cholesky(ctx.handle, X.handle, int(slab_bytes), ctypes.byref(h)),
                  "tamm_tensor_create_cholesky")
        self.handle = h
        nb, ne = ctypes.c_int64(), ctypes.c_int64()
        ctx.lib.tamm_tensor_info(h, ctypes.byref(nb), ctypes.byref(ne))
        self.n_blocks, self.n_elems = nb.value, ne.value
        self.block_tiles = np.zeros((self.n_blocks, self.nm), np.int64)
        self.block_offsets = np.zeros(self.n_blocks, np.int64)
        if self.n_blocks:
            ctx.lib.tamm_tensor_blocks(h, _ptr(self.block_tiles), _ptr(self.block_offsets))
        self.data = None
        n, f, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_int64()
        ctx.check(ctx.lib.tamm_cholesky_info(h, ctypes.byref(n), ctypes.byref(f), ctypes.byref(b)),
                  "tamm_cholesky_info")
        self.n_slabs, self.form_flops, self.buffer_bytes = n.value, f.value, b.value

    def bind(self, t) -> None:
        raise TammError(TAMM_EUNSUPPORTED, "a lambda tensor has no storage")

    def upload(self, host: np.ndarray) -> None:
        raise TammError(TAMM_EUNSUPPORTED, "a lambda tensor has no storage")

    def download(self) -> np.ndarray:
        raise TammError(TAMM_EUNSUPPORTED, "a lambda tensor has no storage")
