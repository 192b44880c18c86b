"""FP64 CPU oracle for TAMM block-sparse contractions (arXiv:2201.01257, Sec. III).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the GPU library.  The arithmetic
lives in ``tamm_oracle.c`` (plain nested loops over nonzero blocks, FP64); this
module only marshals arguments and runs workload recipes step by step.

Every function here is pinned by ``tests/test_oracle_pins.py`` (brute-force
dense einsum, closed-form block counts, identities, invariants),
``tests/test_oracle_cholesky.py`` (the Cholesky-built tensor) and
``tests/test_oracle_triples.py`` (the (T) correction against the antisymmetrised
construction of its amplitudes); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

import tamm_synth
from tamm_synth import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tamm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SYM = {"dense": 0, "spin": 1, "spin_irrep": 2}


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        # no fused multiply-add contraction: every product and sum is rounded as written, on any host
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str | None = None):
    global _lib
    with _lock:
        if _lib is None or path is not None:
            L = ctypes.CDLL(path or build())
            vp, i64, i64p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)
            dp, cp, d = ctypes.POINTER(ctypes.c_double), ctypes.c_char_p, ctypes.c_double
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_space_create.argtypes = [ctypes.c_int, i64p, ip, ip, i64, ctypes.c_int, i64p]
            L.oracle_space_create.restype = vp
            L.oracle_space_destroy.argtypes = [vp]
            L.oracle_space_ntiles.argtypes = [vp]
            L.oracle_space_size.argtypes = [vp]
            L.oracle_space_size.restype = i64
            L.oracle_space_tile.argtypes = [vp, ctypes.c_int, i64p, i64p, ip, ip]
            L.oracle_tensor_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
            L.oracle_tensor_create.restype = vp
            L.oracle_tensor_destroy.argtypes = [vp]
            L.oracle_tensor_nblocks.argtypes = [vp]
            L.oracle_tensor_nblocks.restype = i64
            L.oracle_tensor_nelems.argtypes = [vp]
            L.oracle_tensor_nelems.restype = i64
            L.oracle_tensor_blocks.argtypes = [vp, i64p, i64p]
            L.oracle_tensor_find_block.argtypes = [vp, i64p]
            L.oracle_tensor_find_block.restype = i64
            L.oracle_contract.argtypes = [d, vp, cp, d, vp, cp, vp, cp, dp, dp, dp]
            L.oracle_contract_blocks.argtypes = [d, vp, cp, d, vp, cp, vp, cp, dp, dp, dp, i64p, i64]
            L.oracle_contract_boxes.argtypes = [d, vp, cp, vp, cp, vp, cp, dp, dp, i64, i64p, i64p, i64p, i64p, dp]
            L.oracle_contract_box.argtypes = [d, vp, cp, d, vp, cp, vp, cp, dp, dp, i64, i64p, i64p, dp, dp]
            L.oracle_add.argtypes = [d, vp, cp, d, vp, cp, dp, dp]
            L.oracle_energy.argtypes = [d, vp, cp, vp, cp, dp, dp, dp]
            L.oracle_norm.argtypes = [vp, dp]
            L.oracle_norm.restype = d
            L.oracle_cholesky_v.argtypes = [vp, vp, dp, dp, i64p, i64]
            L.oracle_triples_energy.argtypes = [vp, dp, vp, dp, vp, dp, vp, dp, vp, dp, dp, dp, dp]
            L.oracle_triples_wy.argtypes = [vp, dp, vp, dp, vp, dp, vp, dp, vp, dp, i64, i64, i64, dp, dp]
            if path is not None:
                return L
            _lib = L
    return _lib


class using_library:
    """Temporarily route every oracle call to another build of ``tamm_oracle.c``
    (used by the mutation tests, which compile deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _load()
        _lib = _load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a, t=ctypes.c_int64):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


class Space:
    """Tiled index space made of (size, spin, irrep) groups (Sec. III.A)."""

    def __init__(self, groups, tile: int = 0, tile_sizes=()):
        L = _load()
        g = list(groups)
        gs = _i64([x[0] for x in g])
        sp = np.ascontiguousarray([int(x[1]) for x in g], dtype=np.int32)
        ir = np.ascontiguousarray([int(x[2]) if len(x) > 2 else 0 for x in g], dtype=np.int32)
        ts = _i64(tile_sizes if len(tile_sizes) else [0])
        self._h = L.oracle_space_create(len(g), _p(gs), _p(sp, ctypes.c_int), _p(ir, ctypes.c_int), int(tile),
                                        len(tile_sizes), _p(ts))
        if not self._h:
            raise OracleError("invalid index space / tiling")
        self._lib = L
        self.n = L.oracle_space_size(self._h)
        self.n_tiles = L.oracle_space_ntiles(self._h)
        self.tiles = []
        for t in range(self.n_tiles):
            o, s = ctypes.c_int64(), ctypes.c_int64()
            spn, irr = ctypes.c_int(), ctypes.c_int()
            L.oracle_space_tile(self._h, t, ctypes.byref(o), ctypes.byref(s), ctypes.byref(spn), ctypes.byref(irr))
            self.tiles.append((o.value, s.value, spn.value, irr.value))

    @classmethod
    def from_spec(cls, spec: wl.SpaceSpec) -> "Space":
        return cls(spec.groups, spec.tile, spec.tile_sizes)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.oracle_space_destroy(self._h)
            self._h = None


class Tensor:
    """Block-sparse FP64 tensor on the host: stored blocks packed in lexicographic tile order."""

    def __init__(self, modes, n_upper: int, sym: str = "spin", alloc: bool = True):
        L = _load()
        self.modes = list(modes)
        self.nm = len(self.modes)
        arr = (ctypes.c_void_p * self.nm)(*[m._h for m in self.modes])
        self._h = L.oracle_tensor_create(self.nm, arr, n_upper, SYM[sym])
        if not self._h:
            raise OracleError("invalid tensor")
        self.n_upper = n_upper
        self.sym = sym
        self.n_blocks = L.oracle_tensor_nblocks(self._h)
        self.n_elems = L.oracle_tensor_nelems(self._h)
        self.block_tiles = np.zeros((self.n_blocks, self.nm), dtype=np.int64)
        self.block_off = np.zeros(self.n_blocks, dtype=np.int64)
        if self.n_blocks:
            L.oracle_tensor_blocks(self._h, _p(self.block_tiles), _p(self.block_off))
        self.data = np.zeros(self.n_elems if alloc else 0, dtype=np.float64)
        self._lib = L

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.oracle_tensor_destroy(self._h)
            self._h = None

    # geometry ---------------------------------------------------------------
    def block_lo_ext(self):
        lo = np.zeros((self.n_blocks, self.nm), dtype=np.int64)
        ext = np.zeros((self.n_blocks, self.nm), dtype=np.int64)
        for b in range(self.n_blocks):
            for m in range(self.nm):
                o, s, _, _ = self.modes[m].tiles[self.block_tiles[b, m]]
                lo[b, m], ext[b, m] = o, s
        return lo, ext

    def find_block(self, tiles) -> int:
        t = _i64(tiles)
        return int(_load().oracle_tensor_find_block(self._h, _p(t)))

    def block_view(self, b: int) -> np.ndarray:
        _, ext = self.block_lo_ext()
        n = int(np.prod(ext[b]))
        return self.data[self.block_off[b]:self.block_off[b] + n].reshape(tuple(ext[b]))

    def dense_shape(self):
        return tuple(m.n for m in self.modes)

    def to_dense(self) -> np.ndarray:
        """Dense array with zeros in every block that is not stored (test helper)."""
        out = np.zeros(self.dense_shape())
        lo, ext = self.block_lo_ext()
        for b in range(self.n_blocks):
            n = int(np.prod(ext[b]))
            sl = tuple(slice(lo[b, m], lo[b, m] + ext[b, m]) for m in range(self.nm))
            out[sl] = self.data[self.block_off[b]:self.block_off[b] + n].reshape(tuple(ext[b]))
        return out

    def from_dense(self, dense: np.ndarray) -> None:
        lo, ext = self.block_lo_ext()
        for b in range(self.n_blocks):
            n = int(np.prod(ext[b]))
            sl = tuple(slice(lo[b, m], lo[b, m] + ext[b, m]) for m in range(self.nm))
            self.data[self.block_off[b]:self.block_off[b] + n] = dense[sl].reshape(-1)

    def fill_synthetic(self, seed: int, spec: wl.TensorSpec) -> None:
        if spec.sigma == 0.0:
            self.data[:] = 0.0
            return
        lo, ext = self.block_lo_ext()
        tamm_synth.fill_boxes(seed, spec.stream, spec.sigma, self.dense_shape(), spec.anti01, spec.anti23,
                              lo, ext, self.block_off, self.data, sym01=spec.sym01)


def _chk(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what} failed ({rc}): invalid labels or spaces")


def contract(alpha: float, C: Tensor, lc: str, beta: float, A: Tensor, la: str, B: Tensor, lb: str) -> None:
    """C(lc) = beta*C + alpha * A(la) * B(lb), in place on C.data (MultOp, grammar figure of Sec. III.A)."""
    _chk(_load().oracle_contract(alpha, C._h, lc.encode(), beta, A._h, la.encode(), B._h, lb.encode(),
                                 _pd(C.data), _pd(A.data), _pd(B.data)), "contract")


def contract_blocks(alpha: float, C: Tensor, lc: str, beta: float, A: Tensor, la: str, B: Tensor, lb: str,
                    blocks) -> None:
    """The contraction restricted to the listed stored blocks of C (in place)."""
    bl = _i64(blocks)
    _chk(_load().oracle_contract_blocks(alpha, C._h, lc.encode(), beta, A._h, la.encode(), B._h, lb.encode(),
                                        _pd(C.data), _pd(A.data), _pd(B.data), _p(bl), len(bl)), "contract_blocks")


def contract_box(alpha: float, C: Tensor, lc: str, beta: float, A: Tensor, la: str, B: Tensor, lb: str,
                 cblock: int, lo, ext, c_in: np.ndarray | None = None) -> np.ndarray:
    """Values of the box [lo, lo+ext) of stored C block ``cblock`` after the contraction."""
    lo, ext = _i64(lo), _i64(ext)
    out = np.zeros(int(np.prod(ext)), dtype=np.float64)
    cin = np.ascontiguousarray(c_in, dtype=np.float64).reshape(-1) if c_in is not None else out
    _chk(_load().oracle_contract_box(alpha, C._h, lc.encode(), beta, A._h, la.encode(), B._h, lb.encode(),
                                     _pd(A.data), _pd(B.data), int(cblock), _p(lo), _p(ext), _pd(cin), _pd(out)),
         "contract_box")
    return out.reshape(tuple(ext))


def contract_boxes(alpha: float, C: Tensor, lc: str, A: Tensor, la: str, B: Tensor, lb: str, cblocks, lo,
                   ext) -> list:
    """Several boxes of stored C blocks (beta = 0), evaluated in parallel; returns one array per box."""
    cb = _i64(cblocks)
    lo = _i64(lo).reshape(len(cb), C.nm)
    ext = _i64(ext).reshape(len(cb), C.nm)
    sizes = ext.prod(axis=1)
    off = _i64(np.concatenate([[0], np.cumsum(sizes)[:-1]]) if len(cb) else [])
    out = np.zeros(int(sizes.sum()) if len(cb) else 1)
    _chk(_load().oracle_contract_boxes(alpha, C._h, lc.encode(), A._h, la.encode(), B._h, lb.encode(), _pd(A.data),
                                       _pd(B.data), len(cb), _p(cb), _p(lo), _p(ext), _p(off), _pd(out)),
         "contract_boxes")
    return [out[o:o + n].reshape(tuple(e)) for o, n, e in zip(off, sizes, ext)]


def add(alpha: float, C: Tensor, lc: str, beta: float, A: Tensor, la: str) -> None:
    """C(lc) = beta*C + alpha * A(la) (AddOp with label permutation)."""
    _chk(_load().oracle_add(alpha, C._h, lc.encode(), beta, A._h, la.encode(), _pd(C.data), _pd(A.data)), "add")


def energy(alpha: float, A: Tensor, la: str, B: Tensor, lb: str) -> float:
    """alpha * sum over all stored entries of A(la) * B(lb) (full contraction to a scalar)."""
    r = ctypes.c_double()
    _chk(_load().oracle_energy(alpha, A._h, la.encode(), B._h, lb.encode(), _pd(A.data), _pd(B.data),
                               ctypes.byref(r)), "energy")
    return r.value


def norm(T: Tensor) -> float:
    return _load().oracle_norm(T._h, _pd(T.data))


def cholesky_v(V: Tensor, X: Tensor, blocks=None) -> None:
    """V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L] (Eq. cc12) into the listed stored blocks of V
    (every block by default), in place on V.data; X has modes (P, R, aux), V modes (P, P, R, R)."""
    if blocks is None:
        _chk(_load().oracle_cholesky_v(V._h, X._h, _pd(X.data), _pd(V.data), None, 0), "cholesky_v")
    else:
        bl = _i64(blocks)
        _chk(_load().oracle_cholesky_v(V._h, X._h, _pd(X.data), _pd(V.data), _p(bl), len(bl)), "cholesky_v")


def _triples_args(T: dict):
    return (T["T"]._h, _pd(T["T"].data), T["t1"]._h, _pd(T["t1"].data), T["V_ooov"]._h, _pd(T["V_ooov"].data),
            T["V_vovv"]._h, _pd(T["V_vovv"].data), T["V_oovv"]._h, _pd(T["V_oovv"].data))


def triples_energy(T: dict, eps_o, eps_v) -> float:
    """E(T) = sum_{i<j<k, a<b<c} (W + Y) W / D (Eqs. cc14, tensort, tensort2) from the tensors T, t1,
    V_ooov, V_vovv, V_oovv of a ``triples`` recipe and the orbital energies."""
    eo = np.ascontiguousarray(eps_o, dtype=np.float64)
    ev = np.ascontiguousarray(eps_v, dtype=np.float64)
    r = ctypes.c_double()
    _chk(_load().oracle_triples_energy(*_triples_args(T), _pd(eo), _pd(ev), ctypes.byref(r)), "triples_energy")
    return r.value


def triples_wy(T: dict, i: int, j: int, k: int) -> tuple:
    """W (Eq. tensort) and Y (Eq. tensort2) of the occupied triple (i, j, k) over every (a, b, c)."""
    nv = T["T"].modes[0].n
    w = np.zeros((nv, nv, nv))
    y = np.zeros((nv, nv, nv))
    _chk(_load().oracle_triples_wy(*_triples_args(T), int(i), int(j), int(k), _pd(w), _pd(y)), "triples_wy")
    return w, y


def antisymmetrize_add(R: Tensor, lr: str, X: Tensor, alpha: float = 1.0) -> None:
    """R(abij) += alpha * P(ab)P(ij) X = alpha*(X(abij) - X(baij) - X(abji) + X(baji))."""
    a, b, i, j = lr
    add(alpha, R, lr, 1.0, X, a + b + i + j)
    add(-alpha, R, lr, 1.0, X, b + a + i + j)
    add(-alpha, R, lr, 1.0, X, a + b + j + i)
    add(alpha, R, lr, 1.0, X, b + a + j + i)


# ---------------------------------------------------------------- workloads

def build_workload(w: wl.Workload, fill: bool = True):
    """Spaces and tensors of a recipe; a tensor formed from Cholesky vectors is stored here in full."""
    spaces = {k: Space.from_spec(s) for k, s in w.spaces.items()}
    tensors = {}
    for name, t in w.tensors.items():
        T = Tensor([spaces[m] for m in t.modes], t.n_upper, t.sym)
        if fill and not t.cholesky:
            T.fill_synthetic(w.seed, t)
        tensors[name] = T
    for name, t in w.tensors.items():
        if fill and t.cholesky:
            cholesky_v(tensors[name], tensors[t.cholesky])
    return spaces, tensors


def run_step(w: wl.Workload, tensors: dict, step) -> float | None:
    if isinstance(step, wl.EnergySpec):
        return energy(step.alpha, tensors[step.a], step.la, tensors[step.b], step.lb)
    if isinstance(step, wl.AddSpec):
        for t, (al, la) in enumerate(step.terms):
            add(al, tensors[step.c], step.lc, step.beta if t == 0 else 1.0, tensors[step.a], la)
        return None
    C, A, B = tensors[step.c], tensors[step.a], tensors[step.b]
    if step.antisym:
        X = Tensor(C.modes, C.n_upper, C.sym)
        contract(step.alpha, X, step.lc, 0.0, A, step.la, B, step.lb)
        if step.beta == 0.0:
            C.data[:] = 0.0
        antisymmetrize_add(C, step.lc, X)
    else:
        contract(step.alpha, C, step.lc, step.beta, A, step.la, B, step.lb)
    return None


def run_workload(w: wl.Workload, tensors: dict) -> dict:
    """Run every step of the recipe in order; returns {energy step name: value}."""
    out = {}
    for s in w.steps:
        r = run_step(w, tensors, s)
        if r is not None:
            out[s.name] = r
    return out
