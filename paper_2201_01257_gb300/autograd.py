"""Gradients of block-sparse contractions through torch.autograd.

Every block-sparse tensor is a torch CUDA buffer holding its packed stored
blocks (the layout of its ``Tensor`` template).  Forward and backward passes
run in the library's kernels:

* contraction C = alpha A(la) B(lb) (Sec. III.A MultOp): its adjoints are
  contractions with the label roles exchanged,
      dA(la) = alpha sum dC(lc) B(lb),   dB(lb) = alpha sum A(la) dC(lc),
  computed by ``tamm_contract_adjoint`` on the same block-sparse machinery;
* full contraction E = alpha sum A(la) B(lb): dA = alpha dE B(perm), a
  permuted add scaled by the incoming derivative dE where it lies on the
  device (``tamm_add_scaled``: no host round trip), and the same for B;
* ``ladder_energy``: the doubles-shaped energy of a ladder update,
      T' = T + 1/2 V_vvvv(abef) T(efij),   E = 1/4 V_oovv(ijab) T'(abij),
  with a hand-written backward (G = dE/dT' = 1/4 dE V_oovv(ijab) as (abij);
  dT = G + 1/2 V_vvvv(abef) G(abij) -> (efij); dV_vvvv = 1/2 G(abij) T(efij);
  dV_oovv = 1/4 dE T'(abij) -> (ijab)) that can recompute T' instead of storing
  it.

Gradients are taken with respect to every stored entry as an independent
variable.  Every forward and backward pass ends with ``tamm_sync``, so that a
device-side failure of its kernels (a bounded wait that ran out) raises there,
attributed to the operation that caused it, instead of leaving partial results.
"""
from __future__ import annotations

import torch

from . import Context, Tensor


def _bind(T: Tensor, buf: torch.Tensor) -> Tensor:
    T.bind(buf)
    return T


class _Twins:
    """Extra handles with a template's block structure, so one layout can be bound to several buffers."""

    def __init__(self):
        self._cache = {}

    def get(self, T: Tensor, k=0) -> Tensor:
        key = (id(T), k)
        if key not in self._cache:
            self._cache[key] = (T, T.ctx.tensor_permuted(T, list(range(T.nm)), allocate=False))
        return self._cache[key][1]


_twins = _Twins()


def _checked(tctx: Context) -> None:
    """Synchronise and raise on any device-side status the pass's kernels recorded."""
    tctx.sync()


def _scale_ptr(g: torch.Tensor) -> tuple:
    """Device pointer of the incoming derivative of a scalar (kept alive by the returned tensor)."""
    g = g.detach().reshape(1).contiguous()
    if g.dtype != torch.float64:
        raise TypeError("the incoming derivative must be float64")
    return g, g.data_ptr()


def _zeros(T: Tensor) -> torch.Tensor:
    return torch.zeros(max(T.n_elems, 1), dtype=torch.float64, device=f"cuda:{T.ctx.device}")


class _Contract(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, b, spec):
        tctx, alpha, C, lc, A, la, B, lb, prec, slices = spec
        out = _zeros(C)
        tctx.contract(alpha, _bind(_twins.get(C, "C"), out), lc, 0.0, _bind(_twins.get(A, "A"), a), la,
                      _bind(_twins.get(B, "B"), b), lb, prec, slices)
        _checked(tctx)
        fctx.save_for_backward(a, b)
        fctx.spec = spec
        return out

    @staticmethod
    def backward(fctx, g):
        a, b = fctx.saved_tensors
        tctx, alpha, C, lc, A, la, B, lb, prec, slices = fctx.spec
        g = g.contiguous()
        ga = _zeros(A) if fctx.needs_input_grad[0] else None
        gb = _zeros(B) if fctx.needs_input_grad[1] else None
        if ga is not None or gb is not None:
            tctx.contract_adjoint(alpha, _bind(_twins.get(C, "gC"), g), lc, _bind(_twins.get(A, "A"), a), la,
                                  _bind(_twins.get(B, "B"), b), lb,
                                  dA=_bind(_twins.get(A, "gA"), ga) if ga is not None else None,
                                  dB=_bind(_twins.get(B, "gB"), gb) if gb is not None else None,
                                  beta=0.0, precision=prec, slices=slices)
            _checked(tctx)
        return ga, gb, None


def contract(tctx: Context, alpha: float, C: Tensor, lc: str, A: Tensor, a: torch.Tensor, la: str, B: Tensor,
             b: torch.Tensor, lb: str, precision: str = "f64", slices: int = 0) -> torch.Tensor:
    """C(lc) = alpha A(la) B(lb) on packed buffers ``a``, ``b`` laid out as templates A, B; differentiable."""
    return _Contract.apply(a, b, (tctx, alpha, C, lc, A, la, B, lb, precision, slices))


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, b, spec):
        tctx, alpha, A, la, B, lb = spec
        out = torch.zeros(1, dtype=torch.float64, device=a.device)
        tctx.energy_async(alpha, _bind(_twins.get(A, "eA"), a), la, _bind(_twins.get(B, "eB"), b), lb,
                          out.data_ptr())
        _checked(tctx)
        fctx.save_for_backward(a, b)
        fctx.spec = spec
        return out[0]

    @staticmethod
    def backward(fctx, g):
        a, b = fctx.saved_tensors
        tctx, alpha, A, la, B, lb = fctx.spec
        g, gp = _scale_ptr(g)
        ga = gb = None
        if fctx.needs_input_grad[0]:
            ga = _zeros(A)
            tctx.add_scaled(_bind(_twins.get(A, "egA"), ga), la, 0.0, _bind(_twins.get(B, "eB"), b), [(alpha, lb)], gp)
        if fctx.needs_input_grad[1]:
            gb = _zeros(B)
            tctx.add_scaled(_bind(_twins.get(B, "egB"), gb), lb, 0.0, _bind(_twins.get(A, "eA"), a), [(alpha, la)], gp)
        _checked(tctx)
        return ga, gb, None


def energy(tctx: Context, alpha: float, A: Tensor, a: torch.Tensor, la: str, B: Tensor, b: torch.Tensor,
           lb: str) -> torch.Tensor:
    """E = alpha sum A(la) B(lb) (full contraction) as a differentiable scalar."""
    return _Energy.apply(a, b, (tctx, alpha, A, la, B, lb))


class _LadderEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v, t, voo, spec):
        tctx, V, T, Voo, prec, slices, recompute = spec
        tp = _ladder_update(tctx, V, v, T, t, prec, slices)
        e = torch.zeros(1, dtype=torch.float64, device=v.device)
        tctx.energy_async(0.25, _bind(_twins.get(Voo), voo), "ijab", _bind(_twins.get(T, 2), tp), "abij",
                          e.data_ptr())
        _checked(tctx)
        if recompute:
            fctx.save_for_backward(v, t, voo)
        else:
            fctx.save_for_backward(v, t, voo, tp)
        fctx.spec = spec
        return e[0]

    @staticmethod
    def backward(fctx, g):
        tctx, V, T, Voo, prec, slices, recompute = fctx.spec
        if recompute:
            v, t, voo = fctx.saved_tensors
            tp = _ladder_update(tctx, V, v, T, t, prec, slices)
        else:
            v, t, voo, tp = fctx.saved_tensors
        g, gp = _scale_ptr(g)
        # G = dE/dT' = 1/4 dE V_oovv(ijab) laid out as (abij)
        G = _zeros(T)
        tctx.add_scaled(_bind(_twins.get(T, 3), G), "abij", 0.0, _bind(_twins.get(Voo), voo), [(0.25, "ijab")], gp)
        # adjoint of the ladder T'(abij) = T + 1/2 V_vvvv(abef) T(efij) for the incoming G (one call):
        #   dT = G + 1/2 sum_ab V_vvvv(abef) G(abij),   dV_vvvv = 1/2 sum_ij G(abij) T(efij)
        dt = G.clone()
        dv = _zeros(V)
        tctx.contract_adjoint(0.5, _twins.get(T, 3), "abij", _bind(_twins.get(V), v), "abef", _bind(_twins.get(T), t),
                              "efij", dA=_bind(_twins.get(V, 1), dv), dB=_bind(_twins.get(T, 4), dt), beta=1.0,
                              precision=prec, slices=slices)
        # dV_oovv = 1/4 dE T'(abij) laid out as (ijab)
        dvoo = _zeros(Voo)
        tctx.add_scaled(_bind(_twins.get(Voo, 1), dvoo), "ijab", 0.0, _bind(_twins.get(T, 2), tp), [(0.25, "abij")],
                        gp)
        _checked(tctx)
        return dv, dt, dvoo, None


def _ladder_update(tctx, V, v, T, t, prec, slices) -> torch.Tensor:
    """T' = T + 1/2 V_vvvv(abef) T(efij)."""
    tp = t.detach().clone()
    tctx.contract(0.5, _bind(_twins.get(T, 2), tp), "abij", 1.0, _bind(_twins.get(V), v), "abef",
                  _bind(_twins.get(T), t), "efij", prec, slices)
    return tp


def ladder_energy(tctx: Context, V: Tensor, v: torch.Tensor, T: Tensor, t: torch.Tensor, Voo: Tensor,
                  voo: torch.Tensor, precision: str = "f64", slices: int = 0,
                  recompute: bool = False) -> torch.Tensor:
    """E = 1/4 V_oovv(ijab) (T + 1/2 V_vvvv(abef) T(efij))(abij), differentiable in v, t and voo.

    ``recompute`` keeps only the inputs for the backward pass and rebuilds T' there.
    """
    return _LadderEnergy.apply(v, t, voo, (tctx, V, T, Voo, precision, slices, recompute))
