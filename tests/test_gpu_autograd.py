"""Gradients through torch.autograd (ladder energy, O=32, V=192 spin-orbitals, tiles 16/32).

E = 1/4 V_oovv(ijab) T'(abij),  T' = T + 1/2 V_vvvv(abef) T(efij).

* FP64 autograd gradients vs the oracle's closed forms on seeded sub-blocks (<= 1e-12);
* vs central finite differences (step 1e-6) of the FP64 forward on 64 seeded stored entries
  (32 of T, 16 of V_vvvv, 16 of V_oovv).  E is affine in every single entry, so the
  difference quotient is exact up to rounding;
* split precision (6 slices, <= 1e-10) and BF16x3 (<= 1e-5) vs FP64 gradients;
* recomputing T' in the backward pass gives the same gradients as storing it;
* the generic contract/energy functions give the same gradients as the fused adjoint.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ladder_energy():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ladder_energy_o32_v192()
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w)
    _, ot = O.build_workload(w)
    return ctx, gt, ot


def grads(ctx, gt, precision="f64", recompute=False):
    import torch

    from paper_2201_01257_gb300 import autograd as ga

    v = gt["V_vvvv"].data.clone().requires_grad_(True)
    t = gt["T"].data.clone().requires_grad_(True)
    voo = gt["V_oovv"].data.clone().requires_grad_(True)
    E = ga.ladder_energy(ctx, gt["V_vvvv"], v, gt["T"], t, gt["V_oovv"], voo, precision, 0, recompute)
    E.backward()
    torch.cuda.synchronize()
    return float(E.item()), {k: x.grad.detach().cpu().numpy()[: gt[n].n_elems]
                             for k, x, n in (("V_vvvv", v, "V_vvvv"), ("T", t, "T"), ("V_oovv", voo, "V_oovv"))}


def oracle_ref_boxes(ot, n_boxes=96, seed=4):
    """Closed-form FP64 gradients on seeded 4^4 boxes: {name: [(block, lo, values)]}."""
    rng = np.random.default_rng(seed)
    T, V, Voo = ot["T"], ot["V_vvvv"], ot["V_oovv"]
    G = O.Tensor(T.modes, 2)
    O.add(0.25, G, "abij", 0.0, Voo, "ijab")
    out = {}
    for name, X in (("T", T), ("V_vvvv", V)):
        _, ext = X.block_lo_ext()
        bl = rng.integers(X.n_blocks, size=n_boxes)
        lo = [[int(rng.integers(0, e - 3)) for e in ext[b]] for b in bl]
        if name == "T":
            vals = O.contract_boxes(0.5, T, "efij", V, "abef", G, "abij", bl, lo, [[4] * 4] * n_boxes)
            gv = [G.block_view(G.find_block(T.block_tiles[b]))[l[0]:l[0] + 4, l[1]:l[1] + 4, l[2]:l[2] + 4,
                                                                l[3]:l[3] + 4] for b, l in zip(bl, lo)]
            vals = [x + y for x, y in zip(vals, gv)]
        else:
            vals = O.contract_boxes(0.5, V, "abef", G, "abij", T, "efij", bl, lo, [[4] * 4] * n_boxes)
        out[name] = list(zip(bl, lo, vals))
    # dE/dV_oovv[ijab] = 1/4 T'[abij], T' = T + 1/2 V T: boxes of T' at the transposed position
    _, ext = Voo.block_lo_ext()
    bl = rng.integers(Voo.n_blocks, size=n_boxes)
    lo = [[int(rng.integers(0, e - 3)) for e in ext[b]] for b in bl]
    tb = [T.find_block(Voo.block_tiles[b][[2, 3, 0, 1]]) for b in bl]
    tlo = [[l[2], l[3], l[0], l[1]] for l in lo]
    lad = O.contract_boxes(0.5, T, "abij", V, "abef", T, "efij", tb, tlo, [[4] * 4] * n_boxes)
    vals = []
    for b, l, x in zip(tb, tlo, lad):
        tp = T.block_view(b)[l[0]:l[0] + 4, l[1]:l[1] + 4, l[2]:l[2] + 4, l[3]:l[3] + 4] + x
        vals.append(0.25 * np.transpose(tp, (2, 3, 0, 1)))
    out["V_oovv"] = list(zip(bl, lo, vals))
    return out


def test_fp64_gradients_match_oracle_closed_forms(ladder_energy):
    ctx, gt, ot = ladder_energy
    E, g = grads(ctx, gt)
    refs = oracle_ref_boxes(ot)
    for name, boxes in refs.items():
        X = ot[name]
        got = gpu_to_oracle_layout_from(gt[name], X, g[name])
        num = den = 0.0
        _, ext = X.block_lo_ext()
        for b, lo, ref in boxes:
            blk = got[X.block_off[b]:X.block_off[b] + int(np.prod(ext[b]))].reshape(tuple(ext[b]))
            sub = blk[lo[0]:lo[0] + 4, lo[1]:lo[1] + 4, lo[2]:lo[2] + 4, lo[3]:lo[3] + 4]
            num += float(np.sum((sub - ref) ** 2))
            den += float(np.sum(ref ** 2))
        err = np.sqrt(num / den)
        print(f"dE/d{name} vs oracle closed form: {err:.2e}")
        assert err <= 1e-12, (name, err)


def gpu_to_oracle_layout_from(G, R, values):
    out = np.empty(R.n_elems)
    idx = {tuple(t): k for k, t in enumerate(G.block_tiles.tolist())}
    ends = list(R.block_off[1:]) + [R.n_elems]
    for b in range(R.n_blocks):
        k = idx[tuple(R.block_tiles[b].tolist())]
        n = ends[b] - R.block_off[b]
        out[R.block_off[b]:R.block_off[b] + n] = values[G.block_offsets[k]:G.block_offsets[k] + n]
    return out


def test_gradients_match_central_differences(ladder_energy):
    import torch

    ctx, gt, ot = ladder_energy
    E0, g = grads(ctx, gt)
    rng = np.random.default_rng(64)
    h = 1e-6
    T, V, Voo = gt["T"], gt["V_vvvv"], gt["V_oovv"]

    def energy(v, t, voo):
        tp = t.clone()
        ctx.contract(0.5, bindT(tp), "abij", 1.0, bindV(v), "abef", bindT2(t), "efij", "f64", 0)
        return ctx.energy(0.25, bindVoo(voo), "ijab", bindT(tp), "abij")

    from paper_2201_01257_gb300 import autograd as ga

    bindT = lambda x: ga._bind(ga._twins.get(T, 7), x)
    bindT2 = lambda x: ga._bind(ga._twins.get(T, 8), x)
    bindV = lambda x: ga._bind(ga._twins.get(V, 7), x)
    bindVoo = lambda x: ga._bind(ga._twins.get(Voo, 7), x)
    v0, t0, voo0 = V.data.clone(), T.data.clone(), Voo.data.clone()
    picks = [("T", 32), ("V_vvvv", 16), ("V_oovv", 16)]
    worst = 0.0
    for name, n in picks:
        host = {"T": t0, "V_vvvv": v0, "V_oovv": voo0}[name].cpu().numpy()
        cand = np.flatnonzero(np.abs(host[: gt[name].n_elems]) > 0)  # stored, off-diagonal entries
        for idx in rng.choice(cand, n, replace=False):
            vals = []
            for s in (1.0, -1.0):
                bufs = {"T": t0.clone(), "V_vvvv": v0, "V_oovv": voo0}
                if name != "T":
                    bufs[name] = bufs[name].clone()
                bufs[name][int(idx)] += s * h
                vals.append(energy(bufs["V_vvvv"], bufs["T"], bufs["V_oovv"]))
            fd = (vals[0] - vals[1]) / (2 * h)
            gr = g[name][int(idx)]
            err = abs(fd - gr)
            worst = max(worst, err / max(abs(gr), 1e-3))
            assert err <= 1e-9 + 1e-6 * abs(gr), (name, int(idx), fd, gr)
    print(f"worst FD relative deviation {worst:.2e}")


@pytest.mark.parametrize("precision,tol", [("ozaki_bf16", 1e-10), ("bf16x3", 1e-5)])
def test_split_precision_gradients(ladder_energy, precision, tol):
    ctx, gt, ot = ladder_energy
    E64, g64 = grads(ctx, gt)
    E, g = grads(ctx, gt, precision)
    for k in g:
        err = rel_err(g[k], g64[k])
        print(f"{precision} dE/d{k}: {err:.2e}")
        assert err <= tol, (k, err)
    assert abs(E - E64) <= tol * abs(E64)


def test_recompute_matches_stored(ladder_energy):
    ctx, gt, ot = ladder_energy
    E1, g1 = grads(ctx, gt, recompute=False)
    E2, g2 = grads(ctx, gt, recompute=True)
    assert E1 == E2
    for k in g1:
        assert np.array_equal(g1[k], g2[k])


def test_generic_functions_match_fused_adjoint(ladder_energy):
    import torch

    from paper_2201_01257_gb300 import autograd as ga

    ctx, gt, ot = ladder_energy
    E1, g1 = grads(ctx, gt)
    T, V, Voo = gt["T"], gt["V_vvvv"], gt["V_oovv"]
    v = V.data.clone().requires_grad_(True)
    t = T.data.clone().requires_grad_(True)
    voo = Voo.data.clone().requires_grad_(True)
    x = ga.contract(ctx, 0.5, T, "abij", V, v, "abef", T, t, "efij")
    tp = t + x  # T and x share one block layout, so T' is the sum of the packed buffers
    E = ga.energy(ctx, 0.25, Voo, voo, "ijab", T, tp, "abij")
    E.backward()
    torch.cuda.synchronize()
    assert abs(float(E.item()) - E1) <= 1e-13 * abs(E1)
    for k, xx in (("V_vvvv", v), ("T", t), ("V_oovv", voo)):
        got = xx.grad.detach().cpu().numpy()[: gt[k].n_elems]
        assert rel_err(got, g1[k]) <= 1e-13, k
