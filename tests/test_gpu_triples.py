"""The perturbative triples correction E(T) (Sec. IV.B, Eqs. cc14, tensort, tensort2) on the GPU
against the oracle on the same seeded inputs (``triples`` recipe: T2, t1, V_ooov, V_vovv, V_oovv,
orbital energies).

* O=16 V=64, even and ragged tiles: E(T) in FP64 (<= 1e-12) and split precision (<= 1e-10);
* each occupied triple's contribution (a<b<c restricted) against the oracle's W and Y of that triple;
* the batching of triples through the workspace changes nothing (bitwise);
* at the benchmark's size (O=32 V=160) sampled triples' contributions against the oracle;
* refusals: another precision, mismatched spaces.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

pytestmark = pytest.mark.gpu


def _setup(O_, V_, to, tv):
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.triples(O_, V_, to, tv)
    ctx = tg.Context(0)
    _, gt = gw.build(ctx, w)
    eo, ev = wl.orbital_energies(w)
    deo = torch.tensor(eo, dtype=torch.float64, device="cuda:0")
    dev = torch.tensor(ev, dtype=torch.float64, device="cuda:0")
    return w, ctx, gt, eo, ev, deo, dev


def _gpu_energy(ctx, gt, deo, dev, precision, slices=0, ws=0, per_triple=False):
    import torch

    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    no = gt["T"].modes[2].n
    n_trip = no * (no - 1) * (no - 2) // 6
    pt = torch.zeros(max(n_trip, 1), dtype=torch.float64, device="cuda:0") if per_triple else None
    ctx.triples_energy(gt["T"], gt["t1"], gt["V_ooov"], gt["V_vovv"], gt["V_oovv"], deo.data_ptr(), dev.data_ptr(),
                       out.data_ptr(), precision, slices, ws, pt.data_ptr() if per_triple else 0)
    ctx.sync()
    return float(out.item()), (pt.cpu().numpy() if per_triple else None)


def _oracle_triple(T, eo, ev, i, j, k):
    """One occupied triple's sum over a<b<c of (W + Y) W / D, from the oracle's W and Y."""
    W, Y = O.triples_wy(T, i, j, k)
    nv = len(ev)
    a, b, c = np.meshgrid(np.arange(nv), np.arange(nv), np.arange(nv), indexing="ij")
    mask = (a < b) & (b < c)
    D = eo[i] + eo[j] + eo[k] - ev[a] - ev[b] - ev[c]
    return float(np.sum(((W + Y) * W / D)[mask]))


@pytest.fixture(scope="module", params=[(16, 64, 4, 16), (16, 64, 3, 12)], ids=["even", "ragged"])
def small(request):
    O_, V_, to, tv = request.param
    w, ctx, gt, eo, ev, deo, dev = _setup(O_, V_, to, tv)
    _, ot = O.build_workload(w)
    e_ref = O.triples_energy(ot, eo, ev)
    return w, ctx, gt, ot, eo, ev, deo, dev, e_ref


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("ozaki_bf16", 1e-10)])
def test_triples_energy_matches_oracle(small, precision, tol):
    w, ctx, gt, ot, eo, ev, deo, dev, e_ref = small
    e, _ = _gpu_energy(ctx, gt, deo, dev, precision)
    err = abs(e - e_ref) / abs(e_ref)
    print(f"{w.name} {precision}: E(T) {e:.15e} oracle {e_ref:.15e} rel err {err:.2e}")
    assert e_ref < 0 and err <= tol


def test_per_triple_contributions_and_batching(small):
    w, ctx, gt, ot, eo, ev, deo, dev, e_ref = small
    e1, pt1 = _gpu_energy(ctx, gt, deo, dev, "f64", per_triple=True)
    no = len(eo)
    trip = list(itertools.combinations(range(no), 3))
    assert len(pt1) == len(trip)
    for n in (0, 1, len(trip) // 2, len(trip) - 1):
        ref = _oracle_triple(ot, eo, ev, *trip[n])
        assert abs(pt1[n] - ref) <= 1e-12 * abs(e_ref), (trip[n], pt1[n], ref)
    # a workspace of one triple at a time: the same partials, so the same sums bit for bit
    e2, pt2 = _gpu_energy(ctx, gt, deo, dev, "f64", ws=8, per_triple=True)
    assert ctx.triples_info(gt["T"], gt["t1"], gt["V_ooov"], gt["V_vovv"], gt["V_oovv"], 8)["n_batches"] == len(trip)
    assert e2 == e1 and np.array_equal(pt1, pt2)
    e3, _ = _gpu_energy(ctx, gt, deo, dev, "ozaki_bf16", ws=1 << 20)
    e4, _ = _gpu_energy(ctx, gt, deo, dev, "ozaki_bf16")
    assert e3 == e4


def test_triples_refusals(small):
    import paper_2201_01257_gb300 as tg

    w, ctx, gt, ot, eo, ev, deo, dev, e_ref = small
    with pytest.raises(tg.TammError) as e:
        _gpu_energy(ctx, gt, deo, dev, "bf16x3")
    assert e.value.status == tg.TAMM_EUNSUPPORTED
    with pytest.raises(tg.TammError) as e:  # V_oovv in the place of V_ooov: wrong spaces
        ctx.triples_energy(gt["T"], gt["t1"], gt["V_oovv"], gt["V_vovv"], gt["V_oovv"], deo.data_ptr(),
                           dev.data_ptr(), deo.data_ptr())
    assert e.value.status == tg.TAMM_EINVAL


@pytest.mark.slow
def test_triples_o32_v160_sampled_triples():
    # the benchmark's workload: split precision and FP64, each sampled triple's contribution
    w, ctx, gt, eo, ev, deo, dev = _setup(32, 160, 16, 80)
    spaces = {k: O.Space.from_spec(s) for k, s in w.spaces.items()}
    ot = {n: O.Tensor([spaces[m] for m in t.modes], t.n_upper, t.sym) for n, t in w.tensors.items()}
    for n, t in w.tensors.items():
        ot[n].fill_synthetic(w.seed, t)
    no = len(eo)
    trip = list(itertools.combinations(range(no), 3))
    rng = np.random.default_rng(32160)
    picks = sorted(int(x) for x in rng.choice(len(trip), 4, replace=False))
    refs = {n: _oracle_triple(ot, eo, ev, *trip[n]) for n in picks}
    for precision, tol in (("ozaki_bf16", 1e-10), ("f64", 1e-12)):
        e, pt = _gpu_energy(ctx, gt, deo, dev, precision, per_triple=True)
        num = sum((pt[n] - refs[n]) ** 2 for n in picks) ** 0.5
        den = sum(refs[n] ** 2 for n in picks) ** 0.5
        print(f"O=32 V=160 {precision}: E(T) {e:.12e}, sampled triples rel err {num / den:.2e}")
        assert num / den <= tol
