"""The benchmark's own workload and configuration against the oracle at full size.

The O=40 V=240 doubles step (tiles 20/40, spin block sparsity) runs exactly as the benchmark runs
it: one FP64 pass, then every contraction autotuned for normwise relative error 1e-10 (slice
count, chunk length, tile policy, grid kind), then the split-precision step with slices = 0.
Each term then runs alone from a zeroed output, in that tuned configuration and in FP64, and is
compared with the oracle on seeded 4x4x4x4 boxes of its output blocks:

* ladder  R = 1/2 V_vvvv(abef) T(efij)
* intermediate W = W0 + V_oovv(mnef) T(efij)   (all of W: it is small)
* oooo    R = 1/4 T(abmn) W(mnij)
* ring    R = P(ab)P(ij) T(aeim) V_ovvo(mbej)  (four permuted oracle boxes per box)
* T1      R = V_vvvo(abej) t1(ei)
* energy  E = 1/4 V_oovv(ijab) T(abij)

Split precision <= 1e-10, FP64 <= 1e-12 (normwise over the sampled boxes).
"""
import numpy as np
import pytest

import oracle as O
import tamm_synth
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = {"ozaki_bf16": 1e-10, "f64": 1e-12}
N_BOXES = 24


def _fill_blocks(w, X, name, blocks):
    spec = w.tensors[name]
    lo, ext = X.block_lo_ext()
    idx = np.array(sorted(set(int(b) for b in blocks)), dtype=np.int64)
    if len(idx):
        tamm_synth.fill_boxes(w.seed, spec.stream, spec.sigma, X.dense_shape(), spec.anti01, spec.anti23,
                              lo[idx], ext[idx], X.block_off[idx], X.data)


def _needed_blocks(C, lc, A, la, B, lb, cblocks):
    """A and B blocks that the listed C blocks read."""
    import itertools

    lab = {}
    for X, l in ((C, lc), (A, la), (B, lb)):
        for m, ch in enumerate(l):
            lab[ch] = X.modes[m]
    summed = [ch for ch in la if ch not in lc]
    na, nb = set(), set()
    for cb in cblocks:
        tile = {ch: int(C.block_tiles[cb, m]) for m, ch in enumerate(lc)}
        for kt in itertools.product(*[range(lab[ch].n_tiles) for ch in summed]):
            tile.update(dict(zip(summed, kt)))
            ab = A.find_block([tile[ch] for ch in la])
            bb = B.find_block([tile[ch] for ch in lb])
            if ab >= 0 and bb >= 0:
                na.add(ab)
                nb.add(bb)
    return na, nb


def _boxes(R, rng, n):
    _, ext = R.block_lo_ext()
    cbs = [int(b) for b in rng.choice(R.n_blocks, n, replace=True)]
    los = [[int(rng.integers(0, e - 3)) for e in ext[b]] for b in cbs]
    return cbs, los


def _gpu_boxes(G, R, got, cbs, los):
    idx = {tuple(x): k for k, x in enumerate(G.block_tiles.tolist())}
    _, ext = R.block_lo_ext()
    out = []
    for b, lo in zip(cbs, los):
        k = idx[tuple(R.block_tiles[b].tolist())]
        blk = got[G.block_offsets[k]:G.block_offsets[k] + int(np.prod(ext[b]))].reshape(tuple(ext[b]))
        out.append(blk[lo[0]:lo[0] + 4, lo[1]:lo[1] + 4, lo[2]:lo[2] + 4, lo[3]:lo[3] + 4])
    return out


def _ring_oracle_boxes(ot, R, cbs, los):
    """Boxes of P(ab)P(ij) X with X = T(aeim) V_ovvo(mbej): four permuted boxes of X per box."""
    X = O.Tensor(R.modes, 2)
    perms = [((0, 1, 2, 3), 1.0), ((1, 0, 2, 3), -1.0), ((0, 1, 3, 2), -1.0), ((1, 0, 3, 2), 1.0)]
    xb, xlo = [], []
    for b, lo in zip(cbs, los):
        t = R.block_tiles[b]
        for p, _ in perms:
            xb.append(X.find_block([int(t[q]) for q in p]))
            xlo.append([lo[q] for q in p])
    vals = O.contract_boxes(1.0, X, "abij", ot["T"], "aeim", ot["V_ovvo"], "mbej", xb, xlo, [[4] * 4] * len(xb))
    out = []
    for i in range(len(cbs)):
        acc = np.zeros((4, 4, 4, 4))
        for k, (p, s) in enumerate(perms):
            acc += s * np.transpose(vals[4 * i + k], np.argsort(p))
        out.append(acc)
    return out


@pytest.fixture(scope="module")
def headline():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_doubles_o40_v240()
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w)
    run = gw.Runner(ctx, w, gsp, gt)
    run.run("f64")  # intermediates hold the values the tuned contractions see
    tuned = run.autotune(1e-10)
    ctx.sync()
    print({k: (v["slices"], v["chunk_k"], v["tile_policy"], v["persistent"]) for k, v in tuned.items()})

    # oracle: full small tensors, only the needed blocks of the large ones
    spaces = {k: O.Space.from_spec(s) for k, s in w.spaces.items()}
    ot = {n: O.Tensor([spaces[m] for m in t.modes], t.n_upper, t.sym) for n, t in w.tensors.items()}
    for n in ("T", "V_oovv", "W0", "V_ovvo", "t1"):
        ot[n].fill_synthetic(w.seed, w.tensors[n])
    rng = np.random.default_rng(2201)
    boxes = {name: _boxes(ot["R"], rng, N_BOXES) for name in ("ladder", "oooo", "ring", "t1")}
    for name, (A, la) in (("ladder", ("V_vvvv", "abef")), ("t1", ("V_vvvo", "abej"))):
        na, _ = _needed_blocks(ot["R"], "abij", ot[A], la, ot["T" if name == "ladder" else "t1"],
                               "efij" if name == "ladder" else "ei", boxes[name][0])
        _fill_blocks(w, ot[A], A, na)
    # W = W0 + V_oovv T in full
    ot["W"].data[:] = ot["W0"].data
    O.contract(1.0, ot["W"], "mnij", 1.0, ot["V_oovv"], "mnef", ot["T"], "efij")
    ref = {
        "ladder": O.contract_boxes(0.5, ot["R"], "abij", ot["V_vvvv"], "abef", ot["T"], "efij", boxes["ladder"][0],
                                   boxes["ladder"][1], [[4] * 4] * N_BOXES),
        "oooo": O.contract_boxes(0.25, ot["R"], "abij", ot["T"], "abmn", ot["W"], "mnij", boxes["oooo"][0],
                                 boxes["oooo"][1], [[4] * 4] * N_BOXES),
        "ring": _ring_oracle_boxes(ot, ot["R"], *boxes["ring"]),
        "t1": O.contract_boxes(1.0, ot["R"], "abij", ot["V_vvvo"], "abej", ot["t1"], "ei", boxes["t1"][0],
                               boxes["t1"][1], [[4] * 4] * N_BOXES),
    }
    energy = O.energy(0.25, ot["V_oovv"], "ijab", ot["T"], "abij")
    return ctx, w, run, gt, ot, boxes, ref, energy


@pytest.mark.parametrize("precision", ["ozaki_bf16", "f64"])
def test_every_term_in_tuned_configuration_matches_oracle(headline, precision):
    import torch

    ctx, w, run, gt, ot, boxes, ref, energy = headline
    steps = {s.name: s for s in w.steps}
    # the whole step first, as the benchmark times it (W must hold W0 + V_oovv T afterwards)
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    run.run(precision, 0, energy_out=e_dev.data_ptr())
    ctx.sync()
    errs = {"W": rel_err(gpu_to_oracle_layout(gt["W"], ot["W"]), ot["W"].data),
            "energy": abs(float(e_dev.item()) - energy) / abs(energy)}
    # then each R term alone, from a zeroed R (the ladder overwrites R; the others accumulate)
    for name in ("ladder", "oooo", "ring", "t1"):
        gt["R"].data.zero_()
        run.run(precision, 0, steps=[steps[name]])
        ctx.sync()
        got = _gpu_boxes(gt["R"], ot["R"], gt["R"].download(), *boxes[name])
        errs[name] = rel_err(np.concatenate([g.ravel() for g in got]),
                             np.concatenate([r.ravel() for r in ref[name]]))
    print(precision, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= TOL[precision], (precision, k, v)
