"""Doubles contractions at full size on the GPU: ladder + ring + oooo, O=80 / V=320 spin-orbitals,
tiles 40/64 (V_vvvv about 31.5 GB FP64).  The oracle recomputes 256 seeded
8x8x8x8 sub-blocks of the outputs (seeded over contraction, output block and
offset); split precision is held to 1e-10 and FP64 to 1e-12 normwise over them.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def doubles80():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_doubles_o80_v320()
    names = {"V_vvvv", "T", "W0", "V_ovvo"}
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w, only=names | {"R", "X"})
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces, {k: w.tensors[k] for k in names | {"R"}}))
    boxes = sample_boxes(ot)
    return ctx, gsp, gt, ot, w, boxes, oracle_refs(ot, boxes)


def sample_boxes(ot, n=256, box=8, seed=5):
    """(contraction, output block, lower corner) triples, seeded."""
    rng = np.random.default_rng(seed)
    R = ot["R"]
    _, ext = R.block_lo_ext()
    out = []
    for _ in range(n):
        c = ["ladder", "ring", "oooo"][int(rng.integers(3))]
        b = int(rng.integers(R.n_blocks))
        lo = [int(rng.integers(0, e - box + 1)) for e in ext[b]]
        out.append((c, b, lo))
    return out


TERMS = {
    "ladder": (0.5, "V_vvvv", "abef", "T", "efij"),
    "oooo": (0.25, "T", "abmn", "W0", "mnij"),
}


def gpu_term(ctx, gt, name, prec):
    R = gt["R"]
    R.data.zero_()
    if name == "ring":
        from paper_2201_01257_gb300 import workload as gw

        step = wl.ContractSpec("ring", "R", "abij", "T", "aeim", "V_ovvo", "mbej", 1.0, beta=0.0, antisym=True)
        gw.Runner(ctx, None, None, gt).run_step(step, prec, 0)
    else:
        al, a, la, b, lb = TERMS[name]
        ctx.contract(al, R, "abij", 0.0, gt[a], la, gt[b], lb, prec, 0)
    ctx.sync()
    return R.download()


def oracle_refs(ot, boxes, box=8):
    """Reference values of every sampled box, evaluated by the oracle in parallel per contraction."""
    R = ot["R"]
    ext = [box] * 4
    refs = {}
    for name in ("ladder", "oooo"):
        sel = [(i, b, lo) for i, (c, b, lo) in enumerate(boxes) if c == name]
        if sel:
            al, a, la, bb, lb = TERMS[name]
            vals = O.contract_boxes(al, R, "abij", ot[a], la, ot[bb], lb, [b for _, b, _ in sel],
                                    [lo for _, _, lo in sel], [ext] * len(sel))
            refs.update({i: v for (i, _, _), v in zip(sel, vals)})
    # ring: P(ab)P(ij) X with X = T(aeim) V(mbej), from the four permuted boxes of X
    sel = [(i, b, lo) for i, (c, b, lo) in enumerate(boxes) if c == "ring"]
    terms = ((1.0, (0, 1, 2, 3)), (-1.0, (1, 0, 2, 3)), (-1.0, (0, 1, 3, 2)), (1.0, (1, 0, 3, 2)))
    jobs = []
    for i, b, lo in sel:
        refs[i] = np.zeros((box,) * 4)
        for sign, perm in terms:
            xb = R.find_block(R.block_tiles[b][list(perm)])
            if xb >= 0:
                jobs.append((i, sign, perm, xb, [lo[p] for p in perm]))
    if jobs:
        vals = O.contract_boxes(1.0, R, "abij", ot["T"], "aeim", ot["V_ovvo"], "mbej", [j[3] for j in jobs],
                                [j[4] for j in jobs], [ext] * len(jobs))
        for (i, sign, perm, _, _), v in zip(jobs, vals):
            refs[i] += sign * np.transpose(v, np.argsort(perm))
    return refs


@pytest.mark.parametrize("prec,tol", [("ozaki_bf16", 1e-10), ("f64", 1e-12)])
def test_doubles_o80_v320_sampled_sub_blocks(doubles80, prec, tol):
    ctx, gsp, gt, ot, w, boxes, refs = doubles80
    R = gt["R"]
    idx = {tuple(t): k for k, t in enumerate(R.block_tiles.tolist())}
    _, ext_all = ot["R"].block_lo_ext()
    for name in ("ladder", "ring", "oooo"):
        sel = [(i, b, lo) for i, (c, b, lo) in enumerate(boxes) if c == name]
        if not sel:
            continue
        got_all = gpu_term(ctx, gt, name, prec)
        num = den = 0.0
        for i, b, lo in sel:
            ext = ext_all[b]
            k = idx[tuple(ot["R"].block_tiles[b].tolist())]
            blk = got_all[R.block_offsets[k]:R.block_offsets[k] + int(np.prod(ext))].reshape(tuple(ext))
            sub = blk[lo[0]:lo[0] + 8, lo[1]:lo[1] + 8, lo[2]:lo[2] + 8, lo[3]:lo[3] + 8]
            ref = refs[i]
            num += float(np.sum((sub - ref) ** 2))
            den += float(np.sum(ref ** 2))
        err = np.sqrt(num / den)
        print(f"O=80 V=320 {name} {prec}: {len(sel)} boxes, rel err {err:.3e}")
        assert err <= tol, (name, prec, err)
