"""Uneven D2h blocks (O=64, V=384 spin-orbitals; irrep counts and tile cuts seeded, tiles
8..96 per (spin, irrep) group), spin and irrep block sparsity.

* The vvvv ladder and the ring term run as one contraction group (one grouped tcgen05 launch over
  every nonzero block pair of both), in split precision and in FP64 one by one; the oracle
  recomputes 192 seeded sub-blocks (up to 4^4, clipped to small tiles) of both outputs.
* Grouped execution is bitwise equal to running the contractions one by one.
* A CUDA graph of the grouped step replays bitwise equal to eager execution, also after the
  inputs change in place.
* A batch of 32 independent ladders with sizes drawn like the full batch and scaled down
  (O/2, V/4, tiles 5/10) runs as one grouped launch inside one graph; each problem's output is
  checked against the oracle on seeded sub-blocks.
* Calls that would break a group or a capture are refused with TAMM_EINVAL.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

pytestmark = pytest.mark.gpu

BOX = 4


@pytest.fixture(scope="module")
def irrep():
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.irrep_doubles()
    stream = torch.cuda.Stream(0)
    ctx = tg.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        gsp, gt = gw.build(ctx, w)
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces,
                                         {k: w.tensors[k] for k in ("V_vvvv", "T", "V_ovvo", "R")}))
    boxes = sample_boxes(ot["R"], 192, seed=3)
    refs = oracle_refs(ot, boxes)
    return ctx, stream, gw.Runner(ctx, w, gsp, gt), ot, boxes, refs


def sample_boxes(R, n, seed):
    rng = np.random.default_rng(seed)
    _, ext = R.block_lo_ext()
    out = []
    for _ in range(n):
        c = ["ladder", "ring"][int(rng.integers(2))]
        b = int(rng.integers(R.n_blocks))
        e = [min(BOX, x) for x in ext[b]]
        lo = [int(rng.integers(0, x - y + 1)) for x, y in zip(ext[b], e)]
        out.append((c, b, lo, e))
    return out


def oracle_refs(ot, boxes):
    R = ot["R"]
    refs = {}
    sel = [(i, b, lo, e) for i, (c, b, lo, e) in enumerate(boxes) if c == "ladder"]
    vals = O.contract_boxes(0.5, R, "abij", ot["V_vvvv"], "abef", ot["T"], "efij", [s[1] for s in sel],
                            [s[2] for s in sel], [s[3] for s in sel])
    refs.update({s[0]: v for s, v in zip(sel, vals)})
    # ring: P(ab)P(ij) X with X(abij) = T(aeim) V_ovvo(mbej), from the four permuted boxes of X
    terms = ((1.0, (0, 1, 2, 3)), (-1.0, (1, 0, 2, 3)), (-1.0, (0, 1, 3, 2)), (1.0, (1, 0, 3, 2)))
    jobs = []
    for i, b, lo, e in [(i, b, lo, e) for i, (c, b, lo, e) in enumerate(boxes) if c == "ring"]:
        refs[i] = np.zeros(tuple(e))
        for sign, perm in terms:
            xb = R.find_block(R.block_tiles[b][list(perm)])
            if xb >= 0:
                jobs.append((i, sign, perm, xb, [lo[p] for p in perm], [e[p] for p in perm]))
    vals = O.contract_boxes(1.0, R, "abij", ot["T"], "aeim", ot["V_ovvo"], "mbej", [j[3] for j in jobs],
                            [j[4] for j in jobs], [j[5] for j in jobs])
    for (i, sign, perm, _, _, _), v in zip(jobs, vals):
        refs[i] += sign * np.transpose(v, np.argsort(perm))
    return refs


def box_error(G, R, got, boxes, refs, name):
    idx = {tuple(t): k for k, t in enumerate(G.block_tiles.tolist())}
    _, ext_all = R.block_lo_ext()
    num = den = 0.0
    for i, (c, b, lo, e) in enumerate(boxes):
        if c != name:
            continue
        k = idx[tuple(R.block_tiles[b].tolist())]
        blk = got[G.block_offsets[k]:G.block_offsets[k] + int(np.prod(ext_all[b]))].reshape(tuple(ext_all[b]))
        sub = blk[tuple(slice(l, l + x) for l, x in zip(lo, e))]
        num += float(np.sum((sub - refs[i]) ** 2))
        den += float(np.sum(refs[i] ** 2))
    return float(np.sqrt(num / den))


def run_step(ctx, stream, runner, prec, grouped):
    import torch

    T = runner.tensors
    with torch.cuda.stream(stream):
        T["R"].data.zero_()
        T["R2"].data.zero_()
    if grouped:
        runner.run_grouped(runner.w.steps, prec)
    else:
        runner.run(prec)
    ctx.sync()
    return T["R"].download(), T["R2"].download()


@pytest.mark.parametrize("prec,tol,grouped", [("ozaki_bf16", 1e-10, True), ("f64", 1e-12, False)])
def test_irrep_doubles_match_oracle(irrep, prec, tol, grouped):
    ctx, stream, runner, ot, boxes, refs = irrep
    R, R2 = run_step(ctx, stream, runner, prec, grouped)
    G = runner.tensors["R"]
    for name, got in (("ladder", R), ("ring", R2)):
        err = box_error(G, ot["R"], got, boxes, refs, name)
        print(f"irrep {name} {prec}: rel err {err:.3e}")
        assert err <= tol, (name, prec, err)


def test_grouped_equals_separate_bitwise(irrep):
    ctx, stream, runner, ot, boxes, refs = irrep
    a = run_step(ctx, stream, runner, "ozaki_bf16", False)
    b = run_step(ctx, stream, runner, "ozaki_bf16", True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graph_replay_equals_eager(irrep):
    import torch

    ctx, stream, runner, ot, boxes, refs = irrep
    T = runner.tensors
    eager = run_step(ctx, stream, runner, "ozaki_bf16", True)  # also creates every plan and the scratch
    n0 = ctx.launch_count()
    with torch.cuda.stream(stream):
        ctx.graph_begin()
        try:
            runner.run_grouped(runner.w.steps, "ozaki_bf16")
        finally:
            g = ctx.graph_end()
    assert ctx.launch_count() - n0 == g.kernel_launches > 0
    for _ in range(2):
        with torch.cuda.stream(stream):
            T["R"].data.fill_(np.nan)  # beta = 0: the replay overwrites every stored entry
            T["R2"].data.zero_()
        g.launch()
        ctx.sync()
        assert np.array_equal(T["R"].download(), eager[0])
        assert np.array_equal(T["R2"].download(), eager[1])
    # the graph reads the inputs at replay time: scale T in place and the outputs follow
    with torch.cuda.stream(stream):
        T["T"].data.mul_(2.0)
        T["R2"].data.zero_()
    g.launch()
    ctx.sync()
    r, r2 = T["R"].download(), T["R2"].download()
    with torch.cuda.stream(stream):
        T["T"].data.mul_(0.5)
    ctx.sync()
    assert np.array_equal(r, 2.0 * eager[0]) and np.array_equal(r2, 2.0 * eager[1])
    g.destroy()


def test_group_and_capture_refusals(irrep):
    import torch

    import paper_2201_01257_gb300 as tg

    ctx, stream, runner, ot, boxes, refs = irrep
    T = runner.tensors
    # an add inside a group, an FP64 contraction inside a group
    ctx.group_begin()
    with pytest.raises(tg.TammError) as e:
        ctx.add(T["R2"], "abij", 1.0, T["R"], [(1.0, "abij")])
    assert e.value.status == tg.TAMM_EINVAL
    with pytest.raises(tg.TammError):
        ctx.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", "f64")
    ctx.lib.tamm_group_cancel(ctx.handle)
    # a contraction whose output is another's input
    ctx.group_begin()
    ctx.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", "ozaki_bf16")
    ctx.contract(0.5, T["R2"], "abij", 0.0, T["V_vvvv"], "abef", T["R"], "efij", "ozaki_bf16")
    with pytest.raises(tg.TammError) as e:
        ctx.group_end()
    assert e.value.status == tg.TAMM_EINVAL and "overlaps" in str(e.value)
    # capture on the legacy default stream, and a synchronising call inside a capture
    ctx0 = tg.Context(0, stream=torch.cuda.default_stream(0))
    with pytest.raises(tg.TammError):
        ctx0.graph_begin()
    with torch.cuda.stream(stream):
        ctx.graph_begin()
        with pytest.raises(tg.TammError):
            ctx.norm(T["R"])
        with pytest.raises(tg.TammError) as e:
            ctx.graph_end()
    assert "failed" in str(e.value)
    ctx.sync()


def test_scaled_batch_in_one_graph(irrep):
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    sizes = [(max(4, o // 2), max(8, v // 4)) for o, v in wl.ladder_batch_sizes()]
    sizes = [(o + o % 2, v + v % 2) for o, v in sizes]
    stream = torch.cuda.Stream(0)
    ctx = tg.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        probs = gw.build_batch(ctx, sizes, wl.SEED_BASE + 300, (5, 10))

        def step():
            with ctx.group():
                for w, r in probs:
                    T = r.tensors
                    ctx.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", "ozaki_bf16")

        ctx.profile(True)
        n0 = ctx.launch_count()
        step()
        ctx.sync()
        eager_launches = ctx.launch_count() - n0
        prof = ctx.profile_read()
        ctx.profile(False)
        eager = [r.tensors["R"].download() for _, r in probs]
        ctx.graph_begin()
        try:
            step()
        finally:
            g = ctx.graph_end()
        for _, r in probs:
            r.tensors["R"].data.fill_(np.nan)
        g.launch()
    ctx.sync()
    # two slicing launches per problem, one grouped GEMM for all 32, and the summed-range reductions
    # of the problems too small to fill the GPU alone
    assert prof["gemm_ozaki"][1] == 1 and prof["slice"][1] == 2 * len(probs)
    assert g.kernel_launches == eager_launches == 2 * len(probs) + 1 + prof["split_reduce"][1]
    for (w, r), e in zip(probs, eager):
        assert np.array_equal(r.tensors["R"].download(), e)
    worst = 0.0
    for k, ((w, r), got) in enumerate(zip(probs, eager)):
        _, ot = O.build_workload(w)
        boxes = [(c, b, lo, ext) for c, b, lo, ext in sample_boxes(ot["R"], 12, seed=k)]
        boxes = [("ladder", b, lo, ext) for _, b, lo, ext in boxes]
        vals = O.contract_boxes(0.5, ot["R"], "abij", ot["V_vvvv"], "abef", ot["T"], "efij",
                                [s[1] for s in boxes], [s[2] for s in boxes], [s[3] for s in boxes])
        err = box_error(r.tensors["R"], ot["R"], got, boxes, dict(enumerate(vals)), "ladder")
        worst = max(worst, err)
        assert err <= 1e-10, (k, w.name, err)
    print(f"scaled batch of {len(probs)} ladders: worst rel err {worst:.3e}")
