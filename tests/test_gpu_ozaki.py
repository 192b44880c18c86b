"""GPU split-precision (BF16-slice Ozaki) path vs the FP64 oracle.

Bound: normwise relative error <= 1e-10 for every contraction at the default
6 slices (41 significant bits per operand row/column); exact results when
every input has few enough bits for the slices to hold it exactly.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def run_both(tg, w, precision="ozaki_bf16", slices=0):
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w)
    runner = gw.Runner(ctx, w, gsp, gt)
    ge = runner.run(precision, slices)
    ctx.sync()
    _, ot = O.build_workload(w)
    oe = O.run_workload(w, ot)
    return ctx, gt, ot, ge, oe


def test_ladder_o8_v32_ozaki(gpu_lib):
    _, gt, ot, _, _ = run_both(gpu_lib, wl.ladder_o8_v32())
    err = rel_err(gpu_to_oracle_layout(gt["R"], ot["R"]), ot["R"].data)
    assert err <= TOL, err


@pytest.mark.parametrize("O_,V_,to,tv", [(8, 24, 2, 4), (12, 36, 3, 5), (10, 34, 4, 7), (16, 40, 8, 10)])
def test_small_doubles_all_steps_ozaki(gpu_lib, O_, V_, to, tv):
    # odd tile sizes: M, N, K not multiples of 128/16, ragged N tiles, padded K
    w = wl.small_doubles(O_, V_, to, tv)
    _, gt, ot, ge, oe = run_both(gpu_lib, w)
    for name in ("R", "W"):
        err = rel_err(gpu_to_oracle_layout(gt[name], ot[name]), ot[name].data)
        assert err <= TOL, (name, err)
    assert abs(ge["energy"] - oe["energy"]) <= 1e-12 * abs(oe["energy"])


def _single_ladder(tg, O_, V_, to, tv, fill, slices=0, beta=0.0):
    """Ladder R = 0.5 V T on custom host data; returns (gpu, oracle) in oracle layout."""
    ctx = tg.Context(0)
    gs = {"o": ctx.space([(O_ // 2, 1, 0), (O_ // 2, -1, 0)], to), "v": ctx.space([(V_ // 2, 1, 0), (V_ // 2, -1, 0)], tv)}
    os_ = {"o": O.Space([(O_ // 2, 1, 0), (O_ // 2, -1, 0)], to), "v": O.Space([(V_ // 2, 1, 0), (V_ // 2, -1, 0)], tv)}
    shapes = {"V": "vvvv", "T": "vvoo", "R": "vvoo"}
    G = {k: ctx.tensor([gs[c] for c in m], 2) for k, m in shapes.items()}
    Ot = {k: O.Tensor([os_[c] for c in m], 2) for k, m in shapes.items()}
    for k in ("V", "T", "R"):
        Ot[k].data[:] = fill(k, Ot[k].n_elems)
        # same values on the GPU side, matched by tile tuple
        idx = {tuple(t): b for b, t in enumerate(Ot[k].block_tiles.tolist())}
        host = np.empty(G[k].n_elems)
        ends = list(Ot[k].block_off[1:]) + [Ot[k].n_elems]
        for gb, t in enumerate(G[k].block_tiles.tolist()):
            ob = idx[tuple(t)]
            n = ends[ob] - Ot[k].block_off[ob]
            host[G[k].block_offsets[gb]:G[k].block_offsets[gb] + n] = Ot[k].data[Ot[k].block_off[ob]:Ot[k].block_off[ob] + n]
        G[k].upload(host)
    ctx.contract(0.5, G["R"], "abij", beta, G["V"], "abef", G["T"], "efij", "ozaki_bf16", slices)
    O.contract(0.5, Ot["R"], "abij", beta, Ot["V"], "abef", Ot["T"], "efij")
    return gpu_to_oracle_layout(G["R"], Ot["R"]), Ot["R"].data


def test_exact_for_short_inputs(gpu_lib):
    # integers in [-16, 16] times powers of two: every slice sum and the FP64 oracle are exact
    rng = np.random.default_rng(7)
    scale = {"V": 2.0 ** -3, "T": 2.0 ** -9, "R": 1.0}
    fill = lambda k, n: (rng.integers(-16, 17, n) * scale[k]).astype(np.float64) if k != "R" else np.zeros(n)
    got, ref = _single_ladder(gpu_lib, 8, 48, 4, 12, fill)
    assert np.array_equal(got, ref)


def test_all_positive_inputs(gpu_lib):
    # no cancellation: worst case for accumulation length, still within the bound
    rng = np.random.default_rng(8)
    fill = lambda k, n: rng.random(n) if k != "R" else rng.random(n)
    got, ref = _single_ladder(gpu_lib, 12, 80, 6, 40, fill, beta=1.0)
    assert rel_err(got, ref) <= TOL
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-9


def test_wide_dynamic_range(gpu_lib):
    # rows whose magnitudes differ by 2^+-200 and exact zeros
    rng = np.random.default_rng(9)

    def fill(k, n):
        x = rng.standard_normal(n)
        if k == "V":
            x *= 2.0 ** rng.integers(-200, 200, n)
            x[rng.random(n) < 0.1] = 0.0
        return x if k != "R" else np.zeros(n)

    got, ref = _single_ladder(gpu_lib, 8, 32, 4, 8, fill)
    assert rel_err(got, ref) <= TOL


def test_zero_operand_gives_beta_c(gpu_lib):
    rng = np.random.default_rng(10)
    fill = lambda k, n: np.zeros(n) if k == "V" else rng.standard_normal(n)
    got, ref = _single_ladder(gpu_lib, 8, 24, 2, 6, fill, beta=1.0)
    assert np.array_equal(got, ref)


def test_error_decreases_with_slices(gpu_lib):
    rng = np.random.default_rng(11)
    errs = []
    for S in (3, 4, 5, 6, 7, 8):
        rng = np.random.default_rng(11)
        fill = lambda k, n: rng.standard_normal(n) if k != "R" else np.zeros(n)
        got, ref = _single_ladder(gpu_lib, 8, 32, 4, 8, fill, slices=S)
        errs.append(rel_err(got, ref))
    print("rel err by slice count 3..8:", errs)
    # truncation error falls by about 2^-7 per slice until the FP32-rounded tail
    # region (products with k + l >= 5) sets a floor near 1e-11
    assert all(errs[i + 1] < errs[i] / 30 for i in range(3)), errs
    assert errs[3] <= TOL and max(errs[3:]) <= 1e-11, errs


def test_doubles_o40_v240_sampled_ladder_ozaki(gpu_lib):
    tg = gpu_lib
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_doubles_o40_v240()
    ctx = tg.Context(0)
    _, gt = gw.build(ctx, w, only={"V_vvvv", "T", "R"})
    ctx.contract(0.5, gt["R"], "abij", 0.0, gt["V_vvvv"], "abef", gt["T"], "efij", "ozaki_bf16", 0)
    got = gt["R"].download()
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces, {k: w.tensors[k] for k in ("V_vvvv", "T", "R")}))
    R = ot["R"]
    rng = np.random.default_rng(1)
    idx = {tuple(x): k for k, x in enumerate(gt["R"].block_tiles.tolist())}
    _, ext_all = R.block_lo_ext()
    num = den = 0.0
    for b in rng.choice(R.n_blocks, 8, replace=False):
        ext = ext_all[b]
        lo = [int(rng.integers(0, e - 3)) for e in ext]
        ref = O.contract_box(0.5, R, "abij", 0.0, ot["V_vvvv"], "abef", ot["T"], "efij", int(b), lo, [4] * 4)
        k = idx[tuple(R.block_tiles[b].tolist())]
        blk = got[gt["R"].block_offsets[k]:gt["R"].block_offsets[k] + int(np.prod(ext))].reshape(tuple(ext))
        sub = blk[lo[0]:lo[0] + 4, lo[1]:lo[1] + 4, lo[2]:lo[2] + 4, lo[3]:lo[3] + 4]
        num += float(np.sum((sub - ref) ** 2))
        den += float(np.sum(ref ** 2))
    assert np.sqrt(num / den) <= TOL


def test_bad_slice_count(gpu_lib):
    tg = gpu_lib
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    _, t = gw.build(ctx, wl.ladder_o8_v32())
    with pytest.raises(tg.TammError) as e:
        ctx.contract(0.5, t["R"], "abij", 0.0, t["V_vvvv"], "abef", t["T"], "efij", "ozaki_bf16", 12)
    assert e.value.status == tg.TAMM_EINVAL


def test_three_slices_after_six_slices(gpu_lib):
    """TMEM keeps an earlier kernel's accumulators: a 3-slice product (no tail region) run after a
    6-slice one must not pick them up, in either split form."""
    rng = np.random.default_rng(12)
    fill = lambda k, n: rng.standard_normal(n) if k != "R" else np.zeros(n)
    tg = gpu_lib
    ctx = tg.Context(0)
    o = ctx.space([(4, 1, 0), (4, -1, 0)], 4)
    v = ctx.space([(12, 1, 0), (12, -1, 0)], 4)
    T = ctx.tensor([v, v, o, o], 2)
    V = ctx.tensor([v] * 4, 2)
    T.upload(rng.standard_normal(T.n_elems))
    ctx.contract(0.5, V, "abef", 0.0, T, "abij", T, "efij", "f64", 0)
    ref = V.download()
    ctx.contract(0.5, V, "abef", 0.0, T, "abij", T, "efij", "ozaki_bf16", 6)
    for prec, S, tol in (("bf16x3", 0, 1e-6), ("ozaki_bf16", 3, 1e-5)):
        ctx.contract(0.5, V, "abef", 0.0, T, "abij", T, "efij", prec, S)
        assert rel_err(V.download(), ref) <= tol, prec


@pytest.mark.parametrize("O_,V_,to,tv", [(8, 24, 2, 4), (16, 40, 8, 10), (40, 80, 20, 40)])
def test_tile_policies_agree(gpu_lib, O_, V_, to, tv):
    """Output columns per work item (four tile policies), the GEMM grid (one CTA per work item, or
    one per SM walking the items) and column panels on or off: every combination gives bitwise
    the same values."""
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(O_, V_, to, tv)
    outs = []
    ctx = gpu_lib.Context(0)
    gsp, gt = gw.build(ctx, w)
    runner = gw.Runner(ctx, w, gsp, gt)
    for policy in (0, 1, 2, 3):
        for persistent in (0, 1):
            for panels in (0, 1):
                ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_TILE_POLICY, policy)
                ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_PERSISTENT, persistent)
                ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_PANELS, panels)
                gt["R"].data.fill_(float("nan"))
                gt["W"].data.fill_(float("nan"))
                runner.run("ozaki_bf16", 0)
                ctx.sync()
                outs.append({k: gt[k].download() for k in ("R", "W")})
    for k in ("R", "W"):
        for p in range(1, len(outs)):
            assert np.array_equal(outs[p][k], outs[0][k]), (k, p, rel_err(outs[p][k], outs[0][k]))


def test_split_summed_ranges(gpu_lib):
    """Few output tiles and long summed extents (O=16, V=64, tiles 8/16): the contractions are split
    into summed ranges (the reduction kernel runs), match the unsplit sums to rounding and the oracle
    to 1e-10."""
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(16, 64, 8, 16)
    outs, reductions = [], []
    for split in (0, 1):
        ctx = gpu_lib.Context(0)
        ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_SPLIT_K, split)
        gsp, gt = gw.build(ctx, w)
        ctx.profile(True)
        gw.Runner(ctx, w, gsp, gt).run("ozaki_bf16", 0)
        ctx.sync()
        reductions.append(ctx.profile_read()["split_reduce"][1])
        outs.append({k: gt[k] for k in ("R", "W")})
    assert reductions[0] == 0 and reductions[1] > 0, reductions
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    for k in ("R", "W"):
        a = gpu_to_oracle_layout(outs[0][k], ot[k])
        b = gpu_to_oracle_layout(outs[1][k], ot[k])
        assert rel_err(b, a) <= 1e-12, (k, rel_err(b, a))
        assert rel_err(b, ot[k].data) <= 1e-10, k


def test_dense4d_matches_oracle(gpu_lib):
    """The paper's dense 4-D contraction C(abcd) = A(abmn) B(mncd) (every block stored), N = 24 in tiles
    of 8 (and a ragged 20 in tiles of 8): FP64 <= 1e-12 and split precision <= 1e-10 vs the oracle."""
    for N, tile in ((24, 8), (20, 8)):
        w = wl.dense4d(N, tile)
        for prec, tol in (("f64", 1e-12), ("ozaki_bf16", 1e-10)):
            _, gt, ot, _, _ = run_both(gpu_lib, w, prec)
            err = rel_err(gpu_to_oracle_layout(gt["C"], ot["C"]), ot["C"].data)
            assert err <= tol, (N, prec, err)
