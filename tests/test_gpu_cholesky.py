"""Cholesky lambda tensor on the GPU (Eq. cc12; Sec. III.A lambda tensors).

* Forming V from the Cholesky vectors (tamm_cholesky_form) matches the oracle's V: FP64 within 1e-12,
  split precision within 1e-10, BF16x3 within 1e-5 (normwise), whatever the slab size.
* The ladder R = 1/2 V T reading the lambda tensor matches the oracle (FP64 1e-12, split 1e-10) for
  one-tile slabs and for the default single slab; beta = 1 accumulates over slabs correctly.
* Reading the lambda tensor equals reading V formed once into storage.
* A captured CUDA graph of the lambda ladder replays bit for bit.
* Every operation that would need V's storage is refused with TAMM_EUNSUPPORTED.
* At O=40 V=240 with 560 vectors (V_vvvv would be 9.95 GB), sampled 4^4 boxes of R against the oracle
  (which forms only the V blocks those boxes read).
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    w = wl.cholesky_ladder_o8_v32()
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    return w, ot


def build_gpu(tg, w, slab_bytes=0):
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w, slab_bytes=slab_bytes)
    return ctx, gsp, gt


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("ozaki_bf16", 1e-10), ("bf16x3", 1e-5)])
@pytest.mark.parametrize("slab", [1, 0])
def test_form_matches_oracle(gpu_lib, small, prec, tol, slab):
    w, ot = small
    ctx, _, gt = build_gpu(gpu_lib, w, slab)
    V = gt["V_chol"]
    assert V.n_slabs == (4 if slab == 1 else 1)
    out = ctx.tensor(V.modes, 2, "spin")
    out.data.fill_(3.0)
    ctx.cholesky_form(V, out, prec)
    ctx.sync()
    err = rel_err(gpu_to_oracle_layout(out, ot["V_chol"]), ot["V_chol"].data)
    print(f"form {prec} slab={slab}: {err:.3e}")
    assert err <= tol


def test_form_independent_of_slab_size(gpu_lib, small):
    w, _ = small
    got = {}
    for slab in (1, 0):
        ctx, _, gt = build_gpu(gpu_lib, w, slab)
        out = ctx.tensor(gt["V_chol"].modes, 2, "spin")
        ctx.cholesky_form(gt["V_chol"], out, "f64")
        ctx.sync()
        got[slab] = out.download()
    assert np.array_equal(got[1], got[0])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("ozaki_bf16", 1e-10)])
@pytest.mark.parametrize("slab", [1, 0])
def test_ladder_matches_oracle(gpu_lib, small, prec, tol, slab):
    from paper_2201_01257_gb300 import workload as gw

    w, ot = small
    ctx, gsp, gt = build_gpu(gpu_lib, w, slab)
    gt["R"].data.fill_(5.0)  # beta = 0 on the first slab overwrites
    run = gw.Runner(ctx, w, gsp, gt)
    run.run(prec, 0)
    ctx.sync()
    err = rel_err(gpu_to_oracle_layout(gt["R"], ot["R"]), ot["R"].data)
    print(f"ladder {prec} slab={slab}: {err:.3e}")
    assert err <= tol
    # the step's flops count forming V once plus the ladder itself
    assert run.flops(w.steps[0]) == gt["V_chol"].form_flops + ctx.flops(gt["R"], "abij", gt["V_chol"], "abef",
                                                                         gt["T"], "efij")


def test_beta_one_accumulates_over_slabs(gpu_lib, small):
    import torch

    w, ot = small
    ctx, _, gt = build_gpu(gpu_lib, w, 1)
    R = gt["R"]
    r0 = torch.randn(R.n_elems, dtype=torch.float64, generator=torch.Generator().manual_seed(4))
    R.data[: R.n_elems].copy_(r0)
    ctx.contract(0.5, R, "abij", 1.0, gt["V_chol"], "abef", gt["T"], "efij", "f64", 0)
    ctx.sync()
    want = gpu_to_oracle_layout_host(r0.numpy(), R, ot["R"]) + ot["R"].data
    assert rel_err(gpu_to_oracle_layout(R, ot["R"]), want) <= 1e-13


def gpu_to_oracle_layout_host(g, G, Rt):
    out = np.empty(Rt.n_elems)
    idx = {tuple(t): k for k, t in enumerate(G.block_tiles.tolist())}
    for b in range(Rt.n_blocks):
        k = idx[tuple(Rt.block_tiles[b].tolist())]
        n = (Rt.block_off[b + 1] if b + 1 < Rt.n_blocks else Rt.n_elems) - Rt.block_off[b]
        out[Rt.block_off[b]:Rt.block_off[b] + n] = g[G.block_offsets[k]:G.block_offsets[k] + n]
    return out


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("ozaki_bf16", 1e-12)])
def test_lambda_equals_stored_formed_v(gpu_lib, small, prec, tol):
    w, _ = small
    ctx, _, gt = build_gpu(gpu_lib, w, 1)
    V, T, R = gt["V_chol"], gt["T"], gt["R"]
    Vs = ctx.tensor(V.modes, 2, "spin")
    ctx.cholesky_form(V, Vs, prec)
    ctx.contract(0.5, R, "abij", 0.0, Vs, "abef", T, "efij", prec, 0)
    ctx.sync()
    stored = R.download()
    ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", prec, 0)
    ctx.sync()
    assert rel_err(R.download(), stored) <= tol


def test_graph_replays_lambda_ladder(gpu_lib, small):
    import torch

    from paper_2201_01257_gb300 import workload as gw

    w, _ = small
    stream = torch.cuda.Stream(0)  # capture needs a created stream
    ctx = gpu_lib.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        _, gt = gw.build(ctx, w, slab_bytes=1)
        V, T, R = gt["V_chol"], gt["T"], gt["R"]
        go = lambda: ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", "ozaki_bf16", 0)
        go()  # builds every plan
        ctx.sync()
        eager = R.download()
        R.data.zero_()
        with ctx.capture() as cap:
            go()
        assert cap.graph.kernel_launches > 0
        cap.graph.launch()
        ctx.sync()
        assert np.array_equal(R.download(), eager)


def test_lambda_refusals_on_device(gpu_lib, small):
    tg = gpu_lib
    w, _ = small
    ctx, _, gt = build_gpu(tg, w)
    V, T, R = gt["V_chol"], gt["T"], gt["R"]
    Vs = ctx.tensor(V.modes, 2, "spin")

    def refused(fn):
        with pytest.raises(tg.TammError) as e:
            fn()
        assert e.value.status == tg.TAMM_EUNSUPPORTED, str(e.value)

    refused(lambda: ctx.add(Vs, "abef", 0.0, V, [(1.0, "abef")]))
    refused(lambda: ctx.energy(1.0, V, "abef", Vs, "abef"))
    refused(lambda: ctx.norm(V))
    refused(lambda: ctx.contract(1.0, V, "abef", 0.0, Vs, "abcd", Vs, "cdef", "f64", 0))
    refused(lambda: ctx.contract(1.0, Vs, "abef", 0.0, V, "abcd", V, "cdef", "f64", 0))
    refused(lambda: ctx.autotune(R, "abij", V, "abef", T, "efij", 1e-10))

    def grouped():
        with ctx.group():
            ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", "ozaki_bf16", 0)

    refused(grouped)
    # the context stays usable
    ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", "f64", 0)
    ctx.sync()


@pytest.mark.parametrize("r_tile", [72, 80])  # 42 KB planes: pair kernel; 52 KB planes: two-term permuted add
def test_cholesky_oovv_shaped(gpu_lib, r_tile):
    """V[m,n,e,f] from X[m,e,L] over (occ, virt, aux) — P and R spaces differ — formed and read by the
    intermediate W(mnij) = V(mnef) T(efij), in FP64 and split precision."""
    from paper_2201_01257_gb300 import workload as gw

    w = wl.Workload(f"cholesky_oovv_R{r_tile}", wl.SEED_BASE + 11,
                    {"occ": wl.spin_space("occ", 8, 4), "virt": wl.spin_space("virt", 2 * r_tile, r_tile),
                     "aux": wl.aux_space("aux", 24, 12)}, {})
    w.tensors = {
        "X": wl.TensorSpec("X", ("occ", "virt", "aux"), 1, sigma=0.05, stream=8),
        "V": wl.TensorSpec("V", ("occ", "occ", "virt", "virt"), 2, cholesky="X"),
        "T": wl.TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True,
                           anti23=True),
        "W": wl.TensorSpec("W", ("occ",) * 4, 2),
    }
    w.steps = [wl.ContractSpec("intermediate", "W", "mnij", "V", "mnef", "T", "efij", 1.0, beta=0.0)]
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    ctx, gsp, gt = build_gpu(gpu_lib, w, 1)
    assert gt["V"].n_slabs == 2
    for prec, tol in (("f64", 1e-12), ("ozaki_bf16", 1e-10)):
        out = ctx.tensor(gt["V"].modes, 2, "spin")
        ctx.cholesky_form(gt["V"], out, prec)
        gw.Runner(ctx, w, gsp, gt).run(prec, 0)
        ctx.sync()
        ev = rel_err(gpu_to_oracle_layout(out, ot["V"]), ot["V"].data)
        ew = rel_err(gpu_to_oracle_layout(gt["W"], ot["W"]), ot["W"].data)
        print(f"oovv-shaped R tile {r_tile} {prec}: V {ev:.3e} W {ew:.3e}")
        assert ev <= tol and ew <= tol


# ------------------------------------------------------------ full size, sampled

@pytest.mark.slow
def test_cholesky_ladder_o40_v240_sampled():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.cholesky_ladder_o40_v240()
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w)
    V = gt["V_chol"]
    assert V.n_elems == 3 * 240 ** 4 // 8  # 9.95 GB that are never stored
    stored = {k: w.tensors[k] for k in ("X", "T", "R")}
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces, stored))
    Vo = O.Tensor(ot["X"].modes[:1] * 2 + ot["X"].modes[1:2] * 2, 2)  # only the blocks the boxes read get formed

    # sampled 4^4 boxes of R inside four (a, b) tile pairs; the oracle forms only the V blocks they read
    rng = np.random.default_rng(17)
    R = ot["R"]
    _, ext = R.block_lo_ext()
    pairs = {}
    for b in range(R.n_blocks):
        pairs.setdefault(tuple(R.block_tiles[b, :2]), []).append(b)
    keys = sorted(pairs)
    chosen = [keys[int(i)] for i in rng.choice(len(keys), size=4, replace=False)]
    blocks, lo = [], []
    for k in chosen:
        for b in rng.choice(pairs[k], size=min(4, len(pairs[k])), replace=False):
            for _ in range(2):
                blocks.append(int(b))
                lo.append([int(rng.integers(0, e - 3)) for e in ext[b]])
    need = [b for b in range(Vo.n_blocks) if tuple(Vo.block_tiles[b, :2]) in set(chosen)]
    O.cholesky_v(Vo, ot["X"], need)
    refs = O.contract_boxes(0.5, R, "abij", Vo, "abef", ot["T"], "efij", blocks, lo, [[4] * 4] * len(blocks))

    def sampled_err(G):
        g = gpu_to_oracle_layout(G, R)
        num = den = 0.0
        for b, l, v in zip(blocks, lo, refs):
            blk = g[R.block_off[b]:R.block_off[b] + int(np.prod(ext[b]))].reshape(tuple(ext[b]))
            sub = blk[l[0]:l[0] + 4, l[1]:l[1] + 4, l[2]:l[2] + 4, l[3]:l[3] + 4]
            num += float(np.sum((sub - v) ** 2))
            den += float(np.sum(v ** 2))
        return float(np.sqrt(num / den))

    run = gw.Runner(ctx, w, gsp, gt)
    for prec, tol in (("ozaki_bf16", 1e-10), ("f64", 1e-12)):
        run.run(prec, 0)
        ctx.sync()
        err = sampled_err(gt["R"])
        print(f"O=40 V=240 L=560 cholesky ladder {prec}: sampled rel err {err:.3e}")
        assert err <= tol
