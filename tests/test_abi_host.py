"""C-ABI library: loads, exports every declared symbol, and its host-side
planning (tiling, block tables, nonzero block pairs) agrees with the oracle's
independent implementation and with closed forms.  No device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2201_01257_gb300 as tg
from tamm_synth import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"TAMM_API\s+[\w\s\*]+?\b(tamm_\w+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    lib = tg.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert {n for n, _, _ in tg.PROTOTYPES} == names


@pytest.fixture(scope="module")
def hctx():
    return tg.Context(-1)


def spaces_for(ctx, w):
    return ({k: ctx.space(s.groups, s.tile, s.tile_sizes) for k, s in w.spaces.items()},
            {k: O.Space.from_spec(s) for k, s in w.spaces.items()})


@pytest.mark.parametrize("name", sorted(wl.WORKLOADS) + ["irrep_doubles", "irrep_doubles_small", "dense4d"])
def test_block_tables_match_oracle(hctx, name):
    if name == "irrep_doubles":
        w = wl.irrep_doubles()
    elif name == "irrep_doubles_small":
        w = wl.irrep_doubles(O=32, V=96)
    elif name == "dense4d":
        w = wl.dense4d(40, 16)
    else:
        w = wl.WORKLOADS[name]()
    gs, os_ = spaces_for(hctx, w)
    for k in gs:
        assert gs[k].n == os_[k].n
        assert list(gs[k].tile_size) == [t[1] for t in os_[k].tiles]
        assert list(gs[k].tile_spin) == [t[2] for t in os_[k].tiles]
    for name, t in w.tensors.items():
        G = hctx.tensor([gs[m] for m in t.modes], t.n_upper, t.sym)
        R = O.Tensor([os_[m] for m in t.modes], t.n_upper, t.sym, alloc=False)
        assert (G.n_blocks, G.n_elems) == (R.n_blocks, R.n_elems), name
        assert np.array_equal(G.block_tiles, R.block_tiles), name
        assert np.array_equal(G.block_offsets, R.block_off), name


def test_irrep_rule_and_explicit_tiles_match_oracle(hctx):
    groups = [(5, 1, 0), (3, 1, 3), (4, 1, 5), (5, -1, 0), (3, -1, 3), (4, -1, 5)]
    tiles = (2, 3, 3, 4, 3, 2, 3, 4)
    g = hctx.space(groups, tile_sizes=tiles)
    o = O.Space(groups, tile_sizes=tiles)
    for sym in ("dense", "spin", "spin_irrep"):
        G = hctx.tensor([g] * 4, 2, sym)
        R = O.Tensor([o] * 4, 2, sym, alloc=False)
        assert np.array_equal(G.block_tiles, R.block_tiles) and np.array_equal(G.block_offsets, R.block_off)


def test_fig_tensor_const_eight_blocks(hctx):
    tM = hctx.space([(30, 1, 0)], tile_sizes=(10, 20))
    tK = hctx.space([(20, 1, 0)], tile=5)
    A = hctx.tensor([tM, tK], 1, "dense")
    assert (A.n_blocks, A.n_elems) == (8, 600)


def test_flop_counts_closed_forms(hctx):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    v = hctx.space([(8, 1, 0), (8, -1, 0)], tile=4)
    V = hctx.tensor([v] * 4, 2)
    T = hctx.tensor([v, v, o, o], 2)
    R = hctx.tensor([v, v, o, o], 2)
    assert hctx.flops(R, "abij", V, "abef", T, "efij") * 32 == 5 * 2 * 16 ** 4 * 8 ** 2
    t1 = hctx.tensor([v, o], 1)
    V3 = hctx.tensor([v, v, v, o], 2)
    assert hctx.flops(R, "abij", V3, "abej", t1, "ei") * 16 == 3 * 2 * 16 ** 3 * 8 ** 2
    # operand order does not change the count
    assert hctx.flops(R, "abij", T, "efij", V, "abef") == hctx.flops(R, "abij", V, "abef", T, "efij")


def test_doubles_o40_v240_flops(hctx):
    w = wl.ccsd_doubles_o40_v240()
    gs, _ = spaces_for(hctx, w)
    T = {n: hctx.tensor([gs[m] for m in t.modes], t.n_upper, t.sym) for n, t in w.tensors.items()}
    f = {s.name: hctx.flops(T[s.c], s.lc, T[s.a], s.la, T[s.b], s.lb) for s in w.steps
         if isinstance(s, wl.ContractSpec)}
    assert f["ladder"] == 5 / 32 * 2 * 240 ** 4 * 40 ** 2
    assert f["intermediate"] == 5 / 32 * 2 * 240 ** 2 * 40 ** 4
    assert f["oooo"] == 5 / 32 * 2 * 240 ** 2 * 40 ** 4
    assert abs(f["ring"] - 2.765e11) / 2.765e11 < 1e-3
    assert abs(f["t1"] - 8.294e9) / 8.294e9 < 1e-3


@pytest.mark.parametrize("lc,la,lb", [
    ("abij", "abef", "efkj"), ("abij", "abij", "efij"), ("abii", "abef", "efij"), ("abij", "abe", "efij")])
def test_invalid_labels_rejected(hctx, lc, la, lb):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    v = hctx.space([(8, 1, 0), (8, -1, 0)], tile=4)
    V, T, R = hctx.tensor([v] * 4, 2), hctx.tensor([v, v, o, o], 2), hctx.tensor([v, v, o, o], 2)
    with pytest.raises(tg.TammError) as e:
        hctx.flops(R, lc, V, la, T, lb)
    assert e.value.status == tg.TAMM_EINVAL


def test_space_errors(hctx):
    with pytest.raises(tg.TammError):
        hctx.space([(10, 1, 0), (10, -1, 0)], tile_sizes=(5, 10, 5))
    with pytest.raises(tg.TammError):
        hctx.space([(10, 2, 0)], tile=4)
    with pytest.raises(tg.TammError):
        hctx.space([(10, 1, 9)], tile=4)


def test_host_only_context_refuses_device_work(hctx):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    T = hctx.tensor([o, o], 1)
    r = ctypes.c_double()
    assert hctx.lib.tamm_norm(hctx.handle, T.handle, ctypes.byref(r)) == tg.TAMM_ECUDA
    assert b"host-only" in hctx.lib.tamm_last_error(hctx.handle)
    assert hctx.lib.tamm_tensor_allocate(T.handle) == tg.TAMM_ECUDA


def test_permuted_tensor_stores_images_of_blocks(hctx):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    v = hctx.space([(6, 1, 0), (6, -1, 0)], tile=3)
    R = hctx.tensor([v, v, o, o], 2)
    X = hctx.tensor_permuted(R, [0, 2, 1, 3])  # (a, i, b, j)
    assert X.n_elems == R.n_elems and X.n_blocks == R.n_blocks
    imgs = {tuple(t[[0, 2, 1, 3]]) for t in R.block_tiles}
    assert {tuple(t) for t in X.block_tiles} == imgs
    with pytest.raises(tg.TammError):
        hctx.tensor_permuted(R, [0, 0, 1, 3])


def test_group_and_graph_calls_need_a_device(hctx):
    assert hctx.lib.tamm_group_begin(hctx.handle) == tg.TAMM_ECUDA
    assert hctx.lib.tamm_graph_begin(hctx.handle) == tg.TAMM_ECUDA
    assert hctx.lib.tamm_group_cancel(hctx.handle) == tg.TAMM_EINVAL  # no group is open
    import ctypes as ct

    g = ct.c_void_p()
    assert hctx.lib.tamm_graph_end(hctx.handle, ct.byref(g)) == tg.TAMM_ECUDA and not g.value
    assert hctx.lib.tamm_graph_launch(None) == tg.TAMM_EINVAL
    hctx.lib.tamm_graph_destroy(None)


# ------------------------------------------------ Cholesky lambda tensor (Eq. cc12)

@pytest.mark.parametrize("recipe", [wl.cholesky_ladder_o8_v32, wl.cholesky_ladder_o40_v240])
def test_cholesky_lambda_block_table_matches_oracle(hctx, recipe):
    w = recipe()
    gs, os_ = spaces_for(hctx, w)
    assert list(gs["aux"].tile_spin) == [0] * gs["aux"].n_tiles  # spinless auxiliary index
    xs, vs = w.tensors["X"], w.tensors["V_chol"]
    X = hctx.tensor([gs[m] for m in xs.modes], xs.n_upper, xs.sym)
    RX = O.Tensor([os_[m] for m in xs.modes], xs.n_upper, xs.sym, alloc=False)
    assert (X.n_blocks, X.n_elems) == (RX.n_blocks, RX.n_elems)
    V = hctx.tensor_cholesky(X)
    R = O.Tensor([os_[m] for m in vs.modes], vs.n_upper, vs.sym, alloc=False)
    # the blocks some aux tile links are exactly the spin-rule blocks of a 2|2 tensor
    assert (V.n_blocks, V.n_elems) == (R.n_blocks, R.n_elems)
    assert np.array_equal(V.block_tiles, R.block_tiles)
    assert np.array_equal(V.block_offsets, R.block_off)
    # forming V once costs 2 * (sum of |p||r| over same-spin tile pairs)^2 * n_aux
    half = gs["virt"].n // 2
    assert V.form_flops == 2.0 * (2 * half * half) ** 2 * gs["aux"].n
    # the ladder's own flops are those of the stored-V ladder
    T = hctx.tensor([gs["virt"], gs["virt"], gs["occ"], gs["occ"]], 2)
    Vs = hctx.tensor([gs["virt"]] * 4, 2)
    assert hctx.flops(T, "abij", V, "abef", T, "efij") == hctx.flops(T, "abij", Vs, "abef", T, "efij")


def test_cholesky_lambda_slab_partition(hctx):
    w = wl.cholesky_ladder_o8_v32()
    gs, _ = spaces_for(hctx, w)
    xs = w.tensors["X"]
    X = hctx.tensor([gs[m] for m in xs.modes], xs.n_upper, xs.sym)
    n_tiles = gs["virt"].n_tiles
    one = hctx.tensor_cholesky(X, 1)  # every tile alone
    whole = hctx.tensor_cholesky(X, 1 << 40)
    assert one.n_slabs == n_tiles and whole.n_slabs == 1
    assert one.form_flops == whole.form_flops
    assert whole.buffer_bytes == 8 * (whole.n_elems + whole.n_elems * 2 // 3)  # V (3/8 dense) + X1 (1/4 dense)
    mid = hctx.tensor_cholesky(X, whole.buffer_bytes // 2)
    assert 2 <= mid.n_slabs < n_tiles and mid.buffer_bytes <= whole.buffer_bytes // 2
    for V in (one, mid, whole):
        assert np.array_equal(V.block_tiles, whole.block_tiles)


def test_cholesky_lambda_refusals(hctx):
    v = hctx.space([(8, 1, 0), (8, -1, 0)], tile=4)
    a = hctx.space([(6, 0, 0)], tile=3)
    X = hctx.tensor([v, v, a], 1)
    V = hctx.tensor_cholesky(X)
    h = ctypes.c_void_p()
    assert hctx.lib.tamm_tensor_create_cholesky(hctx.handle, V.handle, 0, ctypes.byref(h)) == tg.TAMM_EINVAL
    Y = hctx.tensor([v, v, a, a], 2)
    assert hctx.lib.tamm_tensor_create_cholesky(hctx.handle, Y.handle, 0, ctypes.byref(h)) == tg.TAMM_EINVAL
    assert hctx.lib.tamm_tensor_create_cholesky(hctx.handle, X.handle, -1, ctypes.byref(h)) == tg.TAMM_EINVAL
    assert not h.value
    assert hctx.lib.tamm_tensor_allocate(V.handle) == tg.TAMM_EUNSUPPORTED
    assert hctx.lib.tamm_cholesky_info(X.handle, None, None, None) == tg.TAMM_EINVAL
    with pytest.raises(tg.TammError):
        V.bind(None)
    with pytest.raises(tg.TammError):
        hctx.space([(6, 2, 0)], tile=3)


# ------------------------------------------------------------- scheduler levels

def test_scheduler_levels_of_the_doubles_step(hctx):
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_doubles_o40_v240()
    gs, _ = spaces_for(hctx, w)
    T = {name: hctx.tensor([gs[m] for m in t.modes], t.n_upper, t.sym) for name, t in w.tensors.items()}
    sch = gw.Runner(hctx, w, gs, T).scheduled("ozaki_bf16", 0, energy_out=0x1000)
    # recorded: ladder (R =), W = W0, W += V_oovv T, R += 1/4 T W, X = T V_ovvo, R += P(ab)P(ij) X,
    # R += V_vvvo t1, E = 1/4 V_oovv T
    assert sch.levels() == [0, 0, 1, 2, 0, 3, 4, 0]
    # no device: execution fails at its first operation and reports it
    with pytest.raises(tg.TammError) as e:
        sch.execute()
    assert e.value.status == tg.TAMM_ECUDA


def test_scheduler_conflict_kinds(hctx):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    a = hctx.space([(6, 0, 0)], tile=3)
    A, B, C, D = (hctx.tensor([o, o], 1) for _ in range(4))
    sch = hctx.scheduler()
    sch.contract(1.0, C, "ij", 0.0, A, "ik", B, "kj")   # 0: reads A B, writes C
    sch.contract(1.0, D, "ij", 0.0, A, "ik", B, "kj")   # 0: independent (reads only shared)
    sch.add(A, "ij", 0.0, D, [(1.0, "ji")])             # 1: writes A that op 0 reads (WAR), reads D (RAW)
    sch.add(C, "ij", 1.0, B, [(2.0, "ij")])             # 1: beta = 1 reads and writes C (after op 0)
    sch.energy_async(1.0, C, "ij", A, "ij", 0x1000)     # 2: reads C and A written at level 1
    sch.energy_async(1.0, B, "ij", B, "ij", 0x1000)     # 3: same result slot as op 4 (WAW)
    assert sch.levels() == [0, 0, 1, 1, 2, 3]
    # a contraction reading a Cholesky lambda tensor reads its vectors
    X = hctx.tensor([o, o, a], 1)
    V = hctx.tensor_cholesky(X)
    R = hctx.tensor([o, o, o, o], 2)
    sch3 = hctx.scheduler()
    R2 = hctx.tensor([o, o, o, o], 2)
    sch3.contract(1.0, R2, "pqrs", 0.0, V, "pqtu", R, "turs")
    sch3.add(X, "pqL", 0.0, X, [(1.0, "pqL")])  # writes X, which op 0 reads through V
    sch3.contract(1.0, R, "pqrs", 0.0, V, "pqtu", R2, "turs")
    assert sch3.levels() == [0, 1, 2]


def test_scheduler_argument_errors(hctx):
    o = hctx.space([(4, 1, 0), (4, -1, 0)], tile=2)
    A = hctx.tensor([o, o], 1)
    sch = hctx.scheduler()
    with pytest.raises(tg.TammError):
        sch.contract(1.0, A, "ijk", 0.0, A, "ik", A, "kj")
    with pytest.raises(tg.TammError):
        sch.add(A, "ij", 0.0, A, [])
    with pytest.raises(tg.TammError):
        sch.energy_async(1.0, A, "ij", A, "ij", 0)
    assert sch.levels() == []
    sch.execute()  # nothing recorded: nothing to do


def test_cholesky_lambda_irrep_block_table(hctx):
    # X with the spin + irrep rule over an aux index carrying all eight D2h irreps: the blocks some aux
    # tile links are exactly the spin + irrep blocks of a 2|2 tensor (the oracle's rule)
    import numpy as np_

    rng = np_.random.default_rng(3)
    vs = wl.irrep_space("virt", 64, rng, 4, 12)
    aux = wl.SpaceSpec("aux", tuple((10, 0, g) for g in range(8)), tile=5)
    w = wl.Workload("irrep_cholesky", 1, {"virt": vs, "aux": aux}, {})
    gs, os_ = spaces_for(hctx, w)
    X = hctx.tensor([gs["virt"], gs["virt"], gs["aux"]], 1, "spin_irrep")
    V = hctx.tensor_cholesky(X)
    R = O.Tensor([os_["virt"]] * 4, 2, "spin_irrep", alloc=False)
    assert (V.n_blocks, V.n_elems) == (R.n_blocks, R.n_elems)
    assert np.array_equal(V.block_tiles, R.block_tiles)
    # with the aux index in irrep 0 only, X links only same-irrep pairs: fewer blocks than the rule allows
    aux0 = hctx.space([(80, 0, 0)], 5)
    X0 = hctx.tensor([gs["virt"], gs["virt"], aux0], 1, "spin_irrep")
    assert 0 < hctx.tensor_cholesky(X0).n_blocks < R.n_blocks


def test_scheduler_puts_independent_ladders_in_one_level(hctx):
    # the 32 ladder problems of the batch share no tensor: one level, i.e. one contraction group
    sch = hctx.scheduler()
    for k, (o, v) in enumerate(wl.ladder_batch_sizes()[:32]):
        w = wl.ladder_problem(2 * max(o // 8, 2), 2 * max(v // 16, 4), 1 + k, 2, 4)  # small shapes: planning only
        gs, _ = spaces_for(hctx, w)
        T = {n: hctx.tensor([gs[m] for m in t.modes], t.n_upper, t.sym) for n, t in w.tensors.items()}
        st = w.steps[0]
        sch.contract(st.alpha, T[st.c], st.lc, st.beta, T[st.a], st.la, T[st.b], st.lb, "ozaki_bf16")
        # the same problem's energy-style read of its output comes one level later
        sch.energy_async(1.0, T["R"], "abij", T["T"], "abij", 0x1000 + 8 * k)
    assert sch.levels() == [0, 1] * 32


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 with no C++ or torch types
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "tamm_gb300.h"\n'
                   "int main(void) {\n"
                   "  tamm_ctx* ctx = 0; tamm_tensor* t = 0; tamm_sched* s = 0; tamm_graph* g = 0;\n"
                   "  (void)ctx; (void)t; (void)s; (void)g;\n"
                   "  return TAMM_OK;\n"
                   "}\n")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "use.o")])


def test_triples_info_counts(hctx):
    # occupied triples C(n_o, 3); block-GEMM flops = 2 M N K over the block pairs of every triple's U,
    # enumerated here independently from the spin rule of the input tensors
    import itertools

    w = wl.triples(8, 24, 2, 6)
    gs, os_ = spaces_for(hctx, w)
    t = {n: hctx.tensor([gs[m] for m in s.modes], s.n_upper, s.sym, allocate=False) for n, s in w.tensors.items()}
    info = hctx.triples_info(t["T"], t["t1"], t["V_ooov"], t["V_vovv"], t["V_oovv"])
    assert info["n_triples"] == 8 * 7 * 6 // 6 and info["n_batches"] == 1
    occ, vir = os_["occ"].tiles, os_["virt"].tiles
    otile = [k for k, tl in enumerate(occ) for _ in range(tl[1])]
    sp_o = [tl[2] for tl in occ]
    sp_v = [tl[2] for tl in vir]

    def stored(spins_up, spins_lo):
        return sum(spins_up) == sum(spins_lo)

    flops = 0
    for i, j, k in itertools.combinations(range(8), 3):
        s = sp_o[otile[i]] + sp_o[otile[j]] + sp_o[otile[k]]
        for tx, ty, tz in itertools.product(range(len(vir)), repeat=3):
            if sp_v[tx] + sp_v[ty] + sp_v[tz] != s:
                continue
            nxy, nz = vir[tx][1] * vir[ty][1], vir[tz][1]
            for p, q, r in ((i, j, k), (j, k, i), (k, i, j)):
                tp, tq, tr = otile[p], otile[q], otile[r]
                for tm in range(len(occ)):
                    if stored([sp_v[tx], sp_v[ty]], [sp_o[tm], sp_o[tr]]) and \
                            stored([sp_o[tp], sp_o[tq]], [sp_o[tm], sp_v[tz]]):
                        flops += 2 * nxy * nz * occ[tm][1]
                for te in range(len(vir)):
                    if stored([sp_v[te], sp_o[tp]], [sp_v[ty], sp_v[tx]]) and \
                            stored([sp_v[te], sp_v[tz]], [sp_o[tq], sp_o[tr]]):
                        flops += 2 * nxy * nz * vir[te][1]
    assert info["gemm_flops"] == flops
    # a tiny workspace: one triple per batch
    assert hctx.triples_info(t["T"], t["t1"], t["V_ooov"], t["V_vovv"], t["V_oovv"], 8)["n_batches"] == 56
