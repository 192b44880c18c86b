"""Pins for the FP64 oracle against what the paper and mathematics fix.

Each pin is independent of the oracle's own loops: dense ``numpy.einsum`` on
tiny inputs, closed-form block counts, exact identities, invariants.  The
mutation tests at the end compile deliberately broken copies of the oracle
source and check that at least one pin catches each planted mistake.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def spin_space(n, tile):
    return O.Space([(n // 2, 1, 0), (n // 2, -1, 0)], tile)


def filled(modes, n_upper, seed, stream, sigma, a01=True, a23=True, sym="spin"):
    T = O.Tensor(modes, n_upper, sym)
    T.fill_synthetic(seed, wl.TensorSpec("x", (), n_upper, sym, sigma, stream, a01, a23))
    return T


# --------------------------------------------------------------- structure

def test_fig_tensor_const_block_count():
    # Sec. III.A, Fig. "tensor_const": tM = {M, {10, 20}}, tK = {K, 5}; A{tM, tK} is a
    # 30 x 20 matrix with eight blocks.
    tM = O.Space([(30, 1, 0)], tile_sizes=(10, 20))
    tK = O.Space([(20, 1, 0)], tile=5)
    A = O.Tensor([tM, tK], 1, "dense")
    assert A.n_blocks == 8
    assert A.n_elems == 600
    assert [t[1] for t in tM.tiles] == [10, 20]
    assert [t[1] for t in tK.tiles] == [5, 5, 5, 5]


def test_fixed_tiling_remainder_and_group_boundaries():
    s = O.Space([(160, 1, 0), (160, -1, 0)], tile=64)
    assert [t[1] for t in s.tiles] == [64, 64, 32, 64, 64, 32]
    assert [t[2] for t in s.tiles] == [1, 1, 1, -1, -1, -1]
    with pytest.raises(O.OracleError):
        O.Space([(10, 1, 0), (10, -1, 0)], tile_sizes=(5, 10, 5))  # straddles the alpha/beta boundary


@pytest.mark.parametrize("n,tile", [(32, 8), (48, 8), (240, 40)])
def test_spin_storage_fraction_three_eighths(n, tile):
    v = spin_space(n, tile)
    V = O.Tensor([v] * 4, 2, "spin", alloc=False)
    assert V.n_elems * 8 == 3 * n ** 4


def test_vvvv_storage_o80_v320_31gb():
    # O=80 / V=320 spin-orbitals, virtual tile 64: the stored V_vvvv is about 31 GB.
    v = spin_space(320, 64)
    V = O.Tensor([v] * 4, 2, "spin", alloc=False)
    assert V.n_elems == 3 * 320 ** 4 // 8 == 3_932_160_000
    assert abs(V.n_elems * 8 / 1e9 - 31.46) < 0.01


def _pair_flops(C, lc, A, la, B, lb):
    """2*M*N*K summed over every (C block, contracted tile tuple) with A and B blocks stored."""
    spaces = {}
    for T, l in ((C, lc), (A, la), (B, lb)):
        for m, ch in enumerate(l):
            spaces[ch] = T.modes[m]
    free = list(lc)
    summed = [ch for ch in la if ch not in lc]
    total = 0
    import itertools
    for cb in range(C.n_blocks):
        tile = {ch: int(C.block_tiles[cb, m]) for m, ch in enumerate(lc)}
        for kt in itertools.product(*[range(spaces[ch].n_tiles) for ch in summed]):
            tile.update(dict(zip(summed, kt)))
            if A.find_block([tile[ch] for ch in la]) < 0 or B.find_block([tile[ch] for ch in lb]) < 0:
                continue
            size = 1
            for ch in free + summed:
                size *= spaces[ch].tiles[tile[ch]][1]
            total += 2 * size
    return total


def test_ladder_nonzero_flop_fraction_five_32nds():
    o, v = spin_space(8, 2), spin_space(16, 4)
    V = O.Tensor([v] * 4, 2, alloc=False)
    T = O.Tensor([v, v, o, o], 2, alloc=False)
    R = O.Tensor([v, v, o, o], 2, alloc=False)
    assert _pair_flops(R, "abij", V, "abef", T, "efij") * 32 == 5 * 2 * 16 ** 4 * 8 ** 2
    t1 = O.Tensor([v, o], 1, alloc=False)
    Vvvvo = O.Tensor([v, v, v, o], 2, alloc=False)
    assert _pair_flops(R, "abij", Vvvvo, "abej", t1, "ei") * 16 == 3 * 2 * 16 ** 3 * 8 ** 2


# ---------------------------------------------------------- contractions

@pytest.fixture(scope="module")
def small():
    w = wl.small_doubles(O=8, V=12, to=2, tv=3)
    _, T = O.build_workload(w)
    return w, T


def test_ladder_o8_v32_matches_dense_einsum():
    w = wl.ladder_o8_v32()
    _, T = O.build_workload(w)
    O.run_workload(w, T)
    ref = 0.5 * np.einsum("abef,efij->abij", T["V_vvvv"].to_dense(), T["T"].to_dense())
    R = T["R"]
    np.testing.assert_allclose(R.to_dense(), ref, rtol=0, atol=1e-15 * np.abs(ref).max())
    # zero blocks stay zero: the dense product vanishes wherever R stores no block
    mask = np.zeros(R.dense_shape(), bool)
    lo, ext = R.block_lo_ext()
    for b in range(R.n_blocks):
        mask[tuple(slice(lo[b, m], lo[b, m] + ext[b, m]) for m in range(4))] = True
    assert not ref[~mask].any()
    assert np.abs(ref[mask]).max() > 0


@pytest.mark.parametrize("name,expr,lhs,alpha", [
    ("intermediate", "mnef,efij->mnij", ("V_oovv", "T"), 1.0),
    ("oooo", "abmn,mnij->abij", ("T", "W0"), 0.25),
    ("t1", "abej,ei->abij", ("V_vvvo", "t1"), 1.0),
])
def test_doubles_terms_match_dense_einsum(small, name, expr, lhs, alpha):
    _, T = small
    ins, out = expr.split("->")
    la, lb = ins.split(",")
    C = O.Tensor(T["R"].modes if out == "abij" else T["W"].modes, 2)
    C.data[:] = np.random.default_rng(3).standard_normal(C.n_elems)
    c0 = C.to_dense()
    A, B = T[lhs[0]], T[lhs[1]]
    O.contract(alpha, C, out, 1.0, A, la, B, lb)
    ref = c0 + alpha * np.einsum(expr, A.to_dense(), B.to_dense())
    np.testing.assert_allclose(C.to_dense(), ref, rtol=0, atol=1e-14)


def test_ring_with_antisymmetrizer_matches_dense(small):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    step = wl.ContractSpec("ring", "R", "abij", "T", "aeim", "V_ovvo", "mbej", 1.0, antisym=True)
    O.run_step(None, {"R": R, "T": T["T"], "V_ovvo": T["V_ovvo"]}, step)
    X = np.einsum("aeim,mbej->abij", T["T"].to_dense(), T["V_ovvo"].to_dense())
    ref = X - X.transpose(1, 0, 2, 3) - X.transpose(0, 1, 3, 2) + X.transpose(1, 0, 3, 2)
    got = R.to_dense()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)
    # P(ab)P(ij) output is antisymmetric in (a,b) and in (i,j)
    np.testing.assert_allclose(got, -got.transpose(1, 0, 2, 3), atol=1e-16)
    np.testing.assert_allclose(got, -got.transpose(0, 1, 3, 2), atol=1e-16)


def test_ladder_preserves_antisymmetry(small):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    O.contract(0.5, R, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij")
    d = R.to_dense()
    assert np.abs(d).max() > 0
    np.testing.assert_allclose(d, -d.transpose(1, 0, 2, 3), atol=1e-17)
    np.testing.assert_allclose(d, -d.transpose(0, 1, 3, 2), atol=1e-17)


def test_identity_reproduces_input(small):
    # V_I[a,b,e,f] = (d_ae d_bf - d_af d_be)/2; sum_ef V_I T[e,f,i,j] = T[a,b,i,j] for antisymmetric T.
    _, T = small
    v = T["V_vvvv"].modes[0]
    n = v.n
    dI = np.zeros((n,) * 4)
    for a in range(n):
        for b in range(n):
            dI[a, b, a, b] += 0.5
            dI[a, b, b, a] -= 0.5
    VI = O.Tensor([v] * 4, 2)
    VI.from_dense(dI)
    R = O.Tensor(T["R"].modes, 2)
    O.contract(0.5, R, "abij", 0.0, VI, "abef", T["T"], "efij")
    assert np.array_equal(R.data, 0.5 * T["T"].data)


def test_linearity_in_alpha_and_beta_semantics(small):
    _, T = small
    base = np.random.default_rng(1).standard_normal(T["R"].n_elems)
    outs = []
    for alpha in (0.7, 1.4):
        R = O.Tensor(T["R"].modes, 2)
        R.data[:] = base
        O.contract(alpha, R, "abij", 1.0, T["V_vvvv"], "abef", T["T"], "efij")
        outs.append(R.data - base)
    np.testing.assert_allclose(outs[1], 2 * outs[0], rtol=1e-14, atol=4e-15)
    # beta = 0 ("=") overwrites, even NaN
    R = O.Tensor(T["R"].modes, 2)
    R.data[:] = np.nan
    O.contract(0.7, R, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij")
    np.testing.assert_allclose(R.data, outs[0], rtol=1e-14, atol=4e-15)
    # "-=" is a negative alpha
    R.data[:] = base
    O.contract(-0.7, R, "abij", 1.0, T["V_vvvv"], "abef", T["T"], "efij")
    np.testing.assert_allclose(R.data - base, -outs[0], rtol=1e-14, atol=4e-15)


def test_factorization_cc9_equals_cc10_cc11():
    # Sec. IV.A eqs. (cc9)-(cc11): 1/4 v t t computed directly (n_o^4 n_u^4) equals
    # 1/4 I t with the intermediate I = v t.
    o, v = spin_space(4, 1), spin_space(6, 2)
    seed = 99
    Voovv = filled([o, o, v, v], 2, seed, 3, 0.1)
    T = filled([v, v, o, o], 2, seed, 2, 0.01)
    I = O.Tensor([o, o, o, o], 2)
    O.contract(1.0, I, "mnij", 0.0, Voovv, "mnef", T, "efij")
    R = O.Tensor([v, v, o, o], 2)
    O.contract(0.25, R, "abij", 0.0, T, "abmn", I, "mnij")
    vd, td = Voovv.to_dense(), T.to_dense()
    direct = np.zeros(R.dense_shape())
    for a, b, i, j, m, n, e, f in np.ndindex(6, 6, 4, 4, 4, 4, 6, 6):
        direct[a, b, i, j] += 0.25 * vd[m, n, e, f] * td[e, f, i, j] * td[a, b, m, n]
    np.testing.assert_allclose(R.to_dense(), direct, rtol=0, atol=1e-14 * np.abs(direct).max())


def test_dense_ladder_is_textbook_gemm():
    # Sparsity off: C(a,b,c,d) += A(a,b,m,n) B(m,n,c,d) equals C(i,j) += A(i,k) B(k,j)
    # on the N^2 x N^2 reshapes (Sec. V, eqs. 4d_tc_bm / mm_bm).
    N = 6
    s = O.Space([(N, 1, 0)], tile_sizes=(2, 4))
    A = O.Tensor([s] * 4, 2, "dense")
    B = O.Tensor([s] * 4, 2, "dense")
    C = O.Tensor([s] * 4, 2, "dense")
    rng = np.random.default_rng(5)
    Ad, Bd, Cd = (rng.standard_normal((N,) * 4) for _ in range(3))
    A.from_dense(Ad), B.from_dense(Bd), C.from_dense(Cd)
    O.contract(1.0, C, "abcd", 1.0, A, "abmn", B, "mncd")
    a2, b2 = Ad.reshape(N * N, N * N), Bd.reshape(N * N, N * N)
    naive = Cd.reshape(N * N, N * N).copy()
    for i in range(N * N):
        for j in range(N * N):
            acc = 0.0
            for k in range(N * N):
                acc += a2[i, k] * b2[k, j]
            naive[i, j] += acc
    np.testing.assert_allclose(C.to_dense().reshape(N * N, N * N), naive, rtol=1e-13, atol=1e-13)


def test_energy_is_full_contraction(small):
    _, T = small
    E = O.energy(0.25, T["V_oovv"], "ijab", T["T"], "abij")
    ref = 0.25 * np.einsum("ijab,abij->", T["V_oovv"].to_dense(), T["T"].to_dense())
    assert abs(E - ref) <= 1e-14 * abs(ref) + 1e-18
    Tneg = O.Tensor(T["T"].modes, 2)
    Tneg.data[:] = -T["T"].data
    assert O.energy(0.25, T["V_oovv"], "ijab", Tneg, "abij") == -E


def test_add_with_permutation(small):
    _, T = small
    X = T["T"]
    C = O.Tensor(X.modes, 2)
    C.data[:] = 1.0
    c0 = C.to_dense()
    O.add(-2.0, C, "abij", 1.0, X, "baji")
    np.testing.assert_array_equal(C.to_dense(), c0 * (C.to_dense() != 0) - 2.0 * X.to_dense().transpose(1, 0, 3, 2))


def test_norm(small):
    _, T = small
    assert abs(O.norm(T["V_vvvv"]) - np.linalg.norm(T["V_vvvv"].to_dense())) < 1e-12


def test_contract_box_matches_full(small):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    O.contract(0.5, R, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij")
    b = R.n_blocks // 2
    full = R.block_view(b)
    box = O.contract_box(0.5, R, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", b, [1, 0, 0, 1], [2, 3, 1, 1])
    np.testing.assert_array_equal(box, full[1:3, 0:3, 0:1, 1:2])


@pytest.mark.parametrize("lc,la,lb", [
    ("abij", "abef", "efkj"),   # label k only in B
    ("abij", "abef", "efij_"),  # wrong arity
    ("abij", "abij", "efij"),   # output label in both inputs
    ("abii", "abef", "efij"),   # repeated label
])
def test_invalid_labels_rejected(small, lc, la, lb):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    with pytest.raises(O.OracleError):
        O.contract(1.0, R, lc, 0.0, T["V_vvvv"], la, T["T"], lb)


def test_label_bound_to_two_spaces_rejected(small):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    with pytest.raises(O.OracleError):
        O.contract(1.0, R, "abij", 0.0, T["V_oovv"], "abef", T["T"], "efij")


# -------------------------------------------------- spin + irrep (D2h) rule

# Sec. III.A (user-defined non-zero check), read as D2h: the point group is abelian and
# isomorphic to Z2^3, so its eight irreps are labelled 0..7 and the totally symmetric
# irrep is 0.  The pins below never write the XOR rule: they use the eight characters
# chi_s(g) = (-1)^popcount(s & g) of Z2^3 (Fourier analysis on the group) and the
# group-averaging (Reynolds) projection onto invariant tensors.

def _chi(s, g):
    return -1.0 if bin(s & g).count("1") % 2 else 1.0


def _irrep_groups(mult):
    """alpha then beta groups, irrep g holding mult[g] orbitals in each spin."""
    return [(m, sp, g) for sp in (1, -1) for g, m in enumerate(mult) if m]


def _count_invariant(per_mode_mult):
    """Orbital tuples (one orbital per mode) whose irreps multiply to the totally symmetric
    irrep: (1/8) sum_s prod_modes (sum_g m_g chi_s(g)), the orthogonality of Z2^3's characters."""
    total = 0.0
    for s in range(8):
        prod = 1.0
        for mult in per_mode_mult:
            prod *= sum(m * _chi(s, g) for g, m in enumerate(mult))
        total += prod
    return total / 8


@pytest.mark.parametrize("mult_v,mult_o", [((2,) * 8, (1,) * 8), ((3, 1, 0, 2, 5, 1, 4, 2), (1, 2, 0, 1, 1, 0, 2, 1))])
def test_irrep_storage_closed_form(mult_v, mult_o):
    # Spin rule (3/8 of the spin patterns of a 2|2 tensor: aa|aa, bb|bb and the four mixed ones)
    # times the character-sum count of totally symmetric irrep tuples; with every group split
    # evenly over the eight irreps this is 1/8 of the spin-allowed entries, 3/64 of dense.
    v = O.Space(_irrep_groups(mult_v), tile=1)
    o = O.Space(_irrep_groups(mult_o), tile=1)
    for modes, mults in (([v] * 4, [mult_v] * 4), ([v, v, o, o], [mult_v, mult_v, mult_o, mult_o])):
        T = O.Tensor(modes, 2, "spin_irrep", alloc=False)
        assert T.n_elems == 6 * _count_invariant(mults)
    if len(set(mult_v)) == 1:
        n = 2 * sum(mult_v)
        T = O.Tensor([v] * 4, 2, "spin_irrep", alloc=False)
        assert T.n_elems * 64 == 3 * n ** 4
    # one index pair: an (upper, lower) matrix is nonzero only inside same-spin, same-irrep blocks
    T2 = O.Tensor([v, o], 1, "spin_irrep", alloc=False)
    assert T2.n_elems == 2 * sum(a * b for a, b in zip(mult_v, mult_o))


def test_irrep_hand_listed_blocks():
    # four alpha tiles in irreps 0, 3, 5, 6 (a closed subgroup): a 1|1 matrix keeps the diagonal
    s4 = O.Space([(1, 1, 0), (1, 1, 3), (1, 1, 5), (1, 1, 6)], tile=1)
    M = O.Tensor([s4, s4], 1, "spin_irrep", alloc=False)
    assert M.block_tiles.tolist() == [[0, 0], [1, 1], [2, 2], [3, 3]]
    # two alpha tiles in irreps 1 and 2: 1*1*2*2 etc. -- a 4-tuple is totally symmetric exactly
    # when each irrep occurs an even number of times
    s2 = O.Space([(2, 1, 1), (3, 1, 2)], tile_sizes=(2, 3))
    F = O.Tensor([s2] * 4, 2, "spin_irrep", alloc=False)
    want = [[0, 0, 0, 0], [0, 0, 1, 1], [0, 1, 0, 1], [0, 1, 1, 0],
            [1, 0, 0, 1], [1, 0, 1, 0], [1, 1, 0, 0], [1, 1, 1, 1]]
    assert F.block_tiles.tolist() == want
    assert F.n_elems == 2 ** 4 + 6 * 2 * 2 * 3 * 3 + 3 ** 4
    # irreps 1, 2, 3 in one alpha space: the product of 1, 2 and 3 is symmetric, so a 4-tuple holding
    # all three would need a fourth tile in irrep 0, which the space lacks; what remains are
    # (g, g, g, g) and the six arrangements of each pair {g, g, h, h}
    s3 = O.Space([(1, 1, 1), (1, 1, 2), (1, 1, 3)], tile=1)
    G = O.Tensor([s3] * 4, 2, "spin_irrep", alloc=False)
    assert G.n_blocks == 3 + 3 * 6  # (g,g,g,g) and the six arrangements of each pair {g,g,h,h}


def _reynolds(x, phases):
    """Average of x over a finite group acting by per-mode diagonal phases: phases[k][m] is the
    vector by which mode m's orbitals are multiplied under group element k."""
    out = np.zeros(x.shape, dtype=complex)
    for ph in phases:
        y = x.astype(complex)
        for m, p in enumerate(ph):
            shape = [1] * x.ndim
            shape[m] = -1
            y = y * p.reshape(shape)
        out += y
    return out / len(phases)


def _invariant_dense(spaces, n_upper, rng):
    """Dense random tensor projected onto the tensors invariant under D2h (= Z2^3 characters of the
    orbitals' irreps) and under spin rotation about z (U(1): upper modes carry exp(i t s), lower
    exp(-i t s); t over nine angles, which resolves net spin |d| <= 4)."""
    x = rng.standard_normal(tuple(s.n for s in spaces))
    irr = [np.concatenate([[t[3]] * t[1] for t in s.tiles]).astype(int) for s in spaces]
    spn = [np.concatenate([[t[2]] * t[1] for t in s.tiles]).astype(float) for s in spaces]
    d2h = [[np.array([_chi(g, int(q)) for q in irr[m]]) for m in range(len(spaces))] for g in range(8)]
    x = _reynolds(x, d2h).real
    angles = 2 * np.pi * np.arange(9) / 9
    u1 = [[np.exp(1j * t * spn[m] * (1 if m < n_upper else -1)) for m in range(len(spaces))] for t in angles]
    return _reynolds(x, u1).real


def _irrep_einsum_pin_holds(rng_seed=7) -> bool:
    rng = np.random.default_rng(rng_seed)
    v = O.Space(_irrep_groups((2, 1, 0, 1, 2, 1, 1, 0)), tile=1)
    o = O.Space(_irrep_groups((1, 0, 1, 0, 0, 1, 0, 0)), tile=1)
    Vd = _invariant_dense([v] * 4, 2, rng)
    Td = _invariant_dense([v, v, o, o], 2, rng)
    Vd[np.abs(Vd) < 1e-13] = 0.0
    Td[np.abs(Td) < 1e-13] = 0.0
    V = O.Tensor([v] * 4, 2, "spin_irrep")
    T = O.Tensor([v, v, o, o], 2, "spin_irrep")
    V.from_dense(Vd)
    T.from_dense(Td)
    # the stored blocks hold every entry an invariant tensor can have
    if not (np.array_equal(V.to_dense(), Vd) and np.array_equal(T.to_dense(), Td)):
        return False
    R = O.Tensor([v, v, o, o], 2, "spin_irrep")
    O.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij")
    ref = 0.5 * np.einsum("abef,efij->abij", Vd, Td)
    # the product of invariant tensors is invariant: it vanishes outside R's stored blocks and
    # equals the oracle inside them
    mask = np.zeros(R.dense_shape(), bool)
    lo, ext = R.block_lo_ext()
    for b in range(R.n_blocks):
        mask[tuple(slice(lo[b, m], lo[b, m] + ext[b, m]) for m in range(4))] = True
    scale = np.abs(ref).max()
    if not scale > 0 or np.abs(ref[~mask]).max(initial=0.0) > 1e-13 * scale:
        return False
    return bool(np.allclose(R.to_dense()[mask], ref[mask], rtol=0, atol=1e-14 * scale))


def test_irrep_invariant_dense_einsum():
    assert _irrep_einsum_pin_holds()


# --------------------------------------------------------- mutation tests

MUTANTS = {
    "drop_last_contracted_element": ("for (int64_t k = 0; k < kn; ++k) s +=", "for (int64_t k = 0; k + 1 < kn; ++k) s +="),
    "spin_rule_inverted": ("if (up != lo) return 0;", "if (up == lo) return 0;"),
    "transposed_operand": ("kofs[2 * k] = ka;", "kofs[2 * k] = kb;"),
    "alpha_sign": ("out[e] = prev + alpha * acc[e];", "out[e] = prev - alpha * acc[e];"),
    "skip_second_tile_tuple": ("if (ab < 0 || bb < 0) continue;", "if (ab < 0 || bb < 0 || kt == 1) continue;"),
    "beta_ignored": ("double prev = (beta != 0.0 && c_in) ? beta * c_in[e] : 0.0;", "double prev = 0.0;"),
    "irrep_ignored": ("if (T->sym == OR_SYM_SPIN_IRREP && x != 0) return 0;", ""),
    "irrep_or_not_xor": ("x ^= T->sp[m]->irrep[tt[m]];", "x |= T->sp[m]->irrep[tt[m]];"),
    "irrep_sum_not_xor": ("x ^= T->sp[m]->irrep[tt[m]];", "x += T->sp[m]->irrep[tt[m]];"),
}


def _pins_hold() -> bool:
    """A subset of the pins above, re-run on whatever oracle library is active."""
    try:
        o, v = spin_space(4, 2), spin_space(12, 3)  # every tile longer than 1, so strides differ
        V = filled([v] * 4, 2, 42, 1, 0.1)
        T = filled([v, v, o, o], 2, 42, 2, 0.01)
        R = O.Tensor([v, v, o, o], 2)
        R.data[:] = np.random.default_rng(0).standard_normal(R.n_elems)
        r0 = R.to_dense()
        O.contract(0.5, R, "abij", 1.0, V, "abef", T, "efij")
        ref = r0 + 0.5 * np.einsum("abef,efij->abij", V.to_dense(), T.to_dense())
        if V.n_elems * 8 != 3 * 12 ** 4:
            return False
        if not np.allclose(R.to_dense(), ref, rtol=0, atol=1e-14):
            return False
        vi = O.Space(_irrep_groups((2,) * 8), tile=1)
        if O.Tensor([vi] * 4, 2, "spin_irrep", alloc=False).n_elems * 64 != 3 * 32 ** 4:
            return False
        return _irrep_einsum_pin_holds()
    except O.OracleError:
        return False


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_oracle_mistakes(mutant, tmp_path):
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "tamm_oracle.c")).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) == 1, mutant
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", str(path), "-o", str(lib), "-lm"])
    assert _pins_hold()  # the real oracle passes
    with O.using_library(str(lib)):
        caught = not _pins_hold()
    assert caught, f"planted mistake {mutant!r} was not caught"


def test_contract_blocks_matches_full(small):
    _, T = small
    R1 = O.Tensor(T["R"].modes, 2)
    R2 = O.Tensor(T["R"].modes, 2)
    O.contract(0.5, R1, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij")
    pick = [1, 5, R1.n_blocks - 1]
    O.contract_blocks(0.5, R2, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", pick)
    for b in range(R1.n_blocks):
        if b in pick:
            assert np.array_equal(R2.block_view(b), R1.block_view(b))
        else:
            assert not R2.block_view(b).any()


def test_contract_boxes_match_single_box(small):
    _, T = small
    R = O.Tensor(T["R"].modes, 2)
    boxes = [(0, [0, 0, 0, 0], [2, 3, 1, 2]), (R.n_blocks - 1, [1, 1, 0, 0], [2, 2, 2, 2])]
    outs = O.contract_boxes(0.5, R, "abij", T["V_vvvv"], "abef", T["T"], "efij", [b[0] for b in boxes],
                            [b[1] for b in boxes], [b[2] for b in boxes])
    for (b, lo, ext), got in zip(boxes, outs):
        ref = O.contract_box(0.5, R, "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", b, lo, ext)
        assert np.array_equal(got, ref)


def _paper_values():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            vals[k] = v
    return vals


def test_paper_printed_tiling_example():
    v = _paper_values()
    rows = [int(x) for x in v["tensor_const_tiles_rows"].split(",")]
    cols = [int(x) for x in v["tensor_const_tiles_cols"].split(",")]
    tM = O.Space([(int(v["tensor_const_rows"]), 1, 0)], tile_sizes=rows)
    tK = O.Space([(int(v["tensor_const_cols"]), 1, 0)], tile=cols[0])
    A = O.Tensor([tM, tK], 1, "dense")
    assert A.n_blocks == int(v["tensor_const_blocks"])
    assert [t[1] for t in tK.tiles] == cols


def test_oracle_regression_values():
    import json

    g = json.load(open(os.path.join(HERE, "golden", "oracle_ladder_o8_v32.json")))
    w = wl.ladder_o8_v32()
    _, T = O.build_workload(w)
    O.run_workload(w, T)
    assert abs(O.norm(T["R"]) - g["norm_R"]) <= 1e-13 * g["norm_R"]
    assert abs(O.energy(1.0, T["R"], "abij", T["T"], "abij") - g["R_dot_T"]) <= 1e-13 * abs(g["R_dot_T"])
    assert T["R"].n_blocks == g["n_blocks_R"] and T["V_vvvv"].n_elems == g["n_elems_V_vvvv"]
