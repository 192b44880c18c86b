"""Workload recipes: index spaces, tensors and contraction lists of the synthetic
coupled-cluster-doubles-shaped problems.  Pure data; no arithmetic.

Conventions (shared description; each side builds its own structures from it):

* An index space is an ordered list of contiguous orbital groups
  ``(size, spin, irrep)`` with spin +1 (alpha) or -1 (beta).  Alpha orbitals
  come first, then beta.  Tiles never straddle a group; a fixed tile size
  leaves a smaller remainder tile at the end of a group (e.g. 160 at tile 64
  gives 64, 64, 32).
* A tensor lists its modes by space name, the number of leading "upper" modes
  (spin rule: sum of spins of upper modes equals that of the lower modes), the
  symmetry kind ("spin", "spin_irrep", "dense"), and its synthetic values:
  normal(0, sigma) per dense element, antisymmetrised over mode pairs
  (0,1) and/or (2,3) as flagged, drawn from stream ``stream`` of the seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2201012570


@dataclass(frozen=True)
class SpaceSpec:
    name: str
    groups: tuple  # ((size, spin, irrep), ...)
    tile: int = 0  # fixed tile size, or 0 when tile_sizes is given
    tile_sizes: tuple = ()  # explicit tile sizes covering every group in order

    @property
    def size(self) -> int:
        return sum(g[0] for g in self.groups)


@dataclass(frozen=True)
class TensorSpec:
    name: str
    modes: tuple  # space names
    n_upper: int
    sym: str = "spin"
    sigma: float = 0.0  # 0 => tensor starts at zero
    stream: int = 0
    anti01: bool = False
    anti23: bool = False
    sym01: bool = False  # 3-mode tensors: symmetric in modes 0 and 1 (Cholesky vectors X[p,r,L] = X[r,p,L])
    cholesky: str = ""  # formed on the fly from these Cholesky vectors (Eq. cc12); no stored values


@dataclass(frozen=True)
class ContractSpec:
    """``C(lc) = beta*C + alpha * A(la) * B(lb)``; ``antisym`` adds P(ab)P(ij) on the output."""
    name: str
    c: str
    lc: str
    a: str
    la: str
    b: str
    lb: str
    alpha: float
    beta: float = 1.0
    antisym: bool = False


@dataclass(frozen=True)
class AddSpec:
    """``C(lc) = beta*C + alpha * A(la) + sum alpha_t * A(la_t)`` (permuted add; ``more`` holds the
    extra (alpha_t, la_t) terms, at most three)."""
    name: str
    c: str
    lc: str
    a: str
    la: str
    alpha: float
    beta: float = 1.0
    more: tuple = ()

    @property
    def terms(self) -> list:
        return [(self.alpha, self.la)] + list(self.more)


@dataclass(frozen=True)
class EnergySpec:
    name: str
    a: str
    la: str
    b: str
    lb: str
    alpha: float


@dataclass
class Workload:
    name: str
    seed: int
    spaces: dict
    tensors: dict
    steps: list = field(default_factory=list)  # ContractSpec / AddSpec / EnergySpec in step order


def spin_space(name: str, n_spin_orbitals: int, tile: int) -> SpaceSpec:
    half = n_spin_orbitals // 2
    return SpaceSpec(name, ((half, 1, 0), (half, -1, 0)), tile=tile)


def _vt(seed_k: int, O: int, V: int, to: int, tv: int, name: str) -> Workload:
    return Workload(name, SEED_BASE + seed_k,
                    {"occ": spin_space("occ", O, to), "virt": spin_space("virt", V, tv)}, {})


def ladder_o8_v32() -> Workload:
    """Ladder R[a,b,i,j] += 0.5 sum_ef V[a,b,e,f] T[e,f,i,j]; O=8, V=32, tiles 4/8."""
    w = _vt(1, 8, 32, 4, 8, "ladder_O8_V32")
    w.tensors = {
        "V_vvvv": TensorSpec("V_vvvv", ("virt",) * 4, 2, sigma=0.1, stream=1, anti01=True, anti23=True),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "R": TensorSpec("R", ("virt", "virt", "occ", "occ"), 2),
    }
    w.steps = [ContractSpec("ladder", "R", "abij", "V_vvvv", "abef", "T", "efij", 0.5, beta=0.0)]
    return w


def _doubles(w: Workload) -> Workload:
    w.tensors = {
        "V_vvvv": TensorSpec("V_vvvv", ("virt",) * 4, 2, sigma=0.1, stream=1, anti01=True, anti23=True),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "V_oovv": TensorSpec("V_oovv", ("occ", "occ", "virt", "virt"), 2, sigma=0.1, stream=3,
                             anti01=True, anti23=True),
        "W0": TensorSpec("W0", ("occ",) * 4, 2, sigma=0.1, stream=4, anti01=True, anti23=True),
        "V_ovvo": TensorSpec("V_ovvo", ("occ", "virt", "virt", "occ"), 2, sigma=0.1, stream=5),
        "V_vvvo": TensorSpec("V_vvvo", ("virt", "virt", "virt", "occ"), 2, sigma=0.1, stream=6, anti01=True),
        "t1": TensorSpec("t1", ("virt", "occ"), 1, sigma=0.01, stream=7),
        "W": TensorSpec("W", ("occ",) * 4, 2),
        "X": TensorSpec("X", ("virt", "virt", "occ", "occ"), 2),
        "R": TensorSpec("R", ("virt", "virt", "occ", "occ"), 2),
    }
    return w


def doubles_steps(full: bool = True) -> list:
    """One pass of the six CCSD-doubles-shaped contractions.

    W is re-seeded from W0 each pass (``W = W0``) so that every pass does the
    same work on the same values; R starts at zero (the ladder uses beta = 0).
    """
    s = [
        ContractSpec("ladder", "R", "abij", "V_vvvv", "abef", "T", "efij", 0.5, beta=0.0),
        AddSpec("w_copy", "W", "mnij", "W0", "mnij", 1.0, beta=0.0),
        ContractSpec("intermediate", "W", "mnij", "V_oovv", "mnef", "T", "efij", 1.0),
        ContractSpec("oooo", "R", "abij", "T", "abmn", "W", "mnij", 0.25),
        ContractSpec("ring", "R", "abij", "T", "aeim", "V_ovvo", "mbej", 1.0, antisym=True),
        ContractSpec("t1", "R", "abij", "V_vvvo", "abej", "t1", "ei", 1.0),
    ]
    if full:
        s.append(EnergySpec("energy", "V_oovv", "ijab", "T", "abij", 0.25))
    return s


def ccsd_doubles_o40_v240() -> Workload:
    """Six doubles-shaped contractions; O=40, V=240, tiles 20/40."""
    w = _doubles(_vt(2, 40, 240, 20, 40, "ccsd_doubles_O40_V240"))
    w.steps = doubles_steps()
    return w


def ladder_energy_o32_v192() -> Workload:
    """T' = T + 0.5 V_vvvv T; E = 1/4 V_oovv T'; O=32, V=192, tiles 16/32."""
    w = _vt(4, 32, 192, 16, 32, "ladder_energy_O32_V192")
    w.tensors = {
        "V_vvvv": TensorSpec("V_vvvv", ("virt",) * 4, 2, sigma=0.1, stream=1, anti01=True, anti23=True),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "V_oovv": TensorSpec("V_oovv", ("occ", "occ", "virt", "virt"), 2, sigma=0.1, stream=3,
                             anti01=True, anti23=True),
        "Tp": TensorSpec("Tp", ("virt", "virt", "occ", "occ"), 2),
    }
    w.steps = [
        AddSpec("copy", "Tp", "abij", "T", "abij", 1.0, beta=0.0),
        ContractSpec("ladder", "Tp", "abij", "V_vvvv", "abef", "T", "efij", 0.5),
        EnergySpec("energy", "V_oovv", "ijab", "Tp", "abij", 0.25),
    ]
    return w


def ccsd_doubles_o80_v320() -> Workload:
    """Ladder + ring + oooo; O=80, V=320, tiles 40/64 (V_vvvv about 31 GB)."""
    w = _doubles(_vt(5, 80, 320, 40, 64, "ccsd_doubles_O80_V320"))
    s = doubles_steps(full=False)
    w.steps = [x for x in s if x.name in ("ladder", "w_copy", "oooo", "ring")]
    return w


def small_doubles(O: int = 8, V: int = 24, to: int = 2, tv: int = 4, seed_k: int = 9) -> Workload:
    """Small doubles problem (all six contractions) with ragged-free tiny tiles, for tests."""
    w = _doubles(_vt(seed_k, O, V, to, tv, f"ccsd_doubles_O{O}_V{V}"))
    w.steps = doubles_steps()
    return w


def aux_space(name: str, n_aux: int, tile: int) -> SpaceSpec:
    """Auxiliary (Cholesky-vector) index: one spinless group (spin 0, irrep 0) of n_aux vectors."""
    return SpaceSpec(name, ((n_aux, 0, 0),), tile=tile)


def cholesky_sigma(sigma_v: float, n_aux: int) -> float:
    """Standard deviation of the Cholesky vectors that gives the formed V entries (a sum of 2 n_aux products
    of independent draws) the standard deviation sigma_v."""
    return (sigma_v * sigma_v / (2.0 * n_aux)) ** 0.25


def cholesky_ladder(O: int, V: int, to: int, tv: int, n_aux: int, t_aux: int, seed_k: int) -> Workload:
    """Ladder R[a,b,i,j] = 0.5 sum_ef V[a,b,e,f] T[e,f,i,j] with V_vvvv never stored: it is formed on the fly
    from Cholesky vectors X[p,r,L] (symmetric in p, r; spin-diagonal; L spinless) as
    V[a,b,e,f] = sum_L X[a,e,L] X[b,f,L] - X[a,f,L] X[b,e,L]."""
    w = _vt(seed_k, O, V, to, tv, f"cholesky_ladder_O{O}_V{V}_L{n_aux}")
    w.spaces["aux"] = aux_space("aux", n_aux, t_aux)
    w.tensors = {
        "X": TensorSpec("X", ("virt", "virt", "aux"), 1, sigma=cholesky_sigma(0.1, n_aux), stream=8, sym01=True),
        "V_chol": TensorSpec("V_chol", ("virt",) * 4, 2, cholesky="X"),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "R": TensorSpec("R", ("virt", "virt", "occ", "occ"), 2),
    }
    w.steps = [ContractSpec("ladder", "R", "abij", "V_chol", "abef", "T", "efij", 0.5, beta=0.0)]
    return w


def cholesky_ladder_o40_v240() -> Workload:
    """Cholesky-vector ladder at O=40, V=240 (tiles 20/40) with 2(O+V) = 560 vectors in one aux tile."""
    return cholesky_ladder(40, 240, 20, 40, 560, 560, 7)


def cholesky_ladder_o8_v32() -> Workload:
    """Small Cholesky-vector ladder for tests: O=8, V=32 (tiles 4/8), 80 vectors in tiles of 24 (ragged)."""
    return cholesky_ladder(8, 32, 4, 8, 80, 24, 8)


# the spin-block workloads by name
WORKLOADS = {w.__name__: w for w in (ladder_o8_v32, ccsd_doubles_o40_v240, ladder_energy_o32_v192,
                                     ccsd_doubles_o80_v320)}


def dense4d(N: int, tile: int, seed_k: int = 6) -> Workload:
    """The dense 4-D contraction of the paper's performance comparison (Sec. V):
    C(a,b,c,d) = A(a,b,m,n) B(m,n,c,d), every index of extent N in one space of fixed tiles, every
    block stored; A, B ~ N(0, 0.1), not antisymmetrised."""
    w = Workload(f"dense4d_N{N}_tile{tile}", SEED_BASE + seed_k, {"d": SpaceSpec("d", ((N, 1, 0),), tile=tile)}, {})
    w.tensors = {
        "A": TensorSpec("A", ("d",) * 4, 2, "dense", sigma=0.1, stream=1),
        "B": TensorSpec("B", ("d",) * 4, 2, "dense", sigma=0.1, stream=2),
        "C": TensorSpec("C", ("d",) * 4, 2, "dense"),
    }
    w.steps = [ContractSpec("dense4d", "C", "abcd", "A", "abmn", "B", "mncd", 1.0, beta=0.0)]
    return w


# ------------------------------------------------------------ D2h irreps

def irrep_space(name: str, n_spin_orbitals: int, rng, tile_lo: int = 8, tile_hi: int = 96) -> SpaceSpec:
    """Spin orbitals split half alpha / half beta; each spin's orbitals are assigned to the eight
    D2h irreps (labelled 0..7 so that the product is XOR) by one seeded multinomial draw shared by
    alpha and beta; every (spin, irrep) group is cut into tiles of sizes drawn from U{tile_lo..tile_hi}
    (the last tile of a group takes what is left)."""
    half = n_spin_orbitals // 2
    counts = rng.multinomial(half, [1.0 / 8] * 8)
    groups, tiles = [], []
    for spin in (1, -1):
        for irrep in range(8):
            n = int(counts[irrep])
            if n == 0:
                continue
            groups.append((n, spin, irrep))
            left = n
            while left > 0:
                t = min(int(rng.integers(tile_lo, tile_hi + 1)), left)
                tiles.append(t)
                left -= t
    return SpaceSpec(name, tuple(groups), tile=0, tile_sizes=tuple(tiles))


def irrep_doubles(seed_k: int = 3, O: int = 64, V: int = 384) -> Workload:
    """Uneven D2h blocks: O=64, V=384 spin-orbitals (other sizes for small cases), irrep counts and
    tile cuts seeded; the vvvv ladder and the ring term (spin and irrep block sparsity)."""
    import numpy as np

    seed = SEED_BASE + seed_k
    rng = np.random.default_rng(seed)
    occ = irrep_space("occ", O, rng)
    virt = irrep_space("virt", V, rng)
    w = Workload(f"irrep_doubles_O{O}_V{V}", seed, {"occ": occ, "virt": virt}, {})
    si = "spin_irrep"
    w.tensors = {
        "V_vvvv": TensorSpec("V_vvvv", ("virt",) * 4, 2, si, sigma=0.1, stream=1, anti01=True, anti23=True),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, si, sigma=0.01, stream=2, anti01=True, anti23=True),
        "V_ovvo": TensorSpec("V_ovvo", ("occ", "virt", "virt", "occ"), 2, si, sigma=0.1, stream=5),
        "R": TensorSpec("R", ("virt", "virt", "occ", "occ"), 2, si),
        "R2": TensorSpec("R2", ("virt", "virt", "occ", "occ"), 2, si),
    }
    w.steps = [
        ContractSpec("ladder", "R", "abij", "V_vvvv", "abef", "T", "efij", 0.5, beta=0.0),
        ContractSpec("ring", "R2", "abij", "T", "aeim", "V_ovvo", "mbej", 1.0, beta=0.0, antisym=True),
    ]
    return w


def ladder_batch_sizes(n: int = 32, seed_k: int = 3, o_range=(16, 64), v_range=(64, 320)) -> list:
    """(O, V) of the independent ladder problems: even spin-orbital counts drawn uniformly."""
    import numpy as np

    rng = np.random.default_rng(SEED_BASE + 100 + seed_k)
    out = []
    for _ in range(n):
        o = 2 * int(rng.integers(o_range[0] // 2, o_range[1] // 2 + 1))
        v = 2 * int(rng.integers(v_range[0] // 2, v_range[1] // 2 + 1))
        out.append((o, v))
    return out


def ladder_problem(O: int, V: int, seed: int, to: int = 20, tv: int = 40) -> Workload:
    """One ladder R = 1/2 V_vvvv T of the batch (spin block sparsity)."""
    w = Workload(f"ladder_O{O}_V{V}", seed, {"occ": spin_space("occ", O, to), "virt": spin_space("virt", V, tv)}, {})
    w.tensors = {
        "V_vvvv": TensorSpec("V_vvvv", ("virt",) * 4, 2, sigma=0.1, stream=1, anti01=True, anti23=True),
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "R": TensorSpec("R", ("virt", "virt", "occ", "occ"), 2),
    }
    w.steps = [ContractSpec("ladder", "R", "abij", "V_vvvv", "abef", "T", "efij", 0.5, beta=0.0)]
    return w


def batch_memory_bytes(O: int, V: int, slices: int = 6) -> int:
    """Device bytes of one batch ladder: FP64 V_vvvv, T, R and the slice images of V_vvvv and T."""
    vvvv = 3 * V ** 4 // 8
    t = 3 * V ** 2 * O ** 2 // 8
    return 8 * (vvvv + 2 * t) + 2 * slices * (vvvv + t)


def triples(O: int, V: int, to: int, tv: int, seed_k: int = 7) -> Workload:
    """Inputs of the perturbative triples correction E(T) (Sec. IV.B, Eqs. cc14, tensort, tensort2):
    T2[a,b,i,j] ~ N(0, 0.01) and t1[a,i] ~ N(0, 0.01) as in the doubles recipes, and the three
    two-electron blocks the equations read, V_ooov[i,j,m,a] (antisymmetric in i, j), V_vovv[e,i,a,b]
    (antisymmetric in a, b) and V_oovv[i,j,a,b] (both pairs), ~ N(0, 0.1); spin block sparsity;
    orbital energies from ``orbital_energies``.  The restricted sums run over occupied and
    virtual spin-orbital triples i<j<k, a<b<c."""
    w = _vt(seed_k, O, V, to, tv, f"triples_O{O}_V{V}")
    w.tensors = {
        "T": TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "t1": TensorSpec("t1", ("virt", "occ"), 1, sigma=0.01, stream=7),
        "V_ooov": TensorSpec("V_ooov", ("occ", "occ", "occ", "virt"), 2, sigma=0.1, stream=8, anti01=True),
        "V_vovv": TensorSpec("V_vovv", ("virt", "occ", "virt", "virt"), 2, sigma=0.1, stream=9, anti23=True),
        "V_oovv": TensorSpec("V_oovv", ("occ", "occ", "virt", "virt"), 2, sigma=0.1, stream=3,
                             anti01=True, anti23=True),
    }
    return w


def orbital_energies(w: Workload) -> tuple:
    """Seeded spin-orbital energies (alpha block, then the same values for beta), sorted within each
    spin: occupied -(0.3 + 0.7|z|), virtual 0.2 + 0.8|z| with z a Philox normal, so every triples
    denominator e_i + e_j + e_k - e_a - e_b - e_c is at most -1.5."""
    import tamm_synth

    O, V = w.spaces["occ"].size, w.spaces["virt"].size
    zo = [abs(tamm_synth.normal(w.seed, 10, p)) for p in range(O // 2)]
    zv = [abs(tamm_synth.normal(w.seed, 11, p)) for p in range(V // 2)]
    eo = np.sort(-(0.3 + 0.7 * np.array(zo)))
    ev = np.sort(0.2 + 0.8 * np.array(zv))
    return np.concatenate([eo, eo]), np.concatenate([ev, ev])


def ccsd_residual(O: int, V: int, to: int, tv: int, seed_k: int = 8) -> Workload:
    """One full CCSD residual (T1 and T2 equations and the correlation energy) in spin orbitals,
    canonical Hartree-Fock reference, as a list of library operations: the Stanton-Gauss
    intermediates (tau~, tau, F_ae, F_mi, F_me, W_mnij, W_abef, W_mbej) and then every term of the
    T1 and T2 residuals, each a binary contraction or a permuted add (P(ab), P(ij) and P(ab)P(ij) as
    multi-term adds).  Canonical orbitals make the Fock matrix diagonal, so it enters only the
    amplitude update, not the residual.  Integrals by index type, drawn independently (N(0, 0.1),
    antisymmetrised within same-space pairs); amplitudes T2 ~ N(0, 0.01), t1 ~ N(0, 0.01).
    <mb||ij> is read as <ij||mb> (V_ooov; real orbitals); <am||ef> = -<ma||ef>, <mn||ej> = -<mn||je>,
    <na||if> = -<na||fi>, <nm||ei> = -<nm||ie> (antisymmetry of the lower pair)."""
    w = _vt(seed_k, O, V, to, tv, f"ccsd_residual_O{O}_V{V}")
    o, v = "occ", "virt"
    ts = {
        "T": ((v, v, o, o), 2, 0.01, 2, True, True), "t1": ((v, o), 1, 0.01, 7, False, False),
        "V_oooo": ((o, o, o, o), 2, 0.1, 4, True, True), "V_ooov": ((o, o, o, v), 2, 0.1, 8, True, False),
        "V_oovv": ((o, o, v, v), 2, 0.1, 3, True, True), "V_ovvv": ((o, v, v, v), 2, 0.1, 12, False, True),
        "V_ovvo": ((o, v, v, o), 2, 0.1, 5, False, False), "V_vvvv": ((v, v, v, v), 2, 0.1, 1, True, True),
        "V_vvvo": ((v, v, v, o), 2, 0.1, 6, True, False),
    }
    w.tensors = {n: TensorSpec(n, m, nu, sigma=sg, stream=st, anti01=a01, anti23=a23)
                 for n, (m, nu, sg, st, a01, a23) in ts.items()}
    work = {"Tt": (v, v, o, o), "Tau": (v, v, o, o), "Fvv": (v, v), "Foo": (o, o), "Fov": (o, v),
            "Woooo": (o, o, o, o), "Xoooo": (o, o, o, o), "Wvvvv": (v, v, v, v), "Yvvvv": (v, v, v, v),
            "Wovvo": (o, v, v, o), "Y1": (o, o, v, o), "R1": (v, o), "R2": (v, v, o, o), "Fbe": (v, v),
            "X1": (v, v, o, o), "Fmj": (o, o), "X2": (v, v, o, o), "X3": (v, v, o, o), "Y2": (o, v, o, o),
            "X4": (v, v, o, o), "X5": (v, v, o, o), "Y3": (o, v)}
    for n, m in work.items():
        w.tensors[n] = TensorSpec(n, m, len(m) // 2)
    C, A = ContractSpec, AddSpec
    w.steps = [
        # tau~ = T + 1/2 (t t - t t),  tau = T + (t t - t t)
        A("tt_copy", "Tt", "abij", "T", "abij", 1.0, beta=0.0),
        C("tt_1", "Tt", "abij", "t1", "ai", "t1", "bj", 0.5),
        C("tt_2", "Tt", "abij", "t1", "bi", "t1", "aj", -0.5),
        A("tau_copy", "Tau", "abij", "T", "abij", 1.0, beta=0.0),
        C("tau_1", "Tau", "abij", "t1", "ai", "t1", "bj", 1.0),
        C("tau_2", "Tau", "abij", "t1", "bi", "t1", "aj", -1.0),
        # F_ae, F_mi, F_me
        C("fae_1", "Fvv", "ae", "V_ovvv", "mafe", "t1", "fm", 1.0, beta=0.0),
        C("fae_2", "Fvv", "ae", "Tt", "afmn", "V_oovv", "mnef", -0.5),
        C("fmi_1", "Foo", "mi", "V_ooov", "mnie", "t1", "en", 1.0, beta=0.0),
        C("fmi_2", "Foo", "mi", "V_oovv", "mnef", "Tt", "efin", 0.5),
        C("fme", "Fov", "me", "V_oovv", "mnef", "t1", "fn", 1.0, beta=0.0),
        # W_mnij = <mn||ij> + P(ij) t_j^e <mn||ie> + 1/4 tau_ij^ef <mn||ef>
        A("wmnij_copy", "Woooo", "mnij", "V_oooo", "mnij", 1.0, beta=0.0),
        C("wmnij_x", "Xoooo", "mnij", "V_ooov", "mnie", "t1", "ej", 1.0, beta=0.0),
        A("wmnij_pij", "Woooo", "mnij", "Xoooo", "mnij", 1.0, more=((-1.0, "mnji"),)),
        C("wmnij_tau", "Woooo", "mnij", "V_oovv", "mnef", "Tau", "efij", 0.25),
        # W_abef = <ab||ef> - P(ab) t_m^b <am||ef> + 1/4 tau_mn^ab <mn||ef>
        A("wabef_copy", "Wvvvv", "abef", "V_vvvv", "abef", 1.0, beta=0.0),
        C("wabef_y", "Yvvvv", "abef", "V_ovvv", "maef", "t1", "bm", 1.0, beta=0.0),
        A("wabef_pab", "Wvvvv", "abef", "Yvvvv", "abef", 1.0, more=((-1.0, "baef"),)),
        C("wabef_tau", "Wvvvv", "abef", "Tau", "abmn", "V_oovv", "mnef", 0.25),
        # W_mbej = <mb||ej> + t_j^f <mb||ef> - t_n^b <mn||ej> - (1/2 t_jn^fb + t_j^f t_n^b) <mn||ef>
        A("wmbej_copy", "Wovvo", "mbej", "V_ovvo", "mbej", 1.0, beta=0.0),
        C("wmbej_1", "Wovvo", "mbej", "V_ovvv", "mbef", "t1", "fj", 1.0),
        C("wmbej_2", "Wovvo", "mbej", "V_ooov", "mnje", "t1", "bn", 1.0),
        C("wmbej_3", "Wovvo", "mbej", "T", "fbjn", "V_oovv", "mnef", -0.5),
        C("wmbej_y", "Y1", "mnej", "V_oovv", "mnef", "t1", "fj", 1.0, beta=0.0),
        C("wmbej_4", "Wovvo", "mbej", "Y1", "mnej", "t1", "bn", -1.0),
        # T1 residual (terms that read only inputs first)
        C("r1_ovvo", "R1", "ai", "V_ovvo", "nafi", "t1", "fn", 1.0, beta=0.0),
        C("r1_ovvv", "R1", "ai", "V_ovvv", "maef", "T", "efim", -0.5),
        C("r1_ooov", "R1", "ai", "T", "aemn", "V_ooov", "nmie", 0.5),
        C("r1_fae", "R1", "ai", "Fvv", "ae", "t1", "ei", 1.0),
        C("r1_fmi", "R1", "ai", "t1", "am", "Foo", "mi", -1.0),
        C("r1_fme", "R1", "ai", "T", "aeim", "Fov", "me", 1.0),
        # T2 residual (terms in the order their inputs become ready)
        A("r2_v", "R2", "abij", "V_oovv", "ijab", 1.0, beta=0.0),
        C("r2_vvvo", "X4", "abij", "V_vvvo", "abej", "t1", "ei", 1.0, beta=0.0),
        A("r2_vvvo_pij", "R2", "abij", "X4", "abij", 1.0, more=((-1.0, "abji"),)),
        C("r2_ooov", "X5", "abij", "t1", "am", "V_ooov", "ijmb", 1.0, beta=0.0),
        A("r2_ooov_pab", "R2", "abij", "X5", "abij", -1.0, more=((1.0, "baij"),)),
        C("r2_wmnij", "R2", "abij", "Tau", "abmn", "Woooo", "mnij", 0.5),
        C("r2_wabef", "R2", "abij", "Wvvvv", "abef", "Tau", "efij", 0.5),
        A("fbe_copy", "Fbe", "be", "Fvv", "be", 1.0, beta=0.0),
        C("fbe_1", "Fbe", "be", "t1", "bm", "Fov", "me", -0.5),
        C("r2_fbe", "X1", "abij", "T", "aeij", "Fbe", "be", 1.0, beta=0.0),
        A("r2_fbe_pab", "R2", "abij", "X1", "abij", 1.0, more=((-1.0, "baij"),)),
        A("fmj_copy", "Fmj", "mj", "Foo", "mj", 1.0, beta=0.0),
        C("fmj_1", "Fmj", "mj", "Fov", "me", "t1", "ej", 0.5),
        C("r2_fmj", "X2", "abij", "T", "abim", "Fmj", "mj", 1.0, beta=0.0),
        A("r2_fmj_pij", "R2", "abij", "X2", "abij", -1.0, more=((1.0, "abji"),)),
        C("r2_y2", "Y2", "mbij", "V_ovvo", "mbej", "t1", "ei", 1.0, beta=0.0),
        C("r2_wmbej", "X3", "abij", "T", "aeim", "Wovvo", "mbej", 1.0, beta=0.0),
        C("r2_tty", "X3", "abij", "t1", "am", "Y2", "mbij", -1.0),
        A("r2_ring_pabij", "R2", "abij", "X3", "abij", 1.0,
          more=((-1.0, "baij"), (-1.0, "abji"), (1.0, "baji"))),
        # correlation energy and squared residual norms
        EnergySpec("e_t2", "V_oovv", "ijab", "T", "abij", 0.25),
        C("e_y3", "Y3", "jb", "V_oovv", "ijab", "t1", "ai", 1.0, beta=0.0),
        EnergySpec("e_t1t1", "Y3", "jb", "t1", "bj", 0.5),
        EnergySpec("r1_sq", "R1", "ai", "R1", "ai", 1.0),
        EnergySpec("r2_sq", "R2", "abij", "R2", "abij", 1.0),
    ]
    return w
