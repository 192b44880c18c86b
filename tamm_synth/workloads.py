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
    """``C(lc) = beta*C + alpha * A(la)`` (permuted add)."""
    name: str
    c: str
    lc: str
    a: str
    la: str
    alpha: float
    beta: float = 1.0


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


def config1() -> Workload:
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


def config2() -> Workload:
    """Six doubles-shaped contractions; O=40, V=240, tiles 20/40."""
    w = _doubles(_vt(2, 40, 240, 20, 40, "ccsd_doubles_O40_V240"))
    w.steps = doubles_steps()
    return w


def config4() -> Workload:
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


def config5() -> Workload:
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


CONFIGS = {1: config1, 2: config2, 4: config4, 5: config5}
