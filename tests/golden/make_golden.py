"""Write tests/golden/oracle_ladder_o8_v32.json and oracle_cholesky_ladder_o8_v32.json from the FP64
oracle only.

Regression values for the 8/32 spin-orbital ladder (tiles 4/8), with V_vvvv stored and with V_vvvv formed
from 80 Cholesky vectors (Eq. cc12): norms and scalar contractions.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from tamm_synth import workloads as wl  # noqa: E402


def main():
    w = wl.ladder_o8_v32()
    _, T = O.build_workload(w)
    O.run_workload(w, T)
    out = {
        "workload": "ladder O=8 V=32 tiles 4/8, seed %d" % w.seed,
        "norm_R": O.norm(T["R"]),
        "norm_V_vvvv": O.norm(T["V_vvvv"]),
        "R_dot_T": O.energy(1.0, T["R"], "abij", T["T"], "abij"),
        "n_blocks_R": int(T["R"].n_blocks),
        "n_elems_V_vvvv": int(T["V_vvvv"].n_elems),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_ladder_o8_v32.json"), "w") as f:
        json.dump(out, f, indent=1)

    w = wl.cholesky_ladder_o8_v32()
    _, T = O.build_workload(w)
    O.run_workload(w, T)
    out = {
        "workload": "Cholesky ladder O=8 V=32 tiles 4/8, 80 vectors in tiles of 24, seed %d" % w.seed,
        "norm_X": O.norm(T["X"]),
        "norm_V": O.norm(T["V_chol"]),
        "norm_R": O.norm(T["R"]),
        "R_dot_T": O.energy(1.0, T["R"], "abij", T["T"], "abij"),
        "n_elems_X": int(T["X"].n_elems),
        "n_elems_V": int(T["V_chol"].n_elems),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cholesky_ladder_o8_v32.json"),
              "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
