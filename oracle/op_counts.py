"""Algorithmic operation counts of the definitions (test and measurement infrastructure).

Writes ``profiles/algorithmic_ops.json``: for each named mechanism, the floating-point operations
the oracle's definitions perform at one point (counted by its instrumented scalar type, one
count per add/subtract, multiply and divide, and the transcendental calls separately), for the
rates (NASA-7 thermo, rate constants, equilibrium constants, rates of progress, omega_k and the
heat release) and for transport (pure-species fits and mixture rules).  The benchmark reads the
file for its algorithmic flop rates; it does not run the oracle itself.

    python -m oracle.op_counts

The counts come from a point of the flame field (the benchmark's workload); the definitions
have no data-dependent branches but the NASA-7 range choice, which changes no count.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(ROOT, "profiles", "algorithmic_ops.json")
MECHS = ("h2_9sp_21rx", "ch4_53sp_325rx", "big_120sp_700rx")


def counts() -> dict:
    import oracle
    from paper_2409_06404_gb300 import synth
    res = {}
    for name in MECHS:
        mech = synth.mechanism(name)
        st = synth.states_flame(mech.K, 8, seed=7)
        i = st.n // 2
        rec = {}
        for which in ("rates", "transport"):
            c = oracle.count_ops(mech, float(st.T[i]), float(st.p[i]), st.Y[:, i].copy(), which=which)
            c = {k: int(v) for k, v in c.items()}
            c["flops"] = c["add"] + c["mul"] + c["div"]
            c["transcendentals"] = c["exp"] + c["log"] + c["pow"] + c["sqrt"]
            rec[which] = c
        res[name] = {"K": mech.K, "R": mech.R, "per_point": rec}
    return res


def main():
    data = {"source": "oracle.count_ops (instrumented scalar type of oracle/nkoracle.cpp), one point of the "
                      "flame field; flops = add + mul + div, transcendentals = exp + log + pow + sqrt",
            "command": "python -m oracle.op_counts",
            "mechanisms": counts()}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
        f.write("\n")
    print(OUT)


if __name__ == "__main__":
    main()
