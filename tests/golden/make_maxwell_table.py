"""Writes maxwell_9_49.json: coexistence densities (rho_v, rho_l) of the vdW
fluid P = rho T / (1 - b rho) - a rho^2 with a = 9/49, b = 2/21 (T_c = 4/7,
rho_c = 3.5) on a grid of reduced temperatures T_r = T / T_c from 0.690 to
0.995 in steps of 0.001, computed by the oracle's Maxwell construction
(oracle/thermo.py: equal pressure and equal chemical potential).  The sweep
of bench.py lays out its planar slabs from this table (linear
interpolation), so that the benchmark itself executes no oracle code.

    python tests/golden/make_maxwell_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import thermo as TH  # noqa: E402

A, B = 9.0 / 49.0, 2.0 / 21.0


def main():
    Tc = 8 * A / (27 * B)
    trs = [round(0.690 + 0.001 * i, 3) for i in range(306)]
    rows = []
    for tr in trs:
        rv, rl = TH.maxwell(tr * Tc, A, B)
        rows.append([tr, rv, rl])
    out = {"what": "Maxwell coexistence densities of the vdW fluid a = 9/49, b = 2/21 (T_c = 4/7)",
           "source": "oracle/thermo.py maxwell(), written by tests/golden/make_maxwell_table.py",
           "columns": ["T_r", "rho_v", "rho_l"], "rows": rows}
    with open(os.path.join(HERE, "maxwell_9_49.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
