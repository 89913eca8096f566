"""Write the table of Maxwell coexistence densities used to build initial fields.

TEST/DATA INFRASTRUCTURE: calls only ``oracle.maxwell``.  Output:
``paper_1705_10045_gb300/coexistence_vdw.json`` with rho_v, rho_l and the
saturation pressure p~_s of the reduced van der Waals EOS (Sec. 3) for
T = 0.50, 0.51, ..., 0.99.  The input generators interpolate it linearly in T;
they do no EOS arithmetic themselves.

Run:  python -m oracle.gen_coexistence
"""
import json
import os

from oracle.maxwell import coexistence

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1705_10045_gb300", "coexistence_vdw.json")


def main():
    rows = []
    for i in range(50, 100):
        T = i / 100.0
        rv, rl, ps = coexistence(T)
        rows.append([T, rv, rl, ps])
    doc = {"eos": "reduced van der Waals p = 8 rho T/(3 - rho) - 3 rho^2",
           "rule": "Maxwell equal-area construction",
           "columns": ["T", "rho_v", "rho_l", "p_s"], "rows": rows}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
