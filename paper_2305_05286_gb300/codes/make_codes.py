"""Regenerate the committed QC base matrices of this directory.

Run from the repository root:  python -m paper_2305_05286_gb300.codes.make_codes
The text files are the source of truth; this script only documents how they were drawn.
"""
import os

from paper_2305_05286_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    b = inputs.make_dual_diagonal_code(mb=12, nb=24, Z=24, col_weight=3, seed=1)
    inputs.save_base(os.path.join(HERE, "qc_12x24_z24_seed1.txt"), b, 24,
                     "12x24 base, Z=24 (N=576, rate 1/2), seed 1.\n"
                     "Info columns 0-11: weight 3, shifts uniform in [0,Z), 4-cycles rejected.\n"
                     "Parity columns 12-23: lower bidiagonal of identity blocks (last column weight 1).")
    b = inputs.make_dual_diagonal_code(mb=12, nb=24, Z=96, col_weight=3, seed=4)
    inputs.save_base(os.path.join(HERE, "qc_12x24_z96_seed4.txt"), b, 96,
                     "12x24 base, Z=96 (N=2304, rate 1/2), seed 4; same structure as the Z=24 code.")
    b = inputs.make_dual_diagonal_code(mb=12, nb=24, Z=96, col_weight=3, seed=4, parity="hb")
    inputs.save_base(os.path.join(HERE, "qc_12x24_z96_seed4_hb.txt"), b, 96,
                     "12x24 base, Z=96 (N=2304, rate 1/2), seed 4, info columns by the same recipe.\n"
                     "Parity columns 12-23 in the IEEE 802.16e form: column 12 has weight 3 (rows 0\n"
                     "and 11 shift 1, row 6 shift 0), columns 13-23 hold rows j-1 and j (shift 0).")
    b = inputs.make_extension_code(mb=46, nb=68, kb=22, core=4, Z=384, density=0.25, seed=2)
    inputs.save_base(os.path.join(HERE, "qc_46x68_z384_seed2.txt"), b, 384,
                     "46x68 base, Z=384 (N=26112, K=8448, rate 22/68), seed 2.\n"
                     "Rows 0-3 x columns 22-25: dual-diagonal (lower bidiagonal) core, shift 0.\n"
                     "Rows 4-45: weight-1 extension column 22+r, shift 0.\n"
                     "Info columns (all rows) and core parity columns (extension rows): density 0.25,\n"
                     "shifts uniform in [0,Z), 4-cycles rejected; then every info column is topped up\n"
                     "to two entries in the core rows 0-3.")


# PEG codes of the paper's simulations (Sec. V): rate 1/2, N = 2048.
PEG_IRREGULAR_LAMBDA = {2: 0.45, 3: 0.3708, 4: 0.0307, 12: 0.1485}


def make_peg():
    import numpy as np

    rows = inputs.peg_graph(np.full(2048, 3), 1024, seed=5)
    inputs.save_rows(os.path.join(HERE, "peg_3_6_n2048_seed5.txt"), rows, 2048,
                     "Regular (3,6) PEG code, N=2048, M=1024 (rate 1/2), seed 5; "
                     "one line of variable indices per check")
    deg = inputs.peg_degrees(2048, PEG_IRREGULAR_LAMBDA)
    rows = inputs.peg_graph(deg, 1024, seed=6)
    inputs.save_rows(os.path.join(HERE, "peg_irr_n2048_seed6.txt"), rows, 2048,
                     "Irregular PEG code, N=2048, M=1024, lambda(x) = 0.45x + 0.3708x^2 + "
                     "0.0307x^3 + 0.1485x^11 (edge perspective), seed 6; "
                     "one line of variable indices per check")


# Mixed batch: eight codes of the same dual-diagonal structure, (Z, rate, mb x nb).
MIXED = [(16, "1/3", 16, 24), (32, "2/5", 15, 25), (64, "1/2", 12, 24), (96, "2/3", 8, 24),
         (128, "3/4", 6, 24), (192, "5/6", 4, 24), (256, "8/9", 3, 27), (384, "1/2", 12, 24)]


def mixed_name(i):
    Z, _, mb, nb = MIXED[i]
    return f"mix{i}_{mb}x{nb}_z{Z}"


def make_mixed():
    for i, (Z, rate, mb, nb) in enumerate(MIXED):
        b = inputs.make_dual_diagonal_code(mb=mb, nb=nb, Z=Z, col_weight=min(3, mb), seed=300 + i)
        inputs.save_base(os.path.join(HERE, mixed_name(i) + ".txt"), b, Z,
                         f"Mixed-batch code {i}: {mb}x{nb} base, Z={Z}, rate {rate}, seed {300 + i}.\n"
                         "Info columns: weight min(3, mb), shifts uniform, 4-cycles rejected;\n"
                         "parity columns: lower bidiagonal of identity blocks.")


if __name__ == "__main__":
    main()
    make_mixed()
    make_peg()
