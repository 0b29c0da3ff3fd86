"""Writes elibb_printed_weights.txt: the interpolation weights printed in the
paper (Sec. II.B Eq. bfl; Sec. II.D ELIBB-U and Eq. linear_broken_method),
evaluated exactly with fractions. Calls nothing but the printed formulas."""
import os
from fractions import Fraction as Fr

HEADER = """\
# Interpolation weights printed in the paper, evaluated exactly at several q.
# ELIBB-U: Sec. II.D, a4 = 1-q (wall population at s=0), a5 = q (post-collision wall population).
# ELIBB-F: Sec. II.D, Eq. linear_broken_method. q<1/2: a4 on f~_i^{t+1}(x_W), a2 on f*_ibar(x_F);
#   q>=1/2: a2 on f*_ibar(x_F), a5 on f~*_i(x_W). The printed labels are swapped for q<1/2 and the
#   printed q>=1/2 value (2-2q)/q sums to 1/q with a5 (not a partition of unity, and twice
#   half-way bounce-back at q=1/2); the reading used is (1-q)/q, the Lagrange weight of Eq. poli_coeff.
# BFL: Sec. II.B, Eq. bfl. q<1/2: 2q on f*_ibar(x_F), 1-2q on f*_ibar(x_FF);
#   q>=1/2: 1/(2q) on f*_ibar(x_F), (2q-1)/(2q) on f*_i(x_F).
# columns: scheme q point weight   (points: F0=f~_i^{t+1}(x_W) G=f*_ibar(x_F) F1=f~*_i(x_W)
#                                    H=f*_i(x_F) FF=f*_ibar(x_FF))"""


def main():
    qs = [Fr(1, 100), Fr(1, 10), Fr(3, 10), Fr(1, 2), Fr(7, 10), Fr(9, 10), Fr(1)]
    lines = HEADER.splitlines()
    for q in qs:
        lines += [f"U {q} F0 {1 - q}", f"U {q} F1 {q}"]
        if q < Fr(1, 2):
            lines += [f"F {q} F0 {(1 - 2 * q) / (1 - q)}", f"F {q} G {q / (1 - q)}"]
            lines += [f"BFL {q} G {2 * q}", f"BFL {q} FF {1 - 2 * q}"]
        else:
            lines += [f"F {q} G {(1 - q) / q}", f"F {q} F1 {(2 * q - 1) / q}"]
            lines += [f"BFL {q} G {1 / (2 * q)}", f"BFL {q} H {(2 * q - 1) / (2 * q)}"]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "elibb_printed_weights.txt")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
