"""Writes tests/golden/l2_coeffs.txt from the oracle only (Eq. "l2cost",
exact rational minimiser of int_0^1 (1 - z p(z))^2 dz).

Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pp_oracle as O  # noqa: E402


def main():
    lines = ["# l2-optimal polynomial coefficients c[0..d], p(z) = sum_i c[i] z^i",
             "# Eq. l2cost (Sec. 3.1): p = argmin_q int_0^1 (1 - q(z) z)^2 dz",
             "# written by tests/golden/make_golden.py from oracle.pp_oracle.poly_coeffs_l2",
             "# format: d: c0 c1 ... cd   (exact rationals)"]
    for d in range(0, 9):
        lines.append("%d: %s" % (d, " ".join(str(c) for c in O.poly_coeffs_l2(d))))
    with open(os.path.join(HERE, "l2_coeffs.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
