"""Writes eq18_values.txt: the paper's closed form, eq. 18 (Sect. 5, the
rescaled exact solution 1 - pi/(2x) + sqrt(1-x^2)/x arccos(x) of its 4-D worked
example), at points of the paper's own evaluation grid (Sect. 5.4: 128 x 128
over -5 <= Re x, Im x <= 5), evaluated with mpmath at 40 digits. Uses nothing
but mpmath and the formula; run from the repository root."""
import os

import mpmath as mp

mp.mp.dps = 40
HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    m = n = 128
    rows = []
    # a fixed spread of grid indices over all four quadrants, near and far
    # from the cut x <= -1 and from the origin
    idx = [(0, 0), (0, 127), (127, 0), (127, 127), (63, 64), (64, 63), (40, 90), (90, 40),
           (20, 70), (20, 57), (50, 100), (100, 20), (30, 30), (110, 110), (60, 75), (70, 52),
           (5, 66), (5, 61), (120, 66), (45, 64), (45, 63), (80, 100), (10, 10), (64, 127)]
    for i, j in idx:
        x = mp.mpc(-5 + (i + mp.mpf(1) / 2) * 10 / m, -5 + (j + mp.mpf(1) / 2) * 10 / n)
        g = 1 - mp.pi / (2 * x) + mp.sqrt(1 - x * x) / x * mp.acos(x)
        rows.append(f"{i} {j} {mp.nstr(x.real, 25)} {mp.nstr(x.imag, 25)} "
                    f"{mp.nstr(g.real, 30)} {mp.nstr(g.imag, 30)}")
    with open(os.path.join(HERE, "eq18_values.txt"), "w") as f:
        f.write("# eq. 18 (Sect. 5.1) on the paper's 128x128 grid over [-5,5]^2 (Sect. 5.4),\n")
        f.write("# cell-centred; columns: i j Re(x) Im(x) Re(G) Im(G); written by make_eq18.py\n")
        f.write("\n".join(rows) + "\n")


if __name__ == "__main__":
    main()
