"""Writes q1_element_h1.txt: the Q1 (trilinear) hexahedron stiffness K_e, mass
M_e and top-face boundary mass B_f of the unit cube, as exact rationals.

Derivation (standard Q1 FEM, written out here independently of helmgen): with
the 1-D linear-element matrices on [0, 1]
    K1 = [[1, -1], [-1, 1]],   M1 = [[2, 1], [1, 2]] / 6,
the element matrices are tensor products over the axes,
    K_e = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1,   M_e = M1 x M1 x M1,
    B_f = M1 x M1 on the face z = 1 (zero elsewhere),
with local node a = ax + 2 ay + 4 az.  For an element of size h they scale as
K_e h, M_e h^3, B_f h^2.  Run: python tests/golden/make_q1_element.py
"""
import os
from fractions import Fraction as Fr

K1 = [[Fr(1), Fr(-1)], [Fr(-1), Fr(1)]]
M1 = [[Fr(2, 6), Fr(1, 6)], [Fr(1, 6), Fr(2, 6)]]


def bits(a):
    return a & 1, (a >> 1) & 1, (a >> 2) & 1


def matrices():
    K = [[Fr(0)] * 8 for _ in range(8)]
    M = [[Fr(0)] * 8 for _ in range(8)]
    B = [[Fr(0)] * 8 for _ in range(8)]
    for a in range(8):
        ax, ay, az = bits(a)
        for b in range(8):
            bx, by, bz = bits(b)
            K[a][b] = (K1[ax][bx] * M1[ay][by] * M1[az][bz] + M1[ax][bx] * K1[ay][by] * M1[az][bz]
                       + M1[ax][bx] * M1[ay][by] * K1[az][bz])
            M[a][b] = M1[ax][bx] * M1[ay][by] * M1[az][bz]
            if az == 1 and bz == 1:
                B[a][b] = M1[ax][bx] * M1[ay][by]
    return K, M, B


def main():
    K, M, B = matrices()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "q1_element_h1.txt")
    with open(path, "w") as f:
        f.write("# Q1 hexahedron on the unit cube, exact: see make_q1_element.py\n")
        for name, A in (("K", K), ("M", M), ("B", B)):
            f.write(f"{name}\n")
            for row in A:
                f.write(" ".join(str(v) for v in row) + "\n")


if __name__ == "__main__":
    main()
