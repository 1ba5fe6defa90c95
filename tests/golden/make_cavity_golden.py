"""Write the closed-form resonance frequencies of a 2D Yee PEC cavity.

For E_z on the vertices of an n x n grid with E_z = 0 on the walls, the
semi-discrete Maxwell system (eq. (mxw) with sigma = 0, eps = mu = 1)
reduces to E_z'' = -(D_x^T D_x + D_y^T D_y) E_z, whose eigenvalues are those
of the Dirichlet five-point Laplacian:
    omega_pq = sqrt( (2 sin(p pi / 2n))^2 + (2 sin(q pi / 2n))^2 ),
    p, q = 1 .. n-1.
This is textbook mathematics (no oracle call).  Run from the repository
root:  python tests/golden/make_cavity_golden.py
"""
import math
import os

N = 6
HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    vals = []
    for p in range(1, N):
        for q in range(1, N):
            vals.append(math.sqrt((2 * math.sin(p * math.pi / (2 * N))) ** 2
                                  + (2 * math.sin(q * math.pi / (2 * N))) ** 2))
    vals.sort()
    with open(os.path.join(HERE, "cavity_2d_n6.txt"), "w") as f:
        f.write("# 2D Yee PEC cavity, n=6 cells, vacuum: closed-form omega_pq, sorted\n")
        f.write("# source: Dirichlet five-point Laplacian eigenvalues; see make_cavity_golden.py\n")
        for v in vals:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
