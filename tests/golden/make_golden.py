"""Write the O2 and small regional golden fixtures from the oracle alone.

The paper prints no worked example for the grids or operators (it names the
"O32" grid in Sec. 4.3 only), so these fixtures freeze the oracle's own O2
mesh and dual, and the geometry of a 4 x 3 Lambert conformal grid, for
regression: connectivity as integers, geometry as hex-encoded float64.  Run
``python tests/golden/make_golden.py`` from the repository root; it imports
nothing but ``oracle`` and the domain table of ``synthetic/regional.py``.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle.oracle import Mesh, RegionalMesh  # noqa: E402
from synthetic.regional import DOMAINS  # noqa: E402

R = 6371220.0


def main():
    m = Mesh(2, R)
    d = m.mesh()
    du = m.dual()
    with open(os.path.join(HERE, "o2_connectivity.txt"), "w") as fh:
        fh.write("# O2 octahedral mesh from oracle/atlas_oracle.c: nnodes ntri nedges\n")
        fh.write("%d %d %d\n" % (m.nnodes, m.ntri, m.nedges))
        fh.write("# e2n (a b is_pole), one edge per line, sorted by (a, b)\n")
        for (a, b), p in zip(d["e2n"], d["is_pole"]):
            fh.write("%d %d %d\n" % (a, b, p))
        fh.write("# n2e_ptr\n" + " ".join(str(int(x)) for x in d["n2e_ptr"]) + "\n")
    with open(os.path.join(HERE, "o2_dual.txt"), "w") as fh:
        fh.write("# O2 median dual, R = 6371220 m, float64 as hex: V per node, then S (lambda, phi) per edge\n")
        for v in du["V"]:
            fh.write(float(v).hex() + "\n")
        for s0, s1 in du["S"]:
            fh.write("%s %s\n" % (float(s0).hex(), float(s1).hex()))

    proj, kw = DOMAINS["lambert"]
    g = RegionalMesh(proj, 4, 3, **kw).geometry()
    with open(os.path.join(HERE, "lambert_4x3.txt"), "w") as fh:
        fh.write("# 4 x 3 Lambert conformal grid (synthetic/regional.py 'lambert') from oracle/regional_oracle.c:\n")
        fh.write("# per node, float64 as hex: lon lat (radians) h_x h_y area (m^2)\n")
        for i in range(len(g["lon"])):
            fh.write(" ".join(float(g[k][i]).hex() for k in ("lon", "lat", "hx", "hy", "area")) + "\n")


if __name__ == "__main__":
    main()
