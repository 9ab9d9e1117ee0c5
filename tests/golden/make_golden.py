"""Writes the stored reference values of tests/golden/ from the oracle only
(route 1, the direct sum of the definition, Eqs. 6 and 9).

    python tests/golden/make_golden.py

The values are a regression fixture for the oracle and a fixed target for
the GPU path: a 16^3 uniform sphere (the unit-box sphere of radius 1/4, as
the 32^3 configuration at half the resolution) and an anisotropic 12x10x8
random source, each at a fixed set of cells.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1106_0557_gb300 import sources  # noqa: E402


def cases():
    w = sources.single_sphere(16)
    yield "sphere16", w.source(), w.h, [0, 7 * 16 * 16 + 7 * 16 + 7, 8 * 16 * 16 + 8 * 16 + 8, 16 ** 3 - 1, 1234]
    g = np.random.default_rng(2024)
    src = g.uniform(0.0, 1.0, (8, 10, 12))
    yield "random12x10x8_h", src, (0.5, 0.25, 1.0), [0, 17, 333, 959, 500]


def main():
    for name, src, h, cells in cases():
        vals = oracle.direct_points(src, h, np.asarray(cells))
        path = os.path.join(HERE, name + ".txt")
        with open(path, "w") as f:
            f.write("# %s: potential at flat C-order cells by the direct sum of Eqs. 6 and 9 (oracle route 1)\n" % name)
            f.write("# written by tests/golden/make_golden.py; widths h = %r, shape (z, y, x) = %r\n"
                    % (tuple(h), src.shape))
            for c, v in zip(cells, vals):
                f.write("%d %.17e\n" % (c, v))
        print("wrote", path)


if __name__ == "__main__":
    main()
