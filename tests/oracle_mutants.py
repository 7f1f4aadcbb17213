"""Planted mistakes in a copy of the oracle, to show that a pin catches them.

A mutant is the oracle's C source with one textual replacement, compiled into
a temporary directory; ``mutant(name)`` swaps it in for the oracle's library
for the duration of a ``with`` block. Nothing here runs on a GPU and the
committed oracle is never modified.
"""
from __future__ import annotations

import contextlib
import os
import re
import tempfile

import oracle

_UNWEIGHTED_CONDUCTANCE = """static double edge_conductance(const og_grid *g, int a, const int n[3]) {
  double W, Se, Ss, Sk;
  edge_sums(g, a, n, &W, &Se, &Ss, &Sk);
  int b = (a + 1) % 3, c = (a + 2) % 3, cnt = 0;
  double ks = 0.0;
  for (int db = -1; db <= 0; db++)
    for (int dc = -1; dc <= 0; dc++) {
      int cell[3];
      cell[a] = n[a];
      cell[b] = n[b] + db;
      cell[c] = n[c] + dc;
      if (cell[b] < 0 || cell[b] >= n_of(g, b) || cell[c] < 0 || cell[c] >= n_of(g, c)) continue;
      ks += prop(g, voxel(g, cell), T_K);
      cnt++;
    }
  return (cnt ? ks / cnt : 0.0) * W / g->h[a][n[a]];
}
"""

# name -> list of (regex, replacement); every regex must match exactly once
MUTANTS = {
    # edge conductivity as the harmonic (series) mean of the edge's voxels
    "harmonic_conductance": [
        (r"\*Sk \+= w \* prop\(g, m, T_K\);", "*Sk += w / prop(g, m, T_K);"),
        (r"return Sk / g->h\[a\]\[n\[a\]\];", "return W * W / Sk / g->h[a][n[a]];"),
    ],
    # edge conductivity as the plain (unweighted) mean of the edge's voxels
    "unweighted_conductance": [
        (r"static double edge_conductance\(const og_grid \*g, int a, const int n\[3\]\) \{.*?\n\}\n",
         _UNWEIGHTED_CONDUCTANCE),
    ],
    # the edge's voxels taken from the cell layer below the edge along its axis
    "edge_cell_off_by_one": [
        (r"(\*W = \*Se = \*Ss = \*Sk = 0\.0;.*?)cell\[a\] = n\[a\];",
         r"\1cell[a] = n[a] > 0 ? n[a] - 1 : n[a];"),
    ],
    # thermal strain from the element-centroid rise instead of the Gauss-point rise
    "centroid_rise": [
        (r"dT \+= N\[a\] \* \(T\[", "dT += 0.125 * (T["),
    ],
    # thermal strain from the rise of the element's first node only (a nodal lump)
    "nodal_lump_rise": [
        (r"for \(int a = 0; a < 8; a\+\+\) dT \+= N\[a\] \* \(T\[elem_node\(g, i, j, k, a\)\] - Tref\);",
         "dT = T[elem_node(g, i, j, k, 0)] - Tref;"),
    ],
}


def mutant_source(name: str) -> str:
    with open(oracle._SRC) as f:
        src = f.read()
    for pat, rep in MUTANTS[name]:
        src, n = re.subn(pat, lambda m, r=rep: m.expand(r), src, flags=re.S)
        assert n == 1, f"mutant {name}: pattern {pat!r} matched {n} times"
    return src


@contextlib.contextmanager
def mutant(name: str):
    """Run the enclosed oracle calls against the mutant `name`."""
    saved = (oracle._SRC, oracle._LIB_PATH, oracle._lib)
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "cosim_oracle.c")
        with open(src, "w") as f:
            f.write(mutant_source(name))
        oracle._SRC, oracle._LIB_PATH, oracle._lib = src, os.path.join(d, "mutant.so"), None
        try:
            oracle.lib()
            yield
        finally:
            oracle._SRC, oracle._LIB_PATH, oracle._lib = saved
