"""The library's slice and composite-layer helpers against the oracle, on the CPU.

The integer device helpers of csrc/fields.cuh and csrc/common.cuh are compiled with the host C++
compiler against a stand-in for the CUDA runtime header and must equal the oracle exactly on seeded
lattices of every boundary kind:
* TNMCMC-1 slices (Algorithm 2): slice geometry with its Philox fixed lines, held-layer field
  energies and in-plane bond energies of Ising and Potts spins (oracle/model.py);
* TNMCMC-2 composite layers (SM II.B): superspin states, superspin field energies, the two-layer bond
  tables and the composite sweep schedule (oracle/superspin.py).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import model, superspin
from paper_2509_23945_gb300 import inputs, tnmc

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_23945_gb300", "csrc")

CASES = [
    (model.MODEL_EA_PM, (3, 2, 4), (0, 0, 1), 2, 1, model.FIX_R1),
    (model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 2, 0, model.FIX_R1),
    (model.MODEL_EA_GAUSS, (3, 3, 3), (1, 1, 1), 0, 1, model.FIX_R1),
    (model.MODEL_EA_PM, (4, 3, 3), (1, 1, 1), 2, 2, model.FIX_R2),
    (model.MODEL_EA_GAUSS, (2, 3, 2), (1, 0, 0), 0, 1, model.FIX_R1),
    (model.MODEL_EA_GAUSS, (2, 4, 3), (1, 0, 1), 0, 0, model.FIX_R1),
    (model.MODEL_EA_PM, (4, 3, 4), (1, 1, 1), 1, 2, model.FIX_R1),
    (model.MODEL_EA_GAUSS, (6, 6, 6), (1, 1, 1), 1, 5, model.FIX_R1),
    (model.MODEL_EA_PM, (5, 5, 5), (1, 1, 1), 2, 4, model.FIX_R2),
    (model.MODEL_EA_GAUSS, (3, 4, 5), (0, 0, 0), 0, 1, model.FIX_R1),
]


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("composite") / "slice_helpers")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(HERE, "host_shim"), "-I", CSRC,
                    os.path.join(HERE, "host_shim", "slice_helpers.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_composite_helpers_equal_oracle(helper, ci):
    mdl, dims, bc, axis, k, fix = CASES[ci]
    for seed in range(2):
        J = inputs.make_couplings(mdl, dims, bc, seed + 10 * ci)
        spins = inputs.make_spins(1, dims, 2, seed + 7)[0]
        sd, st, ch = 1000 + seed, 3 + ci, seed % 3
        text = f"{dims[0]} {dims[1]} {dims[2]} {bc[0]} {bc[1]} {bc[2]} {mdl} {fix} {axis} {k} {sd} {st} {ch}\n"
        text += " ".join(str(int(v)) for v in spins.reshape(-1)) + "\n"
        text += " ".join(str(int(v)) for v in J.reshape(-1)) + "\n"
        out = subprocess.run([helper], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
        g = superspin.geometry(dims, bc, axis, k, fix, sd, st, ch)
        assert tuple(map(int, out[0].split())) == (g.m, g.Lc, g.y0, g.x0)
        eh, ev, hf = superspin.terms(mdl, dims, spins, J, g)
        so = superspin.active_superspins(spins, dims, g)
        line = 1
        for r in range(g.m):
            for x in range(g.Lc):
                vals = list(map(int, out[line].split()))
                line += 1
                assert vals[0] == so[r, x]
                assert vals[1:5] == list(hf[r, x])
                assert vals[5:21] == list(eh[r, x].reshape(-1))
                assert vals[21:37] == list(ev[r, x].reshape(-1))
        for ln in out[line:]:
            head, tail = ln.split(":")
            n, per, off, c = map(int, head.split()[1:])
            got = list(map(int, tail.split()))
            for classes in (superspin.composite_classes(n, bool(per), off), tnmc.composite_classes(n, bool(per), off)):
                assert got == (classes[c] if c < len(classes) else []), (n, per, off, c)


SINGLE_CASES = [
    (model.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 2, 1, model.FIX_R1),
    (model.MODEL_EA_GAUSS, (4, 3, 5), (1, 1, 1), 0, 2, model.FIX_R2),
    (model.MODEL_EA_PM, (3, 3, 3), (0, 0, 0), 1, 0, model.FIX_R1),
    (model.MODEL_EA_GAUSS, (4, 3, 4), (0, 1, 1), 2, 3, model.FIX_R1),
    (model.MODEL_POTTS, (3, 4, 3), (1, 1, 1), 1, 2, model.FIX_R1),
    (model.MODEL_POTTS, (4, 3, 5), (0, 0, 0), 2, 4, model.FIX_R1),
    (model.MODEL_EA_PM, (2, 3, 2), (1, 1, 0), 0, 1, model.FIX_R2),
]


@pytest.mark.parametrize("ci", range(len(SINGLE_CASES)))
def test_slice_helpers_equal_oracle(helper, ci):
    mdl, dims, bc, axis, k, fix = SINGLE_CASES[ci]
    d = 3 if mdl == model.MODEL_POTTS else 2
    table = model.pair_table(mdl, d)
    for seed in range(2):
        J = inputs.make_couplings(mdl, dims, bc, seed + 20 * ci)
        spins = inputs.make_spins(1, dims, d, seed + 3)[0]
        sd, st, ch = 500 + seed, 1 + ci, seed
        text = f"{dims[0]} {dims[1]} {dims[2]} {bc[0]} {bc[1]} {bc[2]} {mdl} {fix} {axis} {k} {sd} {st} {ch}\n"
        text += " ".join(str(int(v)) for v in spins.reshape(-1)) + "\n"
        text += " ".join(str(int(v)) for v in J.reshape(-1)) + "\n"
        out = subprocess.run([helper, "1"], input=text, capture_output=True, text=True,
                             check=True).stdout.splitlines()
        g = model.slice_geometry(dims, bc, axis, k, fix, sd, st, ch)
        assert tuple(map(int, out[0].split())) == (g.m, g.Lc, g.y0, g.x0)
        Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
        s_old = model.active_spins(spins, dims, g)
        line = 1
        for r in range(g.m):
            for x in range(g.Lc):
                vals = list(map(int, out[line].split()))
                line += 1
                assert vals[0] == s_old[r, x]
                assert vals[1:1 + d] == list(hf[r, x])
                eh = (Jh[r, x] * table).reshape(-1) if (x + 1 < g.Lc or g.ring) else np.zeros(d * d, dtype=np.int64)
                ev = (Jv[r, x] * table).reshape(-1) if r + 1 < g.m else np.zeros(d * d, dtype=np.int64)
                assert vals[1 + d:1 + d + d * d] == list(eh)
                assert vals[1 + d + d * d:] == list(ev)
