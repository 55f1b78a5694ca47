"""The ctypes mirrors of the C ABI's structs (binding.py) have the C layout:
every field at the offset the C compiler gives it, and the same total size.
A small C program built from include/qttpdip.h prints the offsets (host only)."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1808_02558_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (C type, ctypes class, [(C field, ctypes field)])
LAYOUTS = [
    ("qp_scene", binding.Scene,
     [("M", "M"), ("pos", "pos"), ("vel", "vel"), ("omega", "omega"), ("radius", "radius"), ("inv_mass", "inv_mass"),
      ("inv_inertia", "inv_inertia"), ("floor_z", "floor_z"), ("gravity", "gravity"), ("dt", "dt"),
      ("delta", "delta"), ("mu", "mu"), ("slots", "slots"), ("nwalls", "nwalls"), ("wall_axis", "wall_axis"),
      ("wall_sign", "wall_sign"), ("wall_offset", "wall_offset")]),
    ("qp_contacts", binding.Contacts,
     [("M", "M"), ("Nc", "Nc"), ("L", "L"), ("slots", "slots"), ("P", "P"), ("body_a", "body_a"),
      ("body_b", "body_b"), ("phi", "phi"), ("frame", "frame"), ("point", "point"), ("arm_a", "arm_a"),
      ("arm_b", "arm_b"), ("key", "key"), ("r", "r"), ("plane", "plane")]),
    ("qp_state", binding.State, [("gamma", "gamma"), ("lambda", "lam"), ("t", "t")]),
    ("qp_prev_contacts", binding.PrevContacts,
     [("Nc", "Nc"), ("slots", "slots"), ("body_a", "body_a"), ("body_b", "body_b"), ("gamma", "gamma"),
      ("plane", "plane")]),
    ("qp_solve_opts", binding.SolveOpts,
     [("precond", "precond"), ("X", "X"), ("tol", "tol"), ("maxit", "maxit"), ("mixed", "mixed"),
      ("inner_tol", "inner_tol"), ("max_outer", "max_outer"), ("core_dtype", "core_dtype"), ("krylov", "krylov")]),
    ("qp_solve_stats", binding.SolveStats,
     [("status", "status"), ("iters", "iters"), ("outer", "outer"), ("rel_res", "rel_res"), ("ms", "ms"),
      ("fallback", "fallback")]),
    ("qp_pdip_opts", binding.PdipOpts,
     [("nu", "nu"), ("alpha", "alpha"), ("beta", "beta"), ("step_frac", "step_frac"), ("max_halvings", "max_halvings"),
      ("solve", "solve"), ("qtt_refresh", "qtt_refresh"), ("qtt_eps", "qtt_eps"), ("qtt_rmax", "qtt_rmax")]),
    ("qp_pdip_stats", binding.PdipStats,
     [("status", "status"), ("eta", "eta"), ("t", "t"), ("r_dual", "r_dual"), ("r_t", "r_t"), ("s", "s"),
      ("halvings", "halvings"), ("solve", "solve"), ("ms_refresh", "ms_refresh")]),
    ("qp_batch_opts", binding.BatchOpts,
     [("tol", "tol"), ("maxit", "maxit"), ("inner_tol", "inner_tol"), ("max_outer", "max_outer"),
      ("block_threads", "block_threads"), ("split", "split"), ("precond", "precond"),
      ("core_dtype", "core_dtype"), ("qtt_tile", "qtt_tile")]),
]


def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qttpdip.h"', "int main(void) {"]
    for ctype, _, fields in LAYOUTS:
        lines.append(f'  printf("{ctype} size %zu\\n", sizeof({ctype}));')
        for cf, _ in fields:
            lines.append(f'  printf("{ctype} {cf} %zu\\n", offsetof({ctype}, {cf}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    return got


def test_struct_layouts_match_the_header():
    lay = c_layout()
    for ctype, cls, fields in LAYOUTS:
        assert C.sizeof(cls) == lay[(ctype, "size")], ctype
        for cf, pf in fields:
            assert getattr(cls, pf).offset == lay[(ctype, cf)], (ctype, cf)
        # every ctypes field is accounted for
        assert [f[0] for f in cls._fields_] == [pf for _, pf in fields], ctype
