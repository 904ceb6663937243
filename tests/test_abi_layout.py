"""The ctypes structures of the Python binding have the layout of the C
header's structs, and the binding's enum constants their values (CPU only:
gcc compiles a probe against include/dmrg3s.h and prints offsetof/sizeof)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mirrors(b):
    return {"dmrg3s_bond": b._Bond, "dmrg3s_site": b._Site, "dmrg3s_env": b._Env,
            "dmrg3s_mpo_site": b._MpoSite, "dmrg3s_update_opts": b._UpdateOpts,
            "dmrg3s_update_info": b._UpdateInfo, "dmrg3s_alpha_rule": b._AlphaRule,
            "dmrg3s_sweep_opts": b._SweepOpts, "dmrg3s_sweep_report": b._SweepReport,
            "dmrg3s_kernel_stats": b._KernelStats}


ENUMS = ["DMRG3S_FP64", "DMRG3S_TF32X3", "DMRG3S_TF32", "DMRG3S_SVD_GESVD", "DMRG3S_SVD_JACOBI",
         "DMRG3S_SVD_AUTO", "DMRG3S_MODEL_XXZ", "DMRG3S_MODEL_HUBBARD", "DMRG3S_MODEL_SPIN_BONDS"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_1501_05504_gb300 import binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dmrg3s.h"', "int main(void) {"]
    for cname, cls in _mirrors(b).items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            cf = fname.rstrip("_")
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, cf, cname, cf))
    for e in ENUMS:
        lines.append('printf("enum %s %%d\\n", (int)%s);' % (e, e))
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines))
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        a, k, v = ln.split()
        res[(a, k)] = int(v)
    return b, res


def test_struct_layouts_match_the_header(c_layout):
    b, res = c_layout
    for cname, cls in _mirrors(b).items():
        assert ctypes.sizeof(cls) == res[(cname, "sizeof")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == res[(cname, fname.rstrip("_"))], (cname, fname)


def test_enum_constants_match_the_header(c_layout):
    b, res = c_layout
    assert b.PRECISIONS["fp64"] == res[("enum", "DMRG3S_FP64")]
    assert b.PRECISIONS["tf32x3"] == res[("enum", "DMRG3S_TF32X3")]
    assert b.PRECISIONS["tf32"] == res[("enum", "DMRG3S_TF32")]
    assert b.SVD_GESVD == res[("enum", "DMRG3S_SVD_GESVD")]
    assert b.SVD_JACOBI == res[("enum", "DMRG3S_SVD_JACOBI")]
    assert b.SVD_AUTO == res[("enum", "DMRG3S_SVD_AUTO")]
    assert b.MODEL_XXZ == res[("enum", "DMRG3S_MODEL_XXZ")]
    assert b.MODEL_HUBBARD == res[("enum", "DMRG3S_MODEL_HUBBARD")]
    assert b.MODEL_SPIN_BONDS == res[("enum", "DMRG3S_MODEL_SPIN_BONDS")]
    # a zero-filled update_opts selects FP64 products and the gesvd SVD
    assert res[("enum", "DMRG3S_FP64")] == 0 and res[("enum", "DMRG3S_SVD_GESVD")] == 0
