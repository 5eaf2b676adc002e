"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/vfpi.h declares; the binding's structures match the C layout.  No
compute call is made (this runs without a GPU)."""
import ctypes as C
import os
import re
import subprocess
import textwrap

import pytest

from paper_2201_09212_gb300 import build, vfpi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vfpi.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return vfpi.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vfpi_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"{n} declared in vfpi.h but not exported"
    assert set(names) == set(vfpi.EXPORTED)


def test_library_is_built_for_sm_103a():
    log = open(os.path.join(build.OUT, "vfpi_f32.log")).read()
    assert "arch=compute_103a,code=sm_103a" in log


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "vfpi.h"
        int main(void) {
          printf("%zu %zu %zu\\n", sizeof(vfpi_bsr), sizeof(vfpi_contacts), sizeof(vfpi_opts));
          printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(vfpi_opts, theta_th), offsetof(vfpi_opts, l_max),
                 offsetof(vfpi_opts, scene_ptr), offsetof(vfpi_opts, force_path),
                 offsetof(vfpi_contacts, phi), offsetof(vfpi_opts, chebyshev_u),
                 offsetof(vfpi_opts, n_halo));
          return 0;
        }"""))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[0] == C.sizeof(vfpi._Bsr)
    assert sizes[1] == C.sizeof(vfpi._Contacts)
    assert sizes[2] == C.sizeof(vfpi._Opts)
    assert sizes[3] == vfpi._Opts.theta_th.offset
    assert sizes[4] == vfpi._Opts.l_max.offset
    assert sizes[5] == vfpi._Opts.scene_ptr.offset
    assert sizes[6] == vfpi._Opts.force_path.offset
    assert sizes[7] == vfpi._Contacts.phi.offset
    assert sizes[8] == vfpi._Opts.chebyshev_u.offset
    assert sizes[9] == vfpi._Opts.n_halo.offset


def test_host_only_entry_points(L):
    o = vfpi._Opts()
    L.vfpi_default_opts(C.byref(o))
    assert (o.dtype, o.w_mode, o.l_max, o.theta_th, o.n_scenes) == (0, 0, 200, 1e-5, 1)
    assert L.vfpi_status_string(-6) == b"VFPI_ERR_CONTACT_OVERLAP"
    # argument checks happen before any CUDA call
    h = C.c_void_p()
    assert L.vfpi_create(None, None, None, C.c_double(1e-3), C.byref(o), None, C.byref(h)) == -1
    assert b"required" in L.vfpi_last_error(None)
    o.l_max = 0
    bsr = vfpi._Bsr(1, 1, None, None, None)
    assert L.vfpi_create(C.byref(bsr), C.c_void_p(1), None, C.c_double(1e-3), C.byref(o), None,
                         C.byref(h)) == -1
    o.l_max = 10
    o.operator_ = 5
    assert L.vfpi_create(C.byref(bsr), C.c_void_p(1), None, C.c_double(1e-3), C.byref(o), None,
                         C.byref(h)) == -1
    o.operator_ = 0
    o.chebyshev_ls = 3
    assert L.vfpi_create(C.byref(bsr), C.c_void_p(1), None, C.c_double(1e-3), C.byref(o), None,
                         C.byref(h)) == -1
    assert L.vfpi_step(None, None) == -1
    L.vfpi_destroy(None)


def test_product_path_has_no_oracle_import():
    """The package and the entry points' product parts never touch oracle/."""
    pkg = os.path.join(ROOT, "paper_2201_09212_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
