"""The C-ABI library builds, loads without a GPU, exports every entry point that include/gsdf.h
declares, and its Python binding agrees with the header's struct layouts (checked by a C
program compiled against the header).  No compute calls: this file runs without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2111_13652_gb300 import build as B
from paper_2111_13652_gb300 import gsdf as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsdf.h")


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsdf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gsdf_create", "gsdf_integrate", "gsdf_track_step", "gsdf_extract_voxels"]:
        assert required in names
    assert set(names) == set(G._SIGS), "binding and header disagree"


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gsdf_[a-z_0-9]+)\b", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    L = C.CDLL(lib_path)  # loads without a GPU
    for name in declared_functions():
        assert getattr(L, name) is not None


def test_status_strings_without_gpu(lib_path):
    L = G.load_library(lib_path)
    assert L.gsdf_status_string(0) == b"ok"
    assert b"capacity" in L.gsdf_status_string(G.GSDF_ERR_CAPACITY)
    assert L.gsdf_status_string(99) == b"unknown status"


def test_argument_errors_without_gpu(lib_path):
    """Null or inconsistent arguments are rejected before any CUDA call."""
    L = G.load_library(lib_path)
    h = C.c_void_p()
    assert L.gsdf_create(None, None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    bad = G.make_config(0.01, hash_slots=1000)  # not a power of two
    assert L.gsdf_create(C.byref(bad), None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    bad = G.make_config(0.01, truncation=0.001)  # T < v_s / 2
    assert L.gsdf_create(C.byref(bad), None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    bad = G.make_config(0.01, dense_dims=(0, 4, 4))
    assert L.gsdf_create(C.byref(bad), None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_sync(None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_destroy(None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_track_step(None, None, None, None, None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_integrate(None, None, None, None, None) == G.GSDF_ERR_INVALID_ARG
    nul = [None] * 3
    assert L.gsdf_gn_update(-1, None, None, 0.0, *nul, None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_gn_update(0, None, None, 0.0, *nul, None) == G.GSDF_OK  # nothing to do
    assert L.gsdf_gn_update(1, None, None, 0.0, *nul, None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_gn_update(0, None, None, -1e-4, *nul, None) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_gn_update(0, None, None, float("nan"), *nul, None) == G.GSDF_ERR_INVALID_ARG


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "gsdf.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gsdf_config), sizeof(gsdf_intrinsics),
         sizeof(gsdf_track_stats), sizeof(gsdf_integrate_stats), sizeof(gsdf_voxel),
         offsetof(gsdf_config, damping));
  printf("%zu %zu %zu\n", offsetof(gsdf_config, hash_slots), offsetof(gsdf_track_stats, xi),
         offsetof(gsdf_voxel, w));
  printf("%zu %zu %zu\n", sizeof(gsdf_point), offsetof(gsdf_point, p), offsetof(gsdf_point, n));
  printf("%zu %zu\n", sizeof(gsdf_triangle), offsetof(gsdf_triangle, v));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [C.sizeof(G.gsdf_config), C.sizeof(G.gsdf_intrinsics), C.sizeof(G.gsdf_track_stats),
                    C.sizeof(G.gsdf_integrate_stats), C.sizeof(G.gsdf_voxel), G.gsdf_config.damping.offset,
                    G.gsdf_config.hash_slots.offset, G.gsdf_track_stats.xi.offset, G.gsdf_voxel.w.offset,
                    C.sizeof(G.gsdf_point), G.gsdf_point.p.offset, G.gsdf_point.n.offset,
                    C.sizeof(G.gsdf_triangle), G.gsdf_triangle.v.offset]
    assert G.TRIANGLE_DTYPE.itemsize == C.sizeof(G.gsdf_triangle) == 52
    assert G.VOXEL_DTYPE.itemsize == C.sizeof(G.gsdf_voxel) == 32
    assert G.POINT_DTYPE.itemsize == C.sizeof(G.gsdf_point) == 40
    assert G.POINT_DTYPE.fields["p"][1] == G.gsdf_point.p.offset and G.POINT_DTYPE.fields["n"][1] == G.gsdf_point.n.offset


def test_gn_update_binding_rejects_bad_tensors_without_gpu(lib_path):
    """The binding checks device, dtype, contiguity and shape before any library call."""
    torch = pytest.importorskip("torch")
    G.load_library(lib_path)
    n = 3
    Hb = torch.zeros((n, 27), dtype=torch.float64)
    nv = torch.zeros(n, dtype=torch.int64)
    T = torch.eye(4, dtype=torch.float64).repeat(n, 1, 1)
    with pytest.raises(ValueError, match="Hb"):
        G.gn_update(Hb, nv, 0.0, T)  # host tensors
    with pytest.raises(ValueError, match="Hb"):
        G.gn_update(Hb.float(), nv, 0.0, T)
