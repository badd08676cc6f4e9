"""The C-ABI library loads and exports every function include/seismic.h
declares; the binding's struct layouts match the header.  CPU only: no
compute call is made (there may be no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "seismic.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path), path


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(seismic_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("seismic_build", "seismic_search", "seismic_search_exact", "seismic_free", "seismic_last_error",
              "seismic_set_knn", "seismic_build_knn", "seismic_save", "seismic_load", "seismic_export",
              "seismic_set_mlp", "seismic_mlp_forward", "seismic_mlp_train_step", "seismic_query_features"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    so, path = lib
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (seismic_[a-z_0-9]+)$", out, flags=re.M))
    assert set(_declared()) <= exported


def test_no_gpu_needed_for_error_paths(lib):
    import paper_2509_24815_gb300 as sz
    assert "sm_103a" in sz.seismic_version()
    # a NULL index is rejected on the host, before any device work
    rc = sz._lib.seismic_search(None, None, None, None, None, 0, None, None)
    assert rc == sz.EINVAL and "NULL" in sz.seismic_last_error()


def test_struct_layouts_match_header(tmp_path):
    """Compile a tiny C program against the header and compare sizes/offsets."""
    import paper_2509_24815_gb300 as sz
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "seismic.h"
int main(void){
 printf("%zu %zu %zu %zu\n", sizeof(seismic_csr), sizeof(seismic_build_params), sizeof(seismic_search_params),
        sizeof(seismic_index_info));
 printf("%zu %zu %zu\n", offsetof(seismic_build_params, alpha), offsetof(seismic_build_params, lambda_frac),
        offsetof(seismic_search_params, hash_slots));
 printf("%zu\n", offsetof(seismic_build_params, keep_block_summaries));
 return 0;}
"""
    tmp = str(tmp_path)
    c = os.path.join(tmp, "p.c")
    exe = os.path.join(tmp, "p")
    open(c, "w").write(prog)
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
    out = subprocess.check_output([exe], text=True).split()
    sizes = [int(x) for x in out]
    assert sizes[:4] == [ctypes.sizeof(sz._CSR), ctypes.sizeof(sz.BuildParams), ctypes.sizeof(sz.SearchParams),
                         ctypes.sizeof(sz.IndexInfo)]
    assert sizes[4:] == [sz.BuildParams.alpha.offset, sz.BuildParams.lambda_frac.offset,
                         sz.SearchParams.hash_slots.offset, sz.BuildParams.keep_block_summaries.offset]
