"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/blast.h declares; argument validation runs on the host."""
import ctypes
import os
import re

import pytest

from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import build as bld
from paper_2410_03632_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(blast_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    so = bld.build()
    L = ctypes.CDLL(so)
    syms = declared_symbols()
    assert "blast_cl" in syms and "blast_precompute_basis" in syms
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_status_strings_and_pairs():
    assert bl.blast_status_str(bl.BLAST_EINVAL) == "invalid argument"
    assert bl.blast_npairs(5, 5) == 55 and bl.blast_npairs(10, 10) == 210
    assert bl.blast_npairs(0, 3) == 6 and bl.blast_npairs(2, 0) == 3


@pytest.mark.parametrize("field,value", [("n_chi", 3), ("n_R", 7), ("R_min", 1.2), ("n_cheb", 1),
                                         ("n_kquad", 100), ("k_map", 3), ("max_clust", 99)])
def test_plan_rejects_bad_description_before_touching_a_device(field, value):
    spec = synth.plan_spec("tiny")
    setattr(spec, field, value)
    with pytest.raises(bl.BlastError) as ei:
        bl.Plan(spec)
    assert ei.value.status == bl.BLAST_EINVAL


def test_plan_rejects_unsorted_ells():
    spec = synth.plan_spec("tiny")
    spec.ells = spec.ells[::-1].copy()
    with pytest.raises(bl.BlastError):
        bl.Plan(spec)
    spec.ells = spec.ells * 0 + 1
    with pytest.raises(bl.BlastError):
        bl.Plan(spec)


def test_server_entry_points_reject_bad_arguments_on_the_host():
    L = bl.lib()
    out = ctypes.c_void_p()
    t = ctypes.c_uint64()
    d = ctypes.c_int()
    req = bl.blast_request()
    # no plans, no budget, no slots, no output handle: refused before any device work
    assert L.blast_server_create(None, 1, 1 << 20, 4, ctypes.byref(out)) == bl.BLAST_EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    assert L.blast_server_create(arr, 1, 1 << 20, 4, ctypes.byref(out)) == bl.BLAST_EINVAL
    assert L.blast_server_create(arr, 0, 1 << 20, 4, ctypes.byref(out)) == bl.BLAST_EINVAL
    assert L.blast_submit(None, 0, ctypes.byref(req), bl.BLAST_FP64, ctypes.byref(t)) == bl.BLAST_EINVAL
    assert L.blast_poll(None, 1, None, ctypes.byref(d), 0) == bl.BLAST_EINVAL
    assert L.blast_server_destroy(None) == bl.BLAST_EINVAL
    assert L.blast_cl_batch(None, 1, ctypes.byref(req), bl.BLAST_FP64, None, 0, None) == bl.BLAST_EINVAL
