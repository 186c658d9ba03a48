"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads,
exports every function include/gfopt.h declares, and its pure host functions work."""
import ctypes as C
import os
import re

import pytest

from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BLD.build()
    return B.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "gfopt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gf3?_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(B.EXPORTS) <= set(names)


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.gf_version()
    assert lib.gf_status_string(B.GF_ESINGULAR) == b"singular capacitance matrix"
    assert lib.gf_status_string(99) == b"unknown status"


def test_num_candidates_and_workspace(lib):
    g = W.brush_192().geoms[0]
    s = W.brush_192().spec
    gs, ss = B.geom_struct(g), B.spec_struct(s)
    assert lib.gf_num_candidates(C.byref(gs), C.byref(ss)) == 2 * 191 * 191
    s1 = B.spec_struct(W.plain_32().spec)
    g1 = B.geom_struct(W.plain_32().geoms[0])
    assert lib.gf_num_candidates(C.byref(g1), C.byref(s1)) == 1024
    ws = lib.gf_workspace_size(C.byref(gs), 1, B.GF_C128, C.byref(ss))
    n = g.N + 1
    assert ws >= 2 * n * 4 * 16          # C0 and S panels of p = 4 complex128 columns
    assert ws % 256 == 0
    assert lib.gf_workspace_size(C.byref(gs), 0, B.GF_C128, C.byref(ss)) == 0
    assert lib.gf_workspace_size(C.byref(gs), 1, 7, C.byref(ss)) == 0


def test_null_handle_is_rejected(lib):
    g = W.plain_32().geoms[0]
    p = B.problem_struct(g, 16, g.n + 1, 16, 16)
    assert lib.gf_fill_g0(None, C.byref(p), B.GF_C128, None, 0, None) == B.GF_EINVAL
    assert lib.gf_extract_bands(None, C.byref(p), B.GF_C128, None) == B.GF_EINVAL


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.gf_create(C.byref(h), 0)
    assert st == B.GF_ECUDA
    assert len(lib.gf_last_error(None)) > 0


def test_batch_host_checks(lib):
    assert lib.gf_batch_table_size(0) == 0
    assert lib.gf_batch_table_size(B.BATCH_MAX + 1) == 0
    one = lib.gf_batch_table_size(1)
    assert one > 0 and one % 256 == 0
    assert lib.gf_batch_table_size(B.BATCH_MAX) >= B.BATCH_MAX * one // 256 * 0 + one
    assert lib.gf_batch_step(None, None) == B.GF_EINVAL
    assert lib.gf_batch_set_schedule(None, 0) == B.GF_EINVAL
    lib.gf_batch_destroy(None)


def test_workspace_sizes_cover_the_tensor_core_operand_blocks(lib):
    """The complex64 tensor-core update's split-FP16 operand blocks (A: 8 KB per 128-row tile and
    16-deep K chunk; B: 16 KB per pair of 64-column tiles and K chunk, K = 2 P with P = p_max
    rounded to 16) fit in the workspace, for the 2-D top-k workload and the 3-D lens; the refresh
    workspace holds the GMRES basis and the partial sums of its reductions."""
    def blocks(n, pmax):
        P = (pmax + 15) // 16 * 16
        nkc = 2 * P // 16
        nrt, nct = (n + 127) // 128, (2 * n + 127) // 128
        ncp = (nct + 1) // 2
        return nrt * nkc * 8192 + ncp * nkc * 16384
    wl = W.brush_320_topk()
    g, s = wl.geoms[0], wl.spec
    ws = lib.gf_workspace_size(C.byref(B.geom_struct(g)), 1, B.GF_C64, C.byref(B.spec_struct(s)))
    assert ws >= blocks(g.N + 1, 4 * s.k) and ws % 256 == 0
    k1 = W.CandidateSpec(s.kind, s.dir_mask, 1, s.excl_radius)
    assert lib.gf_workspace_size(C.byref(B.geom_struct(g)), 1, B.GF_C64, C.byref(B.spec_struct(k1))) < ws
    ml = W.metalens_3d()
    g3 = B.geom3d_struct(ml.geoms[0])
    n3 = lib.gf3_num_unknowns(C.byref(g3))
    assert n3 == 3 * (120 * 120 * 4 + 1)
    ws3 = lib.gf3_workspace_size(C.byref(g3), B.GF_C64, C.byref(B.spec_struct(ml.spec)))
    assert ws3 >= blocks(n3, 12 * 4) and ws3 % 256 == 0
    gr = B.geom_struct(g)
    rw = lib.gf_refresh_workspace_size(C.byref(gr), 30)
    assert rw >= 16 * (g.N + 1) * 31 + 16 * 31 * 128
    assert lib.gf_refresh_workspace_size(C.byref(gr), 0) == 0
    assert lib.gf_refresh_workspace_size(C.byref(gr), 201) == 0


def test_update_algo_settings(lib):
    assert (B.GF_UPDATE_TC, B.GF_UPDATE_DFMA, B.GF_UPDATE_TENSOR) == (0, 1, 2)
    hdr = open(os.path.join(ROOT, "include", "gfopt.h")).read()
    for name, v in (("GF_UPDATE_TC", 0), ("GF_UPDATE_DFMA", 1), ("GF_UPDATE_TENSOR", 2)):
        assert re.search(r"#define\s+%s\s+%d\b" % (name, v), hdr), name
    assert lib.gf_set_update_algo(None, B.GF_UPDATE_TENSOR) == B.GF_EINVAL
