"""gf_fill_g0_static -- the fill for callers that cannot allocate a workspace -- checked
through the C ABI against gf_fill_g0 on consecutive calls (different grid sizes, so the
shared table is reused with other contents; narrow grids take the blocked fill, grids wider than
2048 pixels the row expansion), plus its size limit.  Kept in a file that is
collected last."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W


def _buffers(g, dtype):
    n = g.N + 1
    ldg = n + (n & 1)
    tdt = torch.complex128 if dtype == B.GF_C128 else torch.complex64
    G = torch.empty((n, ldg), dtype=tdt, device="cuda")
    E = torch.empty(n, dtype=torch.complex128, device="cuda")
    bands = torch.empty(B.GF_NBANDS * g.N, dtype=torch.complex128, device="cuda")
    return G, E, bands, B.problem_struct(g, G, ldg, E, bands)


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_static_fill_matches_workspace_fill_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    lib = B.load()
    h = B.Handle(0)
    stream = torch.cuda.current_stream()
    # the last two grids are wider than the blocked fill handles (nx > 2048), so the static
    # table is read by the row-expansion kernel as well
    for nx, ny, dtype in [(41, 29, B.GF_C128), (23, 17, B.GF_C128), (30, 20, B.GF_C64),
                          (2100, 1, B.GF_C128), (2100, 1, B.GF_C64)]:
        g = W.small(nx, ny).geoms[0]
        Gr, Er, br, pr = _buffers(g, dtype)
        Gs, Es, bs, ps = _buffers(g, dtype)
        ws_bytes = h.gf_workspace_size(g, 1, dtype, W.CandidateSpec())
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        h.gf_fill_g0(pr, dtype, ws, ws_bytes, stream)
        st = lib.gf_fill_g0_static(h.h, C.byref(ps), dtype, C.c_void_p(stream.cuda_stream))
        assert st == B.GF_OK, lib.gf_last_error(h.h)
        torch.cuda.synchronize()
        tol = 1e-12 if dtype == B.GF_C128 else 1e-6
        assert _rel(Gs[:, :g.N + 1], Gr[:, :g.N + 1]) <= tol
        assert _rel(Es, Er) <= 1e-12
        assert _rel(bs, br) <= tol
        assert torch.count_nonzero(Gs[:, g.N + 1:]).item() == 0


def test_static_fill_rejects_grids_beyond_its_table():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    lib = B.load()
    h = B.Handle(0)
    g = W.Geometry(512, 512, 0.05, 1.0, 12.8, 30.0)       # N = 262144 > 131072
    p = B.problem_struct(g, 256, g.N + 1 + ((g.N + 1) & 1), 256, 256)   # never dereferenced
    st = lib.gf_fill_g0_static(h.h, C.byref(p), B.GF_C128, None)
    assert st == B.GF_EINVAL
    assert b"131072" in lib.gf_last_error(h.h)
