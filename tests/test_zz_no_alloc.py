"""The allocation-free residual entry point against the existing block SpMV.

cptr_residual_noalloc keeps its reduction scratch in a fixed device array of
the library; its r = b - A x must match b - cptr_spmv(x) and its norm the
norm of that vector, on consecutive calls that reuse the same scratch.  This
file is collected last so that it also runs after every other test.
"""
import ctypes

import numpy as np
import pytest

from synth import config_system, random_bsr


def _lib():
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def test_noalloc_rejects_sizes_beyond_scratch():
    """Host-side check: too many cells is refused before any device work."""
    P = _lib()
    lib = P._lib.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    st = lib.cptr_residual_noalloc(P.NOALLOC_MAX_CELLS + 1, fake, fake, fake, fake, fake, fake,
                                   fake, None)
    assert st == P._lib.ERR_INVALID
    assert lib.cptr_residual_noalloc(0, fake, fake, fake, fake, fake, fake, fake, None) == \
        P._lib.ERR_INVALID
    with pytest.raises(P.CPTRError, match="exceeds the fixed scratch"):
        P.cptr_residual_noalloc(P.NOALLOC_MAX_CELLS + 1, 256, 256, 256, 256, 256, 256, 256)


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.gpu
def test_noalloc_residual_matches_spmv_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    dev = torch.device("cuda:0")
    # a 64x64x32 reservoir grid (2048 thread blocks, most of the scratch), then
    # a small ragged system with empty rows: the second call reuses the array
    systems = [config_system("c2"), random_bsr(203, avg_offdiag=5, seed=21, empty_rows=0.2)]
    rng = np.random.default_rng(7)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for s in systems:
        rp = torch.from_numpy(s.rowptr).to(dev)
        ci = torch.from_numpy(s.col).to(dev)
        v = torch.from_numpy(np.ascontiguousarray(s.vals)).to(dev)
        outs = []
        for call in range(2):
            x = torch.from_numpy(rng.normal(size=4 * s.n_cells)).to(dev)
            b = torch.from_numpy(rng.normal(size=4 * s.n_cells)).to(dev)
            r = torch.full_like(b, float("nan"))
            rn = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            P.cptr_residual_noalloc(s.n_cells, rp, ci, v, x, b, r, rn, stream)
            torch.cuda.synchronize()
            outs.append((x.cpu().numpy(), b.cpu().numpy(), r.cpu().numpy(), float(rn.item())))
        # the existing entry point on the same inputs
        with P.Solver.from_system(s) as g:
            for x, b, r, rn in outs:
                xd = torch.from_numpy(x).to(dev)
                yd = torch.zeros_like(xd)
                P.cptr_spmv(g.h, xd, yd)
                torch.cuda.synchronize()
                want = b - yd.cpu().numpy()
                assert np.isfinite(r).all()
                assert _relerr(r, want) < 1e-14
                assert abs(rn - np.linalg.norm(want)) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.gpu
def test_noalloc_residual_inside_a_captured_graph():
    """Callers inside a stream capture are who this entry point is for: one call
    captured into a CUDA graph (after an eager first call, which looks up the
    scratch address) and the graph replayed with new x and b written into the
    same buffers gives b - A x and its norm each time (the completion ticket
    is cleared by the captured memset on every replay)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    dev = torch.device("cuda:0")
    s = config_system("c1")
    rng = np.random.default_rng(11)
    rp = torch.from_numpy(s.rowptr).to(dev)
    ci = torch.from_numpy(s.col).to(dev)
    v = torch.from_numpy(np.ascontiguousarray(s.vals)).to(dev)
    n4 = 4 * s.n_cells
    x = torch.zeros(n4, dtype=torch.float64, device=dev)
    b = torch.zeros_like(x)
    r = torch.zeros_like(x)
    rn = torch.zeros(1, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        P.cptr_residual_noalloc(s.n_cells, rp, ci, v, x, b, r, rn, side.cuda_stream)  # eager
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        P.cptr_residual_noalloc(s.n_cells, rp, ci, v, x, b, r, rn,
                                torch.cuda.current_stream(dev).cuda_stream)
    with P.Solver.from_system(s) as g:
        for rep in range(2):
            xh = rng.normal(size=n4)
            bh = rng.normal(size=n4)
            x.copy_(torch.from_numpy(xh))
            b.copy_(torch.from_numpy(bh))
            r.fill_(float("nan"))
            rn.fill_(float("nan"))
            graph.replay()
            torch.cuda.synchronize()
            yd = torch.zeros_like(x)
            P.cptr_spmv(g.h, x, yd)
            torch.cuda.synchronize()
            want = bh - yd.cpu().numpy()
            assert _relerr(r.cpu().numpy(), want) < 1e-14
            assert abs(float(rn.item()) - np.linalg.norm(want)) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.gpu
def test_noalloc_refuses_misaligned_x():
    """x is read two doubles at a time: an address off the 16-byte grid is
    refused before anything runs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = _lib()
    dev = torch.device("cuda:0")
    s = config_system("c1")
    n4 = 4 * s.n_cells
    buf = torch.zeros(n4 + 1, dtype=torch.float64, device=dev)
    rp = torch.from_numpy(s.rowptr).to(dev)
    ci = torch.from_numpy(s.col).to(dev)
    v = torch.from_numpy(np.ascontiguousarray(s.vals)).to(dev)
    b = torch.zeros(n4, dtype=torch.float64, device=dev)
    r = torch.zeros_like(b)
    rn = torch.zeros(1, dtype=torch.float64, device=dev)
    lib = P._lib.load()
    st = lib.cptr_residual_noalloc(s.n_cells, rp.data_ptr(), ci.data_ptr(), v.data_ptr(),
                                   buf.data_ptr() + 8, b.data_ptr(), r.data_ptr(),
                                   rn.data_ptr(), None)
    assert st == P._lib.ERR_INVALID
