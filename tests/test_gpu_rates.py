"""The measured FMA rates (the compute roof beside the HBM roof of the FP64
kernels) and the flop model of the profiled kernels.

cptr_fma_rate checks every thread's chain result against its closed form
before it returns a rate, so a rate means that every counted FMA ran.  FP64
runs far below FP32 on this part (about 1.25 TFLOP/s nominal); the bounds here
are loose, the number itself is reported by the benchmark.
"""
import numpy as np
import pytest

from synth import cartesian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11892_gb300 import build
    build.build()
    import paper_2308_11892_gb300 as P
    return P


def test_fma_rates(P):
    import torch
    f64 = P.cptr_fma_rate(True, 2048, reps=3)
    f32 = P.cptr_fma_rate(False, 1 << 15, reps=3)
    assert 0.1 < f64 < 5.0
    assert f32 > 4.0 * f64
    s = torch.cuda.Stream()
    assert P.cptr_fma_rate(True, 512, reps=2, stream=s.cuda_stream) > 0.1
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kernel_flop_model(P, precision):
    s = cartesian(9, 8, 5, pe=1.0, seed=61)
    kw = {} if precision == "fp64" else {"precision": P.MIXED}
    with P.Solver.from_system(s, restart=20, **kw).setup() as g:
        nnzb = len(s.col)
        fl, f64 = P.cptr_kernel_flops(g.h, P.KERNEL_SPMV)
        assert f64 and fl == 32.0 * nnzb
        # before any solve the multi-dot is profiled at column restart / 2
        fl, f64 = P.cptr_kernel_flops(g.h, P.KERNEL_MDOT)
        assert f64 and fl == 8.0 * s.n_cells * (20 // 2 + 1)
        for k in (P.KERNEL_ILU_FWD, P.KERNEL_ILU_BWD, P.KERNEL_VC_PRE0, P.KERNEL_CORRECTION):
            fl, f64 = P.cptr_kernel_flops(g.h, k)
            assert fl > 0 and f64 == (precision == "fp64")
        # the ILU(0) factors have the matrix's pattern: blocks of L + U = nnzb - N
        lf, _ = P.cptr_kernel_flops(g.h, P.KERNEL_ILU_FWD)
        lb, _ = P.cptr_kernel_flops(g.h, P.KERNEL_ILU_BWD)
        assert lf / 32.0 + (lb - 36.0 * s.n_cells) / 32.0 == nnzb - s.n_cells
        xg, info = g.solve(s.rhs)
        fl, _ = P.cptr_kernel_flops(g.h, P.KERNEL_MDOT)
        assert fl == 8.0 * s.n_cells * (min(info["iters"], 20) // 2 + 1)
    with P.Solver.from_system(s) as g:  # not set up
        with pytest.raises(P.CPTRError):
            P.cptr_kernel_flops(g.h, P.KERNEL_SPMV)
