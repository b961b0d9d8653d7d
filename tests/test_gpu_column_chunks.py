"""The column solve stages its inputs through shared memory in chunks of 4,
6 or 8 levels (the autotuner's candidates).  The chunk length changes how the
data moves, not what is computed: every chunk length gives the same step bit
for bit in FP64 and in the double-word mixed mode, and to rounding in the
mixed mode with the FP64 column solve, here on 45 levels, which none of them
divides (a ragged last chunk in the forward sweep and the back-substitution)."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f64col"])
def test_column_chunk_lengths_agree_bitwise(built_lib, cuda, precision):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(3, 45, 900.0, rayleigh=0.05, seed=4)
    prec = {"fp64": P.ICON_PREC_FP64, "mixed": P.ICON_PREC_MIXED, "mixed_f64col": P.ICON_PREC_MIXED_F64COL}[precision]
    g = P.Grid(grid, radius=op.radius)
    outs = {}
    for kc in (4, 6, 8):
        d = P.Dycore(g, z, gpu_params(op, rayleigh_coeff=0.05, precision=prec, autotune=0, column_chunk=kc))
        assert d.launch_config().endswith("column_chunk=%d" % kc)
        t = to_torch(st, cuda)
        for _ in range(2):
            d.step(t)
        d.synchronize()
        outs[kc] = to_numpy(t)
        d.close()
    for kc in (6, 8):
        for k in outs[4]:
            if precision == "mixed_f64col":
                # FP64 arithmetic on FP32 inputs: the instantiations for the
                # three chunk lengths differ in the last bit at a few points (the
                # compiler's multiply-add contraction); where such a bit flips the
                # rounding of an FP32 mirror, the FP32 stencils carry a difference
                # of FP32 roundings (measured 5e-13 of max |vn| and 5e-9 of max
                # |w| after two steps), below the FP32 rounding unit and far
                # below the mode's 2e-5 error gate against the FP64 oracle
                scale = np.max(np.abs(outs[4][k]))
                assert np.max(np.abs(outs[kc][k] - outs[4][k])) <= 1e-6 * scale, (kc, k)
            else:
                assert np.array_equal(outs[kc][k].view(np.uint64), outs[4][k].view(np.uint64)), (kc, k)
    assert all(np.all(np.isfinite(v)) for v in outs[4].values())


def test_column_chunk_other_lengths_rejected(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    with pytest.raises(P.IconError):
        P.Dycore(g, z, gpu_params(op, autotune=0, column_chunk=5))
