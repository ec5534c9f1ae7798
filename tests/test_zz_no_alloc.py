"""The allocation-free BF16 cost volume, tc_op_correlation_bf16_noalloc, for hosts that
cannot let the library allocate device memory (a memory pool that has reserved the device
up front, or a real-time loop that cannot afford cudaMalloc/cudaFree).  It runs the same
kernels as the allocating entry point tc_op_correlation(TC_BF16), so its output must equal
that entry point's bit for bit, on calls in a row that reuse the same fixed staging array,
and match the FP64 oracle within the BF16 correlation tolerance.

Kept in a file that pytest collects last.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import bf16_round, nchw_to_nhwc, nhwc_to_nchw, to_dev, to_np

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _features(n, h, w, c, seed):
    g = synth.rng(seed)
    return [bf16_round(g.normal(size=(n, c, h, w)).astype(np.float32)) for _ in range(2)]


def test_noalloc_correlation_matches_allocating_entry_point():
    import torch
    # three calls in a row on the shared staging array, with different shapes: two on the
    # tensor cores (c a multiple of 8), one on the CUDA cores (c = 20)
    for n, h, w, c, r, seed in [(2, 40, 56, 32, 4, 1), (1, 34, 60, 128, 3, 2), (3, 17, 29, 20, 2, 3)]:
        f1, f2 = _features(n, h, w, c, seed)
        d1, d2 = to_dev(nchw_to_nhwc(f1)), to_dev(nchw_to_nhwc(f2))
        out = torch.empty((n, h, w, (2 * r + 1) ** 2), device="cuda")
        got = tc.op_correlation_bf16_noalloc(d1, d2, r, out=out)
        torch.cuda.synchronize()
        used_tc = tc.op_last_used_tensor_cores()
        assert used_tc == (c % 8 == 0)
        want = tc.op_correlation(d1, d2, r, precision="bf16")
        torch.cuda.synchronize()
        assert tc.op_last_used_tensor_cores() == used_tc
        assert np.array_equal(to_np(got), to_np(want))
        # and the FP64 oracle on the same bf16 inputs, with the BF16 correlation tolerance
        for i in range(n):
            ref = oracle.correlation(f1[i], f2[i], r)
            np.testing.assert_allclose(nhwc_to_nchw(to_np(got)[i:i + 1])[0], ref, rtol=2 ** -8, atol=1e-4)


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    import torch
    n, h, w, c, r = 2, 256, 256, 64, 4     # 2 x 16 MiB of staged bf16 features > 16 MiB
    f = torch.zeros((n, h, w, c), device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.op_correlation_bf16_noalloc(f, f, r)
    assert e.value.status == tc.TC_ERR_INVALID_ARG and "staging" in str(e.value)
