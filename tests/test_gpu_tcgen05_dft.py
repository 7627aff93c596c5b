"""Batched 1-D DFTs on the tcgen05 tensor cores (ptycho_dft_rows_tc): the
§2.2 precision option (split lower-precision products on the tensor cores)
for the DFTs of §3, against the oracle's own dense DFT matrix, for every
window size, both directions, every split mode, and a ragged number of rows
(several 128-row tiles plus a tail)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, rel_l2
from paper_2505_14372_b300 import PtychoError
from paper_2505_14372_b300.api import dft_rows_tc, dft_rows_tc_check

pytestmark = pytest.mark.gpu

# relative L2 bounds of the split modes: tf32 keeps 11 significant bits, so
# hi + lo carries ~22 (2^-22 = 2.4e-7 per operand, the dropped lo*lo as much)
# and the error is dominated by the accumulation over 2N = 128..512 terms
# inside the MMA (sqrt(2N) 2^-24 = 1.3e-6 for round-to-nearest FP32 at 512;
# measured 2.7e-6 at 2N = 384, so the tensor core's accumulation is a little
# coarser): 1e-5; bf16 keeps 8 bits, hi + lo ~16 (2^-16 = 1.5e-5): 6e-5; one
# tf32 product 2^-11 = 4.9e-4: 2e-3
TOL = {"tf32x3": 1e-5, "bf16x3": 6e-5, "tf32": 2e-3}


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x3", "tf32"])
@pytest.mark.parametrize("N", [64, 128, 192, 256])
def test_dft_rows_tcgen05_against_oracle(N, mode):
    rng = np.random.default_rng(N + len(mode))
    rows = 300
    x = (rng.standard_normal((rows, N)) + 1j * rng.standard_normal((rows, N))).astype(np.complex64)
    F = orc.dft_matrix(N)                      # F[k][n] = exp(-2 pi i k n / N)
    xd = dev(x)
    y = host(dft_rows_tc(xd, mode))
    y2 = host(dft_rows_tc(xd, mode, inverse=True))
    torch.cuda.synchronize()
    dft_rows_tc_check()
    ref = x.astype(np.complex128) @ F
    ref_inv = x.astype(np.complex128) @ np.conj(F)
    assert rel_l2(y, ref) < TOL[mode], rel_l2(y, ref)
    assert rel_l2(y2, ref_inv) < TOL[mode], rel_l2(y2, ref_inv)
    # the same rows alone give the same values (no dependence on the tile)
    one = host(dft_rows_tc(xd[rows - 1:], mode))
    assert np.array_equal(one[0], y[rows - 1])


def test_dft_rows_tcgen05_arguments():
    x = torch.zeros((4, 100), dtype=torch.complex64, device="cuda")
    with pytest.raises(PtychoError):
        dft_rows_tc(x)                          # N = 100 has no table
    y = torch.zeros((4, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(PtychoError):
        dft_rows_tc(y, out=y)                   # in place is refused
    assert dft_rows_tc(torch.zeros((0, 64), dtype=torch.complex64, device="cuda")).shape == (0, 64)
