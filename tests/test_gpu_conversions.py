"""The library's FP64 <-> FP32 conversions (integer rewrites of the IEEE 754
fields, used by the apply's gathers of r and its FP32 scatter-add sums) agree bit
for bit with the hardware conversions on random bit patterns, and an FP32 apply
that uses them still matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, oracle_for, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("seed", [1, 0x5DEECE66D, 2 ** 63 + 12345])
def test_conversions_match_hardware_bitwise(seed):
    from paper_2304_04876_b300 import gdsw
    assert gdsw.check_conversions(seed, 1 << 24) == (0, 0)


def test_conversion_check_counts_nothing_for_empty_input():
    from paper_2304_04876_b300 import gdsw
    assert gdsw.check_conversions(7, 0) == (0, 0)


def test_fp32_apply_with_library_conversions_matches_oracle():
    prob = P.poisson_problem(12, 4)
    M = oracle_for(prob, local="ic0", trsv="levelsched")
    h = gpu_handle(prob, local_solver="ic0", precision="fp32")
    # entries across many binades, exact zeros and FP32-subnormal magnitudes
    rng = np.random.default_rng(3)
    r = rng.uniform(-1, 1, prob.A.n) * np.exp2(rng.integers(-40, 40, prob.A.n))
    r[::17] = 0.0
    r[5::97] = 1e-41
    z = gpu_apply(h, r)
    assert relerr(z, M.apply(r)) <= 2e-5
    h.close()
