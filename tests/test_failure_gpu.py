"""Failure detection on the GPU without a fault: the bounded device-side
wait that the tensor-core residual of the mixed path uses gives up after its
limit and the host reads DF_ERR_TIMEOUT; the device stays usable.

The wait under test is the mbarrier poll that follows each batch of tcgen05
MMAs (a completion that never arrives makes the kernel flag a timeout and
return instead of spinning); here a barrier that nothing completes stands in
for the missing completion.  Nothing traps, faults or hangs.
"""
import numpy as np
import pytest

from oracle import df_oracle as O
from paper_1507_00895_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_00895_gb300 import build
    build.build_lib()
    from paper_1507_00895_gb300 import df as dfm
    return dfm


def test_wait_that_nothing_completes_times_out(df):
    lib = df.load()
    assert lib.df_selftest_wait(0, 2000) == df.DF_ERR_TIMEOUT
    assert lib.df_selftest_wait(0, 1) == df.DF_ERR_TIMEOUT


def test_completed_wait_passes(df):
    lib = df.load()
    assert lib.df_selftest_wait(1, 2000) == df.DF_OK


def test_device_usable_after_a_timeout(df):
    lib = df.load()
    assert lib.df_selftest_wait(0, 2000) == df.DF_ERR_TIMEOUT
    # a mixed-precision pass at n_w = 64 (the tcgen05 residual and its waits) still agrees with the oracle
    w = I.workload("square32_tp", nk=4, n_w=64, m_max=1)
    ref = O.run_workload(w, n_iter=1)
    with df.DualFermion.from_workload(w, precision=df.DF_FP32_IR) as d:
        it, _, _ = d.iterate(1)
        sig = d.get_sigma()
    assert it == 1
    err = np.max(np.abs(sig - ref.sigma)) / np.max(np.abs(ref.sigma))
    assert err < 1e-8, err
