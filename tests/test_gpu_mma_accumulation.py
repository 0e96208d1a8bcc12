"""The tensor cores' FP32 accumulation, measured through the library's
tcgen05 GEMM (gcamb_probe_mma: bf16 operands, kind::f16, FP32 in TMEM).

This is the behaviour the batched path's chain records are built around:
within one MMA the 16 products and the accumulator are aligned to the
largest of them, each keeps its bits down to a quarter ulp of that largest
term, and the sum is truncated (towards zero) to 24 bits.  So every
accumulate step can lose up to a few ulp of the running sum, always
towards zero: a long same-sign sum comes out low, and the loss scales with
the accumulator's magnitude (splitting a sum over several accumulators cuts
it).  The paper does not depend on this; the checks pin the arithmetic the
split-precision error analysis uses."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def mma(A, B):
    C = gcamb.probe_mma(torch.as_tensor(A, dtype=torch.float32, device="cuda"),
                        torch.as_tensor(B, dtype=torch.float32, device="cuda")).cpu().numpy()
    gcamb.sync()
    return C.astype(np.float64)


def test_products_below_a_quarter_ulp_of_the_accumulator_vanish():
    K = 1024
    ulp = 2.0 ** -23
    A = np.ones((128, K))
    for frac, expect_ulp in ((0.125, 0.0), (0.25, 255.0)):
        B = np.full((128, K), frac * ulp)
        B[:, 0] = 1.0
        C = mma(A, B)
        exact = 1.0 + (K - 1) * frac * ulp
        # 1023 terms of an eighth of an ulp are all lost; of a quarter ulp all
        # kept but the first MMA's sum (1 + 15/4 ulp) truncated to 1 + 3 ulp
        assert np.all(C == 1.0 + expect_ulp * ulp), (frac, np.unique(C))
        assert np.all(C < exact)


def test_one_mma_keeps_a_quarter_ulp_of_its_largest_term():
    K = 64
    ulp = 2.0 ** -23
    A = np.zeros((128, K))
    A[:, :16] = 1.0
    B = np.zeros((128, K))
    B[:, 0] = 1.0
    B[:, 1:16] = 0.375 * ulp  # 0.011 in units of ulp(1): counts as 0.25 ulp
    C = mma(A, B)
    assert np.all(C == 1.0 + 3.0 * ulp)  # 15 x 0.25 = 3.75 ulp, truncated to 3


def test_long_same_sign_sums_come_out_low():
    rng = np.random.default_rng(5)
    K = 1024
    to_bf16 = lambda x: torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    A = to_bf16(rng.uniform(0.5, 2.0, (128, K)))
    B = to_bf16(rng.uniform(0.5, 2.0, (128, K)))
    C = mma(A, B)
    exact = A @ B.T
    rel = C / exact - 1
    assert np.all(rel <= 0)                       # never above the exact sum
    assert -2e-6 < rel.mean() < -3e-7            # measured -1.05e-6 on GB300
    # split over four accumulators (four GEMMs over quarters of K, summed in
    # FP64): each holds a quarter of the sum, and the loss shrinks with it
    parts = sum(mma(A[:, q:q + 256], B[:, q:q + 256]) for q in range(0, K, 256))
    rel4 = parts / exact - 1
    assert rel4.mean() > 0.5 * rel.mean()
