"""Logical-error-rate statistics (Sec. 6.1): per-round conversion,
Clopper-Pearson intervals and the 2-sigma agreement test."""
import pytest
from scipy import stats as st

from paper_2607_27644_b300.stats import agree_within, binomial_sigma, clopper_pearson, per_qubit_round, per_round


def test_per_round_inverts_the_block_rate():
    for q in (1e-9, 3e-6, 0.01, 0.2):
        for T in (1, 10, 18):
            assert per_round(1 - (1 - q) ** T, T) == pytest.approx(q, rel=1e-9)
    assert per_qubit_round(0.01, 10, 32) == per_round(0.01, 320)


def test_paper_conversion_of_zsz_lp_160():
    """Table 1: ZSZ-LP-160 at p = 0.1% has LER 2.0e-8 per qubit-round over
    d = 10 rounds and k = 32, i.e. a raw block LER of about 6.4e-6."""
    assert per_qubit_round(6.4e-6, 10, 32) == pytest.approx(2.0e-8, rel=0.01)


@pytest.mark.parametrize("k,n", [(0, 100), (1, 100), (13, 1000), (500, 1000), (1000, 1000), (7, 10 ** 6)])
def test_clopper_pearson_is_the_exact_binomial_interval(k, n):
    lo, hi = clopper_pearson(k, n)
    ci = st.binomtest(k, n).proportion_ci(confidence_level=0.95, method="exact")
    assert lo == pytest.approx(ci.low, abs=1e-12) and hi == pytest.approx(ci.high, abs=1e-12)
    if k == 0:
        assert lo == 0.0 and hi == pytest.approx(1 - 0.025 ** (1 / n), rel=1e-9)
    if k == n:
        assert hi == 1.0 and lo == pytest.approx(0.025 ** (1 / n), rel=1e-9)


def test_two_sigma_agreement():
    assert agree_within(10, 10 ** 6, 10, 10 ** 6)
    assert agree_within(10, 10 ** 6, 6, 10 ** 6) and agree_within(6, 10 ** 6, 10, 10 ** 6)
    assert not agree_within(100, 10 ** 6, 10, 10 ** 6)
    assert binomial_sigma(0, 100) > 0                    # zero failures still carry an error bar
