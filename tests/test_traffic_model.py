"""The schedule's traffic against the paper's I/O lower bounds recast for one
GB300 (Sec. 6.1, 6.2): 152 SMs, M = shared memory + TMEM of one SM
(484 KB = 123,904 FP32 words), words of 4 bytes.  Summed over the SMs the
bound is P x Q_P, independent of P at leading order.  At N = 32768 the
mixed LU (FP16, V = 2048) loads into the SMs less than 2x the bound and
moves less than the bound through HBM; so does the BF16 Cholesky; the split
BF16 Cholesky's three operand segments put its loads above 2x."""
import math

import pytest

import oracle
from tests import traffic_model as tm

P = 152
M = 484 * 1024 / 4
N = 32768


def _bound(kind, n):
    """P x the per-SM bound, in bytes."""
    f = oracle.io_lower_bound_lu if kind == "lu" else oracle.io_lower_bound_chol
    return 4.0 * P * f(float(n), float(P), M)


def test_bound_values():
    # leading terms 2N^3/(3 sqrt M) and N^3/(3 sqrt M) words, sqrt(M) = 352,
    # plus the lower-order N(N-1)/2 (LU) and N^2/2 + N (Cholesky) words
    assert math.sqrt(M) == 352.0
    assert _bound("lu", N) == pytest.approx(4 * (2 * N ** 3 / (3 * 352) + N * (N - 1) / 2), rel=1e-4)
    assert _bound("chol", N) == pytest.approx(4 * (N ** 3 / (3 * 352) + N ** 2 / 2 + N), rel=1e-4)
    assert _bound("lu", N) / 1e9 == pytest.approx(268.7, abs=0.1)
    assert _bound("chol", N) / 1e9 == pytest.approx(135.4, abs=0.1)


def test_lower_tile_count_brute_force():
    for m in (1, 127, 128, 129, 700, 1000):
        tiles = sum(1 for i in range(-(-m // tm.BM)) for j in range(-(-m // tm.BN))
                    if j * tm.BN <= i * tm.BM + tm.BM - 1)
        loads, _ = tm.schur(m, m, 64, lower=True)
        assert loads == tiles * ((tm.BM + tm.BN) * 64 * 2 + tm.BM * tm.BN * 8)


def test_update_bytes_match_flops_intensity():
    # one full 128 x 256 tile of depth K: (128 + 256) K 2 bytes of operands
    loads, hbm = tm.schur(128, 256, 1024)
    assert loads == 384 * 1024 * 2 + 128 * 256 * 8
    assert hbm == 128 * 256 * 8 + 384 * 1024 * 2


@pytest.mark.parametrize("name,parts,kind,loads_x,hbm_x", [
    ("LU FP16 V=2048", lambda: tm.mixed_lu(N, 2048, S=1), "lu", 1.41, 0.40),
    ("Cholesky split BF16 V=1024", lambda: tm.mixed_chol(N, 1024, S=3), "chol", 3.68, 0.64),
    ("Cholesky BF16 V=1024", lambda: tm.mixed_chol(N, 1024, S=1), "chol", 1.56, 0.54),
])
def test_traffic_against_bound(name, parts, kind, loads_x, hbm_x):
    loads, hbm = tm.totals(parts())
    b = _bound(kind, N)
    assert loads / b == pytest.approx(loads_x, abs=0.01), name
    assert hbm / b == pytest.approx(hbm_x, abs=0.01), name
    assert hbm < b
    if loads_x < 2:
        assert loads < 2 * b


def test_hbm_against_the_l2_level_bound():
    """The same bound with the whole GPU as one processor whose fast memory
    is the 129 MB L2 (P = 1): the HBM side's sharper yardstick."""
    ML2 = 129e6 / 4
    for parts, f, x in ((tm.mixed_lu(N, 2048, S=1), oracle.io_lower_bound_lu, 5.77),
                        (tm.mixed_chol(N, 1024, S=3), oracle.io_lower_bound_chol, 8.36),
                        (tm.mixed_chol(N, 1024, S=1), oracle.io_lower_bound_chol, 6.97)):
        b = 4.0 * f(float(N), 1.0, ML2)
        _, hbm = tm.totals(parts)
        assert hbm / b == pytest.approx(x, abs=0.01)
