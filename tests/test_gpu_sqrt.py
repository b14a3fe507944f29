"""The FP64 step's Newton square root (wave speeds of Section 2) against
CUDA's correctly rounded sqrt, and the FP64 wall kernel's division by 3
(adiabatic walls) against CUDA's correctly rounded division, through the
C-ABI self-checks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2006_02602_gb300 as m
    return m


def test_newton_sqrt_within_one_ulp_over_the_normal_range(m):
    rng = np.random.default_rng(7)
    # log-uniform over the whole normal range, and dense where the rates take
    # it: V_d^2 + 4 beta^2 with beta^2 >= kappa u_ref^2
    x = np.concatenate([10.0 ** rng.uniform(-307.0, 307.0, 1 << 20),
                        10.0 ** rng.uniform(-2.0, 8.0, 1 << 20),
                        np.array([np.finfo(np.float64).tiny, np.finfo(np.float64).max, 1.0, 4.0, 2.0])])
    max_rel, n_diff = m.cavity_check_sqrt(x)
    assert max_rel <= 2.0 ** -52
    assert n_diff <= 0.01 * x.size


def test_check_rejects_values_outside_the_range(m):
    for bad in ([0.0], [-1.0], [np.inf], [np.nan], [1e-310]):
        with pytest.raises(m.CavityError):
            m.cavity_check_sqrt(np.array(bad))


def test_division_by_three_is_correctly_rounded(m):
    rng = np.random.default_rng(11)
    # random significands and signs over the normal range, dense near the
    # temperatures the walls see, and exact multiples of 3 and powers of two
    bits = rng.integers(0, 1 << 52, 1 << 20, dtype=np.int64) | (rng.integers(1, 2046, 1 << 20, dtype=np.int64) << 52)
    wide = bits.view(np.float64) * rng.choice([-1.0, 1.0], bits.size)
    wide = wide[np.abs(wide) >= 4 * np.finfo(np.float64).tiny]
    x = np.concatenate([wide, rng.uniform(-2.0, 2.0, 1 << 20), 3.0 * np.arange(1, 4097), 2.0 ** np.arange(-1000, 1000)])
    assert m.cavity_check_div3(x) == 0


def test_div3_check_rejects_values_outside_the_range(m):
    for bad in ([0.0], [np.inf], [np.nan], [1e-310]):
        with pytest.raises(m.CavityError):
            m.cavity_check_div3(np.array(bad))
