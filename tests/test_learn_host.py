"""Host-side logic of the learned-correction driver (learn.py) that needs no
GPU: the golden-section search of the filter calibration, the choice of the
node a snapshot drifts from, and the filter row of a scale factor (against the
oracle's own implementation)."""
import numpy as np
import pytest

pytest.importorskip("torch")

from oracle import cosmology as cm  # noqa: E402
from oracle import learned as ol  # noqa: E402
from paper_1509_04685_gb300 import learn  # noqa: E402


@pytest.mark.parametrize("x0,lo,hi", [(1.3, 0.0, 3.0), (-0.2, -0.3, 4.0), (3.9, -0.3, 4.0)])
def test_golden_section_brackets_the_minimum(x0, lo, hi):
    calls = []

    def f(x):
        calls.append(x)
        return (x - x0) ** 2

    for iters in (8, 20):
        calls.clear()
        x, fx = learn.golden_section(f, lo, hi, iters)
        assert len(calls) == iters + 2
        # the final bracket is (hi - lo) 0.618^iters wide and holds the minimum
        assert abs(x - x0) <= (hi - lo) * 0.6181 ** iters
        assert fx == pytest.approx((x - x0) ** 2)


def test_output_node_is_the_last_node_at_or_before_the_output():
    a = cm.time_nodes(0.05, 1.0, 40)
    assert learn.output_node(a[0], a) == 0
    assert learn.output_node(a[17], a) == 17
    assert learn.output_node(0.5 * (a[17] + a[18]), a) == 17
    assert learn.output_node(1.0, a) == 39
    assert learn.output_node(1.2, a) == 39


def test_filter_row_matches_the_oracle():
    for nrows in (1, 2, 5, 8):
        for a in np.linspace(0.0, 1.1, 111):
            assert learn.filter_row(a, nrows) == ol.filter_row(a, nrows, 0.05, 1.0)


def test_pk_deviation_is_the_mean_relative_difference_up_to_kmax():
    k = np.array([0.1, 0.5, 1.0, 2.0])
    p_ref = np.array([1.0, 2.0, 4.0, 8.0])
    p = np.array([1.1, 1.8, 4.0, 100.0])
    assert learn.pk_deviation(k, p, p_ref, 1.0) == pytest.approx((0.1 + 0.1 + 0.0) / 3)


def test_calibrated_filter_rule():
    # T' = (1 + g (T - 1)) (1 + c shape): g = 1, c = 0 keeps the fitted filter;
    # g = 0 flattens it to 1 before the boost; the boost shape is (a_r / a_f)
    # min(k / k_Ny, 1)^2, zero at k = 0, held beyond k_Ny, growing with a
    import torch

    na, nb = 8, 16
    base = 1.0 + 0.3 * torch.sin(torch.arange(na * nb, dtype=torch.float32)).reshape(na, nb)
    shape = learn.boost_shape(na, nb)
    torch.testing.assert_close(learn.calibrated_filter(base, 1.0, 0.0, shape), base)
    torch.testing.assert_close(learn.calibrated_filter(base, 0.0, 0.5, shape), (1.0 + 0.5 * shape).float())
    assert torch.all(shape[:, 0] == 0)
    kn = np.arange(nb) * np.sqrt(3.0) / (nb - 1)
    beyond = kn >= 1.0
    np.testing.assert_allclose(shape[:, beyond].numpy(), shape[:, beyond][:, :1].numpy().repeat(beyond.sum(), 1))
    np.testing.assert_allclose(shape[:, 4].numpy(), np.linspace(0.05, 1.0, na) * kn[4] ** 2, rtol=1e-12)
    assert torch.all(learn.boost_shape(1, nb)[0] == torch.clamp(torch.tensor(kn), max=1.0) ** 2)
    g, c = 1.4, 0.2
    want = (1.0 + g * (base.double() - 1.0)) * (1.0 + c * shape)
    torch.testing.assert_close(learn.calibrated_filter(base, g, c, shape), want.float())
