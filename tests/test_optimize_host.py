"""Host logic of the Adam driver (no GPU): parameter clamping by texel layout."""
import pytest

torch = pytest.importorskip("torch")

from paper_2012_03939_gb300.optimize import clamp_params_


@pytest.mark.parametrize("width", [5, 7])
def test_clamp_by_layout(width):
    P = torch.linspace(-2.0, 2.0, 9 * width).reshape(9, width).clone()
    raw = P.clone()
    clamp_params_(P)
    r = width - 1                      # roughness is the last column in both layouts
    assert torch.equal(P[:, :r], raw[:, :r].clamp(0.0, 1.0))
    assert torch.equal(P[:, r], raw[:, r].clamp(0.01, 1.0))
    # with 7 columns the fifth is ks_g (an albedo-like value), not roughness
    if width == 7:
        assert float(P[:, 4].min()) == 0.0


def test_clamp_rejects_other_layouts():
    with pytest.raises(ValueError):
        clamp_params_(torch.zeros(4, 6))
