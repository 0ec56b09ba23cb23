"""Host-side logic of the learned parameters (no GPU): the knot
parameterisation and the leg-0 form whose memory strength is fixed."""
import torch

from paper_2607_27644_b300.learned import LearnedParams


def test_knots_start_uniform_and_stay_monotone():
    """Knots start as the K+1 equally spaced points of [gamma_min, gamma_max]
    (the plain method's uniform draw) and stay nondecreasing whatever the raw
    parameters, since each step is a softplus."""
    m = LearnedParams(3, 10, -0.15, 0.61, K=8, device="cpu")
    k = m.knots().detach().double()
    ref = torch.linspace(-0.15, 0.61, 9, dtype=torch.float64)
    assert torch.allclose(k, ref, atol=1e-6)
    with torch.no_grad():
        m.theta.copy_(torch.randn(9, generator=torch.Generator().manual_seed(3)) * 5)
    k = m.knots().detach()
    assert bool((k[1:] >= k[:-1]).all())
    assert {n for n, _ in m.named_parameters()} == {"w", "theta"}


def test_fixed_gamma_gives_two_equal_untrained_knots():
    """The leg-0 form: every variable at gamma0 -- two equal knots, so the
    inverse CDF is constant -- and only the message weights train."""
    m = LearnedParams(4, 12, -0.15, 0.61, device="cpu", fixed_gamma=0.125)
    k = m.knots()
    assert k.shape == (2,) and float(k[0]) == 0.125 and float(k[1]) == 0.125
    assert not k.requires_grad
    assert [n for n, _ in m.named_parameters()] == ["w"]
    assert torch.equal(m.w.detach(), torch.ones(4, 12))


def test_row_tied_weights_expand_to_edges():
    """Row-tied weights [T, C] expand to the edges of each row in CSR order."""
    row_of_edge = [0, 0, 1, 2, 2, 2]
    m = LearnedParams(2, 6, -0.15, 0.61, device="cpu", row_of_edge=row_of_edge, n_rows=3, fixed_gamma=0.125)
    with torch.no_grad():
        m.w.copy_(torch.tensor([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]]))
    ew = m.edge_weights()
    assert torch.equal(ew, torch.tensor([[1.0, 1.0, 2.0, 3.0, 3.0, 3.0], [4.0, 4.0, 5.0, 6.0, 6.0, 6.0]]))
