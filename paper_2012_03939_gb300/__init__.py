"""GB300-native differentiable path tracer (forward + adjoint) behind a C-ABI library."""
