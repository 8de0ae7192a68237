"""GB300-native Moment Tensor Potential hot path (arXiv:2007.08555, Sec. 2)."""
