"""GB300-native two-species MRT lattice Boltzmann hot path (arXiv:1603.08221)."""
