"""GB300-native NCI colour-gradient lattice Boltzmann (arXiv:2003.11069)."""
