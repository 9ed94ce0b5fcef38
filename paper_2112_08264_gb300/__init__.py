"""GB300-native two-component D3Q19 lattice-Boltzmann (Shan-Chen) solver."""
