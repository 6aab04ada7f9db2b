"""FP64 CPU oracle of the DDF lattice Boltzmann update (test infrastructure only)."""
