"""FP64 CPU oracle of the two-fluid kinetic step (test infrastructure only)."""
