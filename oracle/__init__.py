"""FP64 CPU oracle of the PlenOctree render path (test infrastructure only)."""
