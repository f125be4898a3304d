"""FP64 CPU oracle of the active-soil particle step (test infrastructure only)."""
