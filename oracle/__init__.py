"""FP64 CPU oracle of the wall-modelled LBM LES step (test infrastructure only)."""
