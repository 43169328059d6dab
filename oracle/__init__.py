"""FP64 CPU oracle of the multi-hypothesis criticality method -- test infrastructure only."""
