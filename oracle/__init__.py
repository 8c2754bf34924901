"""FP64 CPU oracle of the TLMPM cutting substep (test infrastructure only)."""
