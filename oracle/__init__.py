"""FP64 CPU oracle of GSIS: test infrastructure, not part of the product path."""
