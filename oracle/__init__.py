"""FP64 sequential oracle (test infrastructure)."""
