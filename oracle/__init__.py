"""FP64 CPU oracle (test infrastructure; see lddmm_oracle)."""
