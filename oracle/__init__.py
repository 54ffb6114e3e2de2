"""FP64 CPU oracle for HALLaR -- test infrastructure only (see hallar_oracle)."""
