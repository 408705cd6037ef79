"""CPU FP64 oracle (test infrastructure only; see hz_oracle)."""
