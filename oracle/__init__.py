"""CPU oracle (test infrastructure only; see h2_oracle)."""
