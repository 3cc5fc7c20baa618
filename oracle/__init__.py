"""CPU oracle (test infrastructure only): see lss_oracle."""
