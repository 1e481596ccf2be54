"""CPU oracle (test infrastructure only; see oracle/mwmm_oracle.c)."""
