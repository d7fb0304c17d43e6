"""FP64 CPU oracle (test infrastructure only; see krr_oracle.py)."""
