"""FP64 CPU oracle (test infrastructure only; see fctn_oracle.py)."""
