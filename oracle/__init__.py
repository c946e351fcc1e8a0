"""FP64 CPU oracle: test infrastructure only (see ks_oracle.py)."""
