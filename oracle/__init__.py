"""CPU oracle package (test infrastructure only; see tfde_oracle.py)."""
