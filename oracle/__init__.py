"""CPU oracle for SLR-PCG (test infrastructure only; see slr_oracle.py)."""
