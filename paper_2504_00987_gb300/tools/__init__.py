"""Measurement tools of the package (not used by the solver itself)."""
