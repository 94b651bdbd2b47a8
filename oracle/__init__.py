"""CPU oracle (test infrastructure only; see purify_oracle's docstring)."""
