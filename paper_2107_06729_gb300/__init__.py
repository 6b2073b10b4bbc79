"""GB300-native demag-extrapolated explicit LLG integrator (arXiv 2107.06729)."""
