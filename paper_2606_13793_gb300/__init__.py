"""GB300-native unigrid FMM Poisson solver (package)."""
