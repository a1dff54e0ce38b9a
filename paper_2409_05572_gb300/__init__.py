"""GB300-native shrink-and-expand block eigensolvers (arXiv:2409.05572)."""
