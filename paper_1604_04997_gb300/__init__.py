"""GB300-native linear kernel run-time model (Stevens & Kloeckner, arXiv:1604.04997)."""
