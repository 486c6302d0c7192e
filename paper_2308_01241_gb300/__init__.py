"""GB300-native hot path of the digital twin brain simulator (arXiv 2308.01241)."""
