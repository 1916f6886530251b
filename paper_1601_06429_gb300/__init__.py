"""GB300-native Voronoi cells of every particle (PARAVT hot path, arXiv:1601.06429)."""
