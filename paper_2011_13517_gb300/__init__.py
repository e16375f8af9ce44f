"""GB300-native (sm_103a) Clenshaw-Curtis spectral quadrature (arXiv 2011.13517)."""
