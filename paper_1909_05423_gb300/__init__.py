"""GB300-native FFT / tridiagonal Poisson solver (the hot path of PittPack, arXiv 1909.05423)."""
