"""GB300-native spectral Boltzmann collision operator (Boscheri & Dimarco,
arXiv 2103.14890): Fourier-spectral Q(f,f) per mesh cell and the local
penalised IMEX stage, as hand-written sm_103a CUDA kernels behind a C ABI."""
