"""GB300 (sm_103a) implementation of the O(L^3) hot path of the exact spin spherical harmonic
transform of McEwen, "Fast, exact (but unstable) spin spherical harmonic transforms"
(arXiv:0807.4494): the FP64 recursions for Delta^l = d^l(pi/2) and their contractions with the
torus Fourier coefficients, forward, inverse and adjoint, behind the C ABI of include/ssht.h.

``paper_0807_4494_gb300.ssht`` is the binding (loaded lazily, so that ``inputs`` can be
imported without the CUDA library); ``paper_0807_4494_gb300.build`` compiles the library.
"""
