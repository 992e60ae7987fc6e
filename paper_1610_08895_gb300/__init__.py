"""GB300 implementation of the randomised primal-dual (PD-R) RI imaging path.

arXiv:1610.08895 (Onose, Carrillo, McEwen & Wiaux): Phi = G F Z and its
adjoint, the multi-basis wavelet dictionary Psi, and Algorithm 1 iterations,
all in hand-written CUDA kernels behind the C ABI of include/pd.h.

Submodules: ``api`` (Plan, State), ``autograd`` (PhiFunction), ``synth``
(seeded synthetic inputs), ``build`` (compiles the CUDA library in-tree).
"""


def __getattr__(name):
    if name in ("Plan", "State", "daubechies_filter"):
        from . import api
        return getattr(api, name)
    if name in ("PhiFunction", "phi"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
