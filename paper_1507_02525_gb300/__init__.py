"""GB300-native multiresolution DFT (MrDFT) of Andreatto & Cariow (arXiv:1507.02525).

Public API (PyTorch tensors on a CUDA device; arithmetic in the sm_103a kernels):
    mrdft, mrdft_adjoint, mrdft_ragged, mrdft_ragged_adjoint, MrDFT (autograd)
Low level: ``paper_1507_02525_gb300._lib.Plan`` wraps the C ABI of include/mrdft.h.
Importing the package does not load CUDA; the library loads on first use.
"""

__all__ = ["mrdft", "mrdft_adjoint", "mrdft_loss_grad", "mrdft_ragged", "mrdft_ragged_adjoint", "MrDFT", "get_plan"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
