"""GB300 (sm_103a) LASTO interstitial Poisson step.

The computation lives in ``liblasto_poisson.so`` (CUDA, C ABI in
``include/lasto_poisson.h``); ``binding`` marshals PyTorch device tensors into
it.  Importing the package does not load the library; ``binding.load()`` does,
and fails loudly when the library or a CUDA device is missing.  ``build.build()``
compiles the library in-tree.
"""
