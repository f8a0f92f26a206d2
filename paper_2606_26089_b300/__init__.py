"""B300-native parametric detector response (the TorchDelphes chain of
arXiv:2606.26089, Sec. 2.2 / App. D, with the isolation of Sec. 2.4).

* ``binding``  ctypes binding of the CUDA library ``libpdr.so`` (include/pdr.h)
* ``synth``    seeded synthetic truth-event workloads
* ``build``    nvcc build of the library for sm_103a
* ``cards/``   the detector cards (raw parameters, JSON)
"""
__all__ = ["binding", "synth", "build"]
