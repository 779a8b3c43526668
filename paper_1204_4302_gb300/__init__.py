"""GB300-native FFT demagnetization-tensor (DM) stray-field library.

The computation lives in libdemag.so (CUDA kernels for sm_103a behind the C ABI
of include/demag.h). ``binding`` exposes the C entry points, ``plan.Plan`` wraps
a plan for torch tensors, ``autograd`` provides DemagField / DemagEnergy.
``inputs`` draws the seeded synthetic magnetization states.
"""


def __getattr__(name):
    # lazy: importing the package must not require torch or the built library
    if name == "Plan":
        from .plan import Plan
        return Plan
    if name in ("DemagField", "DemagEnergy", "demag_field", "demag_energy"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
