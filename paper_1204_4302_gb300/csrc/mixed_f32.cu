// FP32 instantiation of the mixed-radix passes.
#include "mixed_impl.cuh"
template struct demag::MixedPasses<float>;
