// FP32 instantiation of the field passes.
#include "passes_impl.cuh"
template struct demag::Passes<float>;
