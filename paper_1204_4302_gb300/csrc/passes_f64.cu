// FP64 instantiation of the field passes (also used by the tensor setup).
#include "passes_impl.cuh"
template struct demag::Passes<double>;
