// float instantiation of the engine (FP32 path: fields, FFTs and RK stages in
// FP32; norms, error norm and energies in FP64).
#include "engine_impl.cuh"

namespace mm {
template void engine_rhs<float>(const Launch&, int, const float*, float*, float*, long long);
template void engine_attempt<float>(const Launch&, const RkBuffers&);
template void engine_neb_attempt<float>(const Launch&, const RkBuffers&);
void engine_set_attributes_f32() { set_attrs<float>(); }
}  // namespace mm
