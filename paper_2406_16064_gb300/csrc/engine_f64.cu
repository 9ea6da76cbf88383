// double instantiation of the engine (FP64 path), plus the precision-free
// control launches.
#include "engine_impl.cuh"

namespace mm {
template void engine_rhs<double>(const Launch&, int, const double*, double*, double*, long long);
template void engine_attempt<double>(const Launch&, const RkBuffers&);
template void engine_neb_attempt<double>(const Launch&, const RkBuffers&);

void engine_set_attributes_f32();
void engine_set_attributes_dd();
void engine_set_attributes() {
    set_attrs<double>();
    engine_set_attributes_f32();
    engine_set_attributes_dd();
}

void engine_bounded_wait(cudaStream_t s, int* flag, long long spins, int* status) {
    k_bounded_wait<<<1, 1, 0, s>>>(flag, spins, status);
}

void engine_after_stage1(const Launch& L) {
    k_after_stage1<<<blocks_for(L.nsims), 128, 0, L.stream>>>(L.desc, L.state, L.nsims);
}
}  // namespace mm
