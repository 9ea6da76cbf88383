// FP64 storage with double-float transforms: the pass kernels of an FP64 context
// compute their FFTs, tensor product and z convolution in dd (ddf.cuh) on the
// FP32 pipe; the RK prologue, the field / torque epilogue and every state
// vector stay FP64.
#include "engine_impl.cuh"

namespace mm {
void engine_rhs_dd(const Launch& L, int mode, const double* m, double* dmdt, double* heff, long long off_adjust) {
    engine_rhs_c<double, dd>(L, mode, m, dmdt, heff, off_adjust);
}
void engine_attempt_dd(const Launch& L, const RkBuffers& B) { engine_attempt_c<double, dd>(L, B); }
void engine_neb_attempt_dd(const Launch& L, const RkBuffers& B) { engine_neb_attempt_c<double, dd>(L, B); }
void engine_set_attributes_dd() { set_attrs<dd>(); }
}  // namespace mm
