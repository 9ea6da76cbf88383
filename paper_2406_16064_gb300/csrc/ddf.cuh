// Double-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the FFT passes of an
// FP64 context compute in this type on the FP32 pipe: the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct through
// the fused multiply-add (Dekker 1971), combined as in the double-double
// algorithms of Hida, Li & Bailey (2001) in their "sloppy" addition form (its
// error is bounded by ~2^-46 of the operands' magnitudes, which is what an FFT
// butterfly needs).  The _rn intrinsics keep the compiler from contracting or
// reordering the compensation terms.  Storage stays FP64: a state vector is
// split into hi + lo when it enters a transform and rounded back to FP64 when
// it leaves.  One dd is 8 bytes, so spectra, tensors and twiddle tables keep
// the FP64 layout and size.
#pragma once
#include <cuda_runtime.h>

struct dd {
    float hi, lo;
    dd() = default;
    // split of an FP64 value: exact to 2^-48 relative (constant arguments fold at compile time)
    __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (a, b any order)
__device__ __forceinline__ void dd_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// renormalise s + e (|e| small against s) to a dd
__device__ __forceinline__ dd dd_quick(float s, float e) {
    const float h = __fadd_rn(s, e);
    return dd(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
    float s, e;
    dd_two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return dd_quick(s, e);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd_quick(p, e);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { a = a + b; return a; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { a = a - b; return a; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { a = a * b; return a; }

// Storage type of a compute type: FP64 contexts keep FP64 state and compute
// their transforms in dd.
template <typename T> struct Store { using type = T; };
template <> struct Store<dd> { using type = double; };
template <typename T> using StoreT = typename Store<T>::type;

// storage value -> compute value and back
template <typename T> __device__ __forceinline__ T to_compute(StoreT<T> x) { return x; }
template <> __device__ __forceinline__ dd to_compute<dd>(double x) { return dd(x); }
template <typename T> __device__ __forceinline__ StoreT<T> to_store(T x) { return x; }
template <> __device__ __forceinline__ double to_store<dd>(dd x) { return (double)x; }

