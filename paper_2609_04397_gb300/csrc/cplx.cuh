// Complex FP64 arithmetic of the VBCSR_C128 operators (periodic operators at a
// reciprocal-space point, Eq. 4): values, X and Y are interleaved (re, im)
// double pairs; a complex multiply-add is four FP64 FMAs; the adjoint product
// multiplies by the conjugate of each stored value (the dagger of Eq. 1).
#pragma once

#include <cuda_runtime.h>

namespace vbcsr {

struct Cplx {
    double re, im;
    __device__ __forceinline__ Cplx() {}
    __device__ __forceinline__ Cplx(int z) : re((double)z), im(0.0) {}
    __device__ __forceinline__ explicit Cplx(double2 v) : re(v.x), im(v.y) {}
    __device__ __forceinline__ Cplx(double r, double i) : re(r), im(i) {}
    __device__ __forceinline__ operator double2() const { return make_double2(re, im); }
};

__device__ __forceinline__ Cplx operator+(Cplx a, Cplx b) { return Cplx(a.re + b.re, a.im + b.im); }

__device__ __forceinline__ Cplx &operator+=(Cplx &a, Cplx b) {
    a.re += b.re;
    a.im += b.im;
    return a;
}

using ::__shfl_xor_sync;

__device__ __forceinline__ Cplx __shfl_xor_sync(unsigned mask, Cplx v, int m) {
    return Cplx(::__shfl_xor_sync(mask, v.re, m), ::__shfl_xor_sync(mask, v.im, m));
}

// acc + a * x
__device__ __forceinline__ Cplx fmat(Cplx a, Cplx x, Cplx acc) {
    return Cplx(fma(a.re, x.re, fma(-a.im, x.im, acc.re)), fma(a.re, x.im, fma(a.im, x.re, acc.im)));
}

// the value as the adjoint product uses it
__device__ __forceinline__ Cplx adj_val(Cplx v) { return Cplx(v.re, -v.im); }

}  // namespace vbcsr
