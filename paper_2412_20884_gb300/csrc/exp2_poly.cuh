// Generated by gen_exp2_poly.py: minimax (relative error) polynomials
// for 2^f on [-1/2, 1/2], coefficients rounded to FP32, in Horner form.
#pragma once

#include <cuda_runtime.h>

namespace kmv {
// degree 3: max relative error 7.480e-05 (FP64 evaluation of the FP32 coefficients)
__host__ __device__ __forceinline__ float exp2_poly3(float f) { return fmaf(fmaf(fmaf(0.0551716685295105f, f, 0.2426111251115799f), f, 0.6932609677314758f), f, 0.9999280571937561f); }
constexpr double kExp2Poly3Err = 7.479879e-05;
// degree 5: max relative error 1.547e-07 (FP64 evaluation of the FP32 coefficients)
__host__ __device__ __forceinline__ float exp2_poly5(float f) { return fmaf(fmaf(fmaf(fmaf(fmaf(0.0013276472454890609f, f, 0.009675540961325169f), f, 0.05550713092088699f), f, 0.24022120237350464f), f, 0.6931469440460205f), f, 1.0000001192092896f); }
constexpr double kExp2Poly5Err = 1.547034e-07;
}  // namespace kmv
