// Generated by fit_exp2_poly.py: minimax (relative error) polynomial for 2^f on [-1/2, 1/2],
// degree 5, constant term 1; max relative error of the float32 Horner evaluation 5.049e-07.
#pragma once
namespace ot {
constexpr int kExp2PolyDeg = 5;
__device__ constexpr float kExp2Poly[kExp2PolyDeg + 1] = {1.0f, 0.693142831325531f, 0.24022351205348969f, 0.05557400360703468f, 0.009666282683610916f, 0.0011125507298856974f};
}  // namespace ot
