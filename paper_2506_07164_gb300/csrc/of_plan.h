// Host-side plan arithmetic (of_plan.cpp).
#pragma once
#include <stdint.h>

namespace ofh {
void level_sizes(int W, int H, int levels, float scale, int32_t* ws, int32_t* hs, double* ls);
void level_quotas(int N, int L, float scale, int32_t* q);
void resize_table(int n_src, int n_dst, int32_t* tab);
bool k_fraction(float k, int64_t* num, int64_t* den);
// (1 / (4*7*255))^4 / den as float: the keypoint response is key * this
// (float arithmetic; within 3e-7 relative of the float64 quotient).
float response_scale(int64_t den);
}  // namespace ofh
