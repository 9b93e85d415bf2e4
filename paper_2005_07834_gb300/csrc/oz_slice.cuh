// Exact bf16 slices of one 32-wide float64 row for the tensor-core
// float64-accurate update (k_ozaki.cu): a warp-collective call, lane k passing
// x = X[row][k] (0 beyond the row's width).  The row is scaled by 2^-e (e from
// the largest exponent of the row, so that every scaled value lies in
// (-1/2, 1/2)) and cut into seven integer slices of at most 8 bits, two per
// 128-byte plane row: planes[t / 2][row][(t % 2) 32 + k].  Integer and fp32
// instructions only (oz_combine.cuh).
#pragma once

#include <cstdint>

#include "oz_combine.cuh"

namespace lrs {

constexpr int OZ_SLICE_COUNT = 7;
constexpr int OZ_PLANE_COUNT = 4;

__device__ __forceinline__ void oz_slice_row(double x, int k, int row, size_t plane_stride, uint16_t* planes,
                                             int* expo) {
  const int e = oz_row_scale((int)__reduce_max_sync(0xffffffffu, (unsigned)oz_exp_field(x)));
  if (k == 0) expo[row] = e;
  // a = x 2^-e as the integer N = round(a 2^56), |N| <= 2^55 (rounding error at most 2^-56 of
  // 2^e), written in base 256 with balanced digits s_6 .. s_1 in [-128, 127] and the leading
  // digit s_0 in [-128, 128]: N = sum_t s_t 256^(6 - t)
  long long N = oz_fixed56(x, e);
  int dig[OZ_SLICE_COUNT];
#pragma unroll
  for (int t = OZ_SLICE_COUNT - 1; t > 0; --t) {
    const long long d = ((N + 128) & 255) - 128;
    dig[t] = (int)d;
    N = (N - d) >> 8;                           // exact
  }
  dig[0] = (int)N;
#pragma unroll
  for (int t = 0; t < 2 * OZ_PLANE_COUNT; ++t)
    planes[(t >> 1) * plane_stride + (size_t)row * 64 + (t & 1) * 32 + k] =
        t < OZ_SLICE_COUNT ? oz_int_to_bf16_bits(dig[t]) : (uint16_t)0;
}

}  // namespace lrs
