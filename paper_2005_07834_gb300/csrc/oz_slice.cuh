// Exact bf16 slices of one 32-wide float64 row for the tensor-core
// float64-accurate update (k_ozaki.cu): a warp-collective call, lane k passing
// x = X[row][k] (0 beyond the row's width).  The row is scaled by 2^-e (e the
// exponent of its largest magnitude) and cut into seven integer slices of at
// most 9 bits (integer arithmetic), two per 128-byte plane row:
// planes[t / 2][row][(t % 2) 32 + k].
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace lrs {

constexpr int OZ_SLICE_COUNT = 7;
constexpr int OZ_PLANE_COUNT = 4;

__device__ __forceinline__ void oz_slice_row(double x, int k, int row, size_t plane_stride, uint16_t* planes,
                                             int* expo) {
  double m = fabs(x);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) frexp(m, &e);                  // m = f 2^e, f in [0.5, 1)
  if (k == 0) expo[row] = e;
  // a = x 2^-e as the integer N = round(a 2^56), |N| < 2^56 (rounding error below 2^-57
  // of the row maximum), written in base 256 with balanced digits s_6 .. s_1 in
  // [-128, 127] and the leading digit s_0 in [-256, 256]: N = sum_t s_t 256^(6 - t)
  long long N = __double2ll_rn(ldexp(x, 56 - e));
  int dig[OZ_SLICE_COUNT];
#pragma unroll
  for (int t = OZ_SLICE_COUNT - 1; t > 0; --t) {
    const long long d = ((N + 128) & 255) - 128;
    dig[t] = (int)d;
    N = (N - d) / 256;                          // exact
  }
  dig[0] = (int)N;
#pragma unroll
  for (int t = 0; t < 2 * OZ_PLANE_COUNT; ++t) {
    const float sl = t < OZ_SLICE_COUNT ? (float)dig[t] : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(sl);   // an integer of at most 9 bits: exact
    planes[(t >> 1) * plane_stride + (size_t)row * 64 + (t & 1) * 32 + k] = __bfloat16_as_ushort(b);
  }
}

}  // namespace lrs
