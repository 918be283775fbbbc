// Self-check of the library's FP64 arithmetic helpers against CUDA's own operations (no paper
// counterpart): the reciprocal-seeded quotient and reciprocals that replace FP64 divisions where
// the FP64 pipe bounds a kernel, and the integer-pipe comparisons of doubles.
#include "mgfld_internal.cuh"

namespace mgfld {

constexpr int kCheckFields = 8;

__global__ void k_arith_check(const double *__restrict__ a, const double *__restrict__ b, int count,
                              double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double x = a[i], y = b[i];
  double *o = out + (size_t)i * kCheckFields;
  o[0] = quot(x, y);
  o[1] = x / y;
  o[2] = recip2(y);
  o[3] = 1.0 / y;
  o[4] = recip(y);
  o[5] = ord_key(x) < ord_key(y) ? 1.0 : 0.0;
  o[6] = x < y ? 1.0 : 0.0;
  o[7] = is_zero(x) ? 1.0 : 0.0;
}

}  // namespace mgfld

using namespace mgfld;

extern "C" mgfld_status mgfld_arith_check(const double *a, const double *b, int count, double *out, void *stream) {
  if (count < 0 || (count > 0 && (!a || !b || !out))) return MGFLD_EINVAL;
  if (count == 0) return MGFLD_OK;
  k_arith_check<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a, b, count, out);
  return cudaGetLastError() == cudaSuccess ? MGFLD_OK : MGFLD_ECUDA;
}
