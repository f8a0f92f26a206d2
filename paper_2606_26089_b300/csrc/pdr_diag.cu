// Diagnostic entry point: the library's single-precision function
// approximations (pdr_math.cuh and the cosh / sinh / asinh / smearing helpers
// of the response kernel, and the float-float exponential and sinh of
// pdr_ff.cuh as their hi and lo parts), evaluated element-wise on device arrays so a test
// can hold each to its stated error bound over its whole input range.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdr.h"
#include "pdr_ff.cuh"
#include "pdr_internal.h"
#include "pdr_math.cuh"

namespace pdr {
int set_last_error(int code, const char* msg);
}  // namespace pdr

using namespace pdr;

namespace {

__global__ void math_eval_kernel(int fn, const float* __restrict__ x, const float* __restrict__ x2,
                                 float* __restrict__ y, uint64_t n) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const float v = x[k];
    float r = 0.0f;
    switch (fn) {
      case PDR_FN_ASIN_HALF: r = asin_half(v); break;
      case PDR_FN_SIN_HALF_TURN: r = sin_half_turn(v); break;
      case PDR_FN_LN_UNIT: r = ln_unit(v); break;
      case PDR_FN_LOG1P_POS: r = log1p_pos(v); break;
      case PDR_FN_COS_TWO_PI: r = cos_two_pi(v); break;
      case PDR_FN_COSH: { float c, s; cosh_sinh(v, c, s); r = c; break; }
      case PDR_FN_SINH: { float c, s; cosh_sinh(v, c, s); r = s; break; }
      case PDR_FN_ASINH: r = asinh_fast(v); break;
      case PDR_FN_U01: r = u01(__float_as_uint(v)); break;
      case PDR_FN_NORMAL: r = normal(__float_as_uint(v), __float_as_uint(x2[k])); break;
      case PDR_FN_RCP: r = rcp_approx(v); break;
      case PDR_FN_SQRT: r = sqrt_approx(v); break;
      case PDR_FN_EXP_FF_HI: r = exp_ff(v).hi; break;
      case PDR_FN_EXP_FF_LO: r = exp_ff(v).lo; break;
      case PDR_FN_SINH_FF_HI: r = sinh_ff(v).hi; break;
      case PDR_FN_SINH_FF_LO: r = sinh_ff(v).lo; break;
      default: break;
    }
    y[k] = r;
  }
}

}  // namespace

extern "C" int pdr_math_eval(int fn, const float* x, const float* x2, float* y, uint64_t n, void* stream) {
  if (fn < 0 || fn >= PDR_FN_COUNT) return set_last_error(PDR_EINVAL, "unknown function");
  if (n == 0) return PDR_OK;
  if (!x || !y || (fn == PDR_FN_NORMAL && !x2)) return set_last_error(PDR_EINVAL, "null array");
  const uint64_t blocks = (n + 255) / 256;
  math_eval_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, (cudaStream_t)stream>>>(fn, x, x2, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PDR_OK : set_last_error(PDR_EDEVICE, cudaGetErrorString(e));
}
