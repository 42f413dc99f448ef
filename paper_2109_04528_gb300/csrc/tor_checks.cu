// tor_checks.cu -- tor_check_recip: the FP64 reciprocal and reciprocal square
// root that every include step's 2x2 pivot uses (rcp64 / rsqrt64 in
// tor_device.cuh: the hardware estimate refined by one cubic series step),
// evaluated beside CUDA's own correctly rounded division 1.0 / x and its
// rsqrt(x) on the same inputs, so their error can be stated and tested.
#include <cuda_runtime.h>

#include "../../include/tor.h"
#include "tor_device.cuh"

namespace tor {
namespace {

__global__ void k_check_recip(const double* x, int count, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = x[i];
  out[4 * i + 0] = rcp64(v);
  out[4 * i + 1] = __ddiv_rn(1.0, v);  // IEEE division, round to nearest
  out[4 * i + 2] = rsqrt64(v);
  out[4 * i + 3] = rsqrt(v);
}

}  // namespace
}  // namespace tor

extern "C" tor_status tor_check_recip(int device, int count, const double* x, double* out) {
  if (count < 0 || (count > 0 && (!x || !out)) || count > (1 << 26)) return TOR_EINVAL;
  if (count == 0) return TOR_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TOR_EINVAL;
  }
  double *dx = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&dx, sizeof(double) * (size_t)count);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 4 * (size_t)count);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int threads = 256;
    tor::k_check_recip<<<(count + threads - 1) / threads, threads>>>(dx, count, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * 4 * (size_t)count, cudaMemcpyDeviceToHost);
  const tor_status st = e == cudaSuccess ? TOR_OK : e == cudaErrorMemoryAllocation ? TOR_ENOMEM : TOR_ECUDA;
  cudaGetLastError();
  if (dx) cudaFree(dx);
  if (dout) cudaFree(dout);
  cudaSetDevice(prev);
  return st;
}
