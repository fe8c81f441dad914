// fam_probe.cu -- measurement helpers exported through the C ABI: the FP64 /
// FP32 fused multiply-add throughput of this GPU (the denominator of the
// ALU roofline), a check hook for the library's reciprocal and square root
// (refined FP32 seeds, fam_common.cuh), and one for its integer-pipe binary64
// multiply (which must equal IEEE round-to-nearest bit for bit).
#include <cuda_runtime.h>

#include "../../include/fam.h"
#include "fam_common.cuh"

namespace {

template <typename T, int CHAINS>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
double measure(int iters) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_loop<T, 8><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_loop<T, 8><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return -1.0;
  return 2.0 * 8.0 * (double)iters * blocks * threads * reps / (ms * 1e-3);
}

__global__ void math_kernel(const double* x, int n, double* rcp, double* rsq, double* sq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rcp[i] = fam::Fast<double>::rcp(x[i]);
    rsq[i] = fam::Fast<double>::rsqrt(x[i]);
    sq[i] = fam::Fast<double>::sqrt_(x[i]);
  }
}

__global__ void int_fp64_kernel(const double* a, const double* b, int n, double* prod) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) prod[i] = fam::dmul_int(a[i], b[i]);
}

}  // namespace

extern "C" fam_status fam_alu_peak(int precision, double* flops_per_s) {
  if (!flops_per_s || (precision != 64 && precision != 32)) return FAM_E_INVAL;
  double v = precision == 64 ? measure<double>(4096) : measure<float>(65536);
  if (v <= 0.0) return FAM_E_CUDA;
  *flops_per_s = v;
  return FAM_OK;
}

extern "C" fam_status fam_selftest_math(const double* x_host, int n, double* rcp_host, double* rsqrt_host,
                                        double* sqrt_host) {
  if (!x_host || n <= 0 || !rcp_host || !rsqrt_host || !sqrt_host) return FAM_E_INVAL;
  const size_t bytes = sizeof(double) * (size_t)n;
  // one checked allocation, sliced: no kernel runs unless all of it exists
  double* buf = nullptr;
  if (cudaMalloc(&buf, 4 * bytes) != cudaSuccess) return FAM_E_NOMEM;
  double *x = buf, *a = buf + n, *b = buf + 2 * (size_t)n, *c = buf + 3 * (size_t)n;
  cudaError_t e = cudaMemcpy(x, x_host, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    math_kernel<<<(n + 255) / 256, 256>>>(x, n, a, b, c);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(rcp_host, a, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(rsqrt_host, b, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(sqrt_host, c, bytes, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  return e == cudaSuccess ? FAM_OK : FAM_E_CUDA;
}

extern "C" fam_status fam_selftest_int_fp64(const double* a_host, const double* b_host, int n, double* prod_host) {
  if (!a_host || !b_host || n <= 0 || !prod_host) return FAM_E_INVAL;
  const size_t bytes = sizeof(double) * (size_t)n;
  double* buf = nullptr;
  if (cudaMalloc(&buf, 3 * bytes) != cudaSuccess) return FAM_E_NOMEM;
  double *a = buf, *b = buf + n, *p = buf + 2 * (size_t)n;
  cudaError_t e = cudaMemcpy(a, a_host, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b, b_host, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    int_fp64_kernel<<<(n + 255) / 256, 256>>>(a, b, n, p);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(prod_host, p, bytes, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  return e == cudaSuccess ? FAM_OK : FAM_E_CUDA;
}
