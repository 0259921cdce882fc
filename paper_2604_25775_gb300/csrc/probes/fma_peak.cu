// fma_peak.cu -- FP32 / FP64 FMA throughput of the device (roofline denominators for the
// FMA-bound kernels): eight independent FMA chains per thread, 8 CTAs of 256 threads per
// SM, one store per thread. Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/fma_peak fma_peak.cu && /tmp/fma_peak
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int CH>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = acc[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename T, int CH>
double run(int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_loop<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  int reps = 5;
  for (int r = 0; r < reps; ++r) fma_loop<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) printf("err %s\n", cudaGetErrorString(err));
  cudaFree(out);
  double flops = 2.0 * CH * (double)iters * blocks * threads * reps;
  return flops / (ms * 1e-3) / 1e12;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("%s SMs=%d cc=%d.%d smem/blk optin=%zu\n", p.name, p.multiProcessorCount, p.major, p.minor, p.sharedMemPerBlockOptin);
  int sms = p.multiProcessorCount;
  printf("fp32 TFLOP/s: %.2f\n", run<float, 8>(sms * 8, 256, 1 << 16));
  printf("fp32 TFLOP/s: %.2f\n", run<float, 8>(sms * 8, 256, 1 << 16));
  printf("fp64 TFLOP/s: %.3f\n", run<double, 8>(sms * 8, 256, 1 << 12));
  printf("fp64 TFLOP/s: %.3f\n", run<double, 8>(sms * 8, 256, 1 << 12));
  return 0;
}
