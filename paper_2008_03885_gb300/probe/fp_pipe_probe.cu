// Floating-point pipe throughput probe for the ALU roofline of the FP64 kernels:
// independent FMA / add / multiply chains per thread, no memory traffic.
#include <cstdio>
#include <cuda_runtime.h>
template <int OP, typename T>
__global__ void k(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (OP == 0) x[c] = fma(x[c], a, b);
      else if (OP == 1) x[c] = x[c] + b;
      else x[c] = x[c] * a;
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int OP, typename T>
void run(const char* name, T a, T b) {
  int blocks = 152 * 8, threads = 256, iters = 2048;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  k<OP, T><<<blocks, threads>>>(out, iters, a, b);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) k<OP, T><<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double ops = 5.0 * blocks * threads * (double)iters * 8;
  printf("%s: %.1f Gop/s (%.3f ms per launch) err=%s\n", name, ops / (ms * 1e-3) / 1e9, ms / 5,
         cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() {
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  printf("SMs %d, clock %d kHz\n", sms, clk);
  run<0, double>("DFMA", 0.999999, 1e-7);
  run<1, double>("DADD", 0.999999, 1e-7);
  run<2, double>("DMUL", 0.999999, 1e-7);
  run<0, float>("FFMA", 0.999999f, 1e-7f);
  run<1, float>("FADD", 0.999999f, 1e-7f);
  return 0;
}
