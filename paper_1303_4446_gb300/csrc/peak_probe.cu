// Peak-rate probe for the roofline denominators of this library on the local GPU:
// FP64 FMA (DFMA), FP64 tensor MMA (mma.sync f64, two shapes) and legacy BF16 mma.sync.
// Register-only loops; prints TFLOP/s.  Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678) out[0] = s;
}

__global__ void dmma884_kernel(double* out, int iters) {
  double a = threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-4;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) { c[i][0] = 0; c[i][1] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  if (s == 12345.678) out[0] = s;
}

__global__ void dmma16816_kernel(double* out, int iters) {
  double a[8], b[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = 1.0 - i * 1e-4;
  double c[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i) for (int j = 0; j < 4; ++j) c[i][j] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                   : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
                   : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                     "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) for (int j = 0; j < 4; ++j) s += c[i][j];
  if (s == 12345.678) out[0] = s;
}

__global__ void bf16mma_kernel(float* out, int iters) {
  unsigned a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u + threadIdx.x;
  b[0] = 0x3f803f80u; b[1] = 0x3f803f81u;
  float c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) c[i][j] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) s += c[i][j];
  if (s == 12345.678f) out[0] = s;
}

int main() {
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceProp prop; CK(cudaGetDeviceProperties(&prop, dev));
  printf("device %s SMs %d cc %d.%d smem/block optin %zu\n", prop.name, nsm, prop.major, prop.minor, prop.sharedMemPerBlockOptin);
  double* d; CK(cudaMalloc(&d, 64));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  for (int occ : {4, 8}) {
    int blocks = nsm * occ, threads = 256, iters = 1 << 14;
    dfma_kernel<<<blocks, threads>>>(d, 16, 1.0000001, 1e-9);
    CK(cudaEventRecord(e0)); dfma_kernel<<<blocks, threads>>>(d, iters, 1.0000001, 1e-9); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("DFMA occ %d: %.3f TFLOP/s (%.3f ms)\n", occ, 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12, ms);
  }
  for (int occ : {2, 4, 8}) {
    int blocks = nsm * occ, threads = 256, iters = 1 << 12;
    dmma884_kernel<<<blocks, threads>>>(d, 16);
    CK(cudaEventRecord(e0)); dmma884_kernel<<<blocks, threads>>>(d, iters); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1));
    double fl = 512.0 * 4 * iters * (double)blocks * (threads / 32);
    printf("DMMA m8n8k4 occ %d: %.3f TFLOP/s (%.3f ms)\n", occ, fl / (ms * 1e-3) / 1e12, ms);
  }
  for (int occ : {2, 4, 8}) {
    int blocks = nsm * occ, threads = 256, iters = 1 << 10;
    dmma16816_kernel<<<blocks, threads>>>(d, 16);
    CK(cudaEventRecord(e0)); dmma16816_kernel<<<blocks, threads>>>(d, iters); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1));
    double fl = 2.0 * 16 * 8 * 16 * 2 * iters * (double)blocks * (threads / 32);
    printf("DMMA m16n8k16 occ %d: %.3f TFLOP/s (%.3f ms)\n", occ, fl / (ms * 1e-3) / 1e12, ms);
  }
  for (int occ : {2, 4}) {
    int blocks = nsm * occ, threads = 256, iters = 1 << 14;
    bf16mma_kernel<<<blocks, threads>>>((float*)d, 16);
    CK(cudaEventRecord(e0)); bf16mma_kernel<<<blocks, threads>>>((float*)d, iters); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1));
    double fl = 2.0 * 16 * 8 * 16 * 4 * iters * (double)blocks * (threads / 32);
    printf("BF16 mma.sync m16n8k16 occ %d: %.3f TFLOP/s (%.3f ms)\n", occ, fl / (ms * 1e-3) / 1e12, ms);
  }
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  return 0;
}
