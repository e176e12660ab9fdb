// fp_peaks.cu -- throughput probe of the arithmetic pipes this engine uses on
// sm_103a: DFMA, DMMA (mma.sync m8n8k4 / m16n8k4 f64), FFMA, mma.sync with
// TF32, BF16, FP16 (FP32 accumulation) and S8 (S32 accumulation) inputs, and
// FP64 DFMA / sqrt / division with 1..32 active lanes per warp (does an FP64
// warp instruction cost the same whatever the number of active lanes?).
// Bounded loops only; prints one JSON object.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                           \
  do {                                                                  \
    cudaError_t e = (x);                                                \
    if (e != cudaSuccess) {                                             \
      printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));            \
      return 1;                                                         \
    }                                                                   \
  } while (0)

template <int IT>
__global__ void k_dfma(double* out, double a, double b, int active) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  if ((threadIdx.x & 31) < active)
    for (int i = 0; i < IT; i++) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int IT>
__global__ void k_dsqrt(double* out, double a, int active) {
  double x0 = threadIdx.x + 2.0, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  if ((threadIdx.x & 31) < active)
    for (int i = 0; i < IT; i++) {
      x0 = sqrt(x0) + a; x1 = sqrt(x1) + a; x2 = sqrt(x2) + a; x3 = sqrt(x3) + a;
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int IT>
__global__ void k_ddiv(double* out, double a, int active) {
  double x0 = threadIdx.x + 2.0, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  if ((threadIdx.x & 31) < active)
    for (int i = 0; i < IT; i++) {
      x0 = a / x0 + 1.5; x1 = a / x1 + 1.5; x2 = a / x2 + 1.5; x3 = a / x3 + 1.5;
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int IT>
__global__ void k_ffma(float* out, float a, float b) {
  float x[16];
  for (int j = 0; j < 16; j++) x[j] = threadIdx.x + j;
  for (int i = 0; i < IT; i++)
#pragma unroll
    for (int j = 0; j < 16; j++) x[j] = fmaf(x[j], a, b);
  float s = 0;
  for (int j = 0; j < 16; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int IT>
__global__ void k_dmma884(double* out) {
  double a = threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-4;
  double c[4][2];
  for (int j = 0; j < 4; j++) c[j][0] = c[j][1] = 0;
  for (int i = 0; i < IT; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a), "d"(b));
  double s = 0;
  for (int j = 0; j < 4; j++) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int IT>
__global__ void k_tf32(float* out) {
  unsigned a0 = __float_as_uint(threadIdx.x * 1e-3f), b0 = __float_as_uint(1.0f);
  float c[4][4];
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) c[j][q] = 0;
  for (int i = 0; i < IT; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                   : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
  float s = 0;
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) s += c[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// mma.sync with 16-bit inputs (m16n8k16, FP32 accumulation): BF16 or FP16
template <int IT, bool BF>
__global__ void k_mma16(float* out) {
  const unsigned a0 = 0x3c003c00u + threadIdx.x, b0 = 0x3c003c00u;
  float c[4][4];
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) c[j][q] = 0;
  for (int i = 0; i < IT; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      if constexpr (BF)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                     : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
      else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                     : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
    }
  float s = 0;
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) s += c[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// mma.sync with S8 inputs (m16n8k32, S32 accumulation)
template <int IT>
__global__ void k_mma_s8(int* out) {
  const unsigned a0 = 0x01020304u + threadIdx.x, b0 = 0x01010101u;
  int c[4][4];
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) c[j][q] = 0;
  for (int i = 0; i < IT; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                   : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
  int s = 0;
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) s += c[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  const int sms = p.multiProcessorCount, blocks = sms * 8, thr = 256, warps = blocks * thr / 32;
  double* d;
  CK(cudaMalloc(&d, sizeof(double) * blocks * thr));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms;
  auto time = [&](auto launch) {
    launch();
    cudaDeviceSynchronize();
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms;
  };
  const int IT = 2048;
  printf("{\"gpu\": \"%s\", \"sms\": %d", p.name, sms);
  double t = time([&] { k_dfma<IT><<<blocks, thr>>>(d, 0.999, 1e-3, 32); });
  printf(", \"dfma_tflops\": %.4f", 2.0 * 4 * IT * warps * 32 / t / 1e9);
  t = time([&] { k_dmma884<IT / 4><<<blocks, thr>>>(d); });
  printf(", \"dmma_m8n8k4_tflops\": %.4f", 512.0 * 4 * (IT / 4) * warps / t / 1e9);
  t = time([&] { k_ffma<IT * 4><<<blocks, thr>>>((float*)d, 0.999f, 1e-3f); });
  printf(", \"ffma_tflops\": %.3f", 2.0 * 16 * IT * 4 * warps * 32 / t / 1e9);
  t = time([&] { k_tf32<IT * 4><<<blocks, thr>>>((float*)d); });
  printf(", \"tf32_mma_sync_tflops\": %.2f", 2048.0 * 4 * (IT * 4) * warps / t / 1e9);
  t = time([&] { k_mma16<IT * 4, true><<<blocks, thr>>>((float*)d); });
  printf(", \"bf16_mma_sync_tflops\": %.2f", 4096.0 * 4 * (IT * 4) * warps / t / 1e9);
  t = time([&] { k_mma16<IT * 4, false><<<blocks, thr>>>((float*)d); });
  printf(", \"fp16_mma_sync_tflops\": %.2f", 4096.0 * 4 * (IT * 4) * warps / t / 1e9);
  t = time([&] { k_mma_s8<IT * 4><<<blocks, thr>>>((int*)d); });
  printf(", \"s8_mma_sync_tops\": %.2f", 8192.0 * 4 * (IT * 4) * warps / t / 1e9);
  printf(", \"fp64_by_active_lanes\": [");
  const int act[5] = {1, 4, 8, 16, 32};
  for (int r = 0; r < 5; r++) {
    const int a = act[r];
    const double tf = time([&] { k_dfma<1024><<<blocks, thr>>>(d, 0.999, 1e-3, a); });
    const double ts = time([&] { k_dsqrt<256><<<blocks, thr>>>(d, 1e-3, a); });
    const double td = time([&] { k_ddiv<256><<<blocks, thr>>>(d, 1.7, a); });
    printf("%s{\"active\": %d, \"dfma_warp_instr_per_ns\": %.3f, \"dfma_ms\": %.3f, \"dsqrt_ms\": %.3f, \"ddiv_ms\": %.3f}",
           r ? ", " : "", a, 4.0 * 1024 * warps / tf / 1e6, tf, ts, td);
  }
  printf("]}\n");
  CK(cudaGetLastError());
  return 0;
}
