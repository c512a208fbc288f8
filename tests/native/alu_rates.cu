// Arithmetic-unit throughput of the current GPU: FP64 FMA, FP32 FMA, packed
// FP32 FMA (two lane FMAs per instruction) and the binary64 -> binary32
// conversion instruction.  Eight independent chains per thread, four CTAs of
// 512 threads per SM, one warm launch before the timed one (CUDA events).
// Prints one JSON object.  Test support: the measured FP64 FMA rate is the
// peak of the FP64-bound orthogonalisation passes' roofline.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int IT = 4096;

__global__ void p_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < IT; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void p_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < 8 * IT; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void p_ffma2(float* out, float a, float b) {
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  float2 x0 = make_float2(threadIdx.x, 1), x1 = make_float2(2, 3), x2 = make_float2(4, 5), x3 = make_float2(6, 7);
  float2 x4 = make_float2(8, 9), x5 = make_float2(10, 11), x6 = make_float2(12, 13), x7 = make_float2(14, 15);
  for (int i = 0; i < 4 * IT; ++i) {
    x0 = __ffma2_rn(x0, A, B); x1 = __ffma2_rn(x1, A, B); x2 = __ffma2_rn(x2, A, B); x3 = __ffma2_rn(x3, A, B);
    x4 = __ffma2_rn(x4, A, B); x5 = __ffma2_rn(x5, A, B); x6 = __ffma2_rn(x6, A, B); x7 = __ffma2_rn(x7, A, B);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] =
      x0.x + x1.x + x2.x + x3.x + x4.x + x5.x + x6.x + x7.x + x0.y + x1.y + x2.y + x3.y + x4.y + x5.y + x6.y + x7.y;
}

// distinct doubles built with integer operations, converted and summed in FP32
__global__ void p_d2f(float* out, int seed) {
  const int hi0 = 0x3ff00000 + (threadIdx.x & 1023), lo0 = seed + threadIdx.x;
  float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int i = 0; i < IT; ++i) {
    s0 += __double2float_rn(__hiloint2double(hi0, lo0 + i));
    s1 += __double2float_rn(__hiloint2double(hi0, lo0 + 2 * i));
    s2 += __double2float_rn(__hiloint2double(hi0, lo0 + 3 * i));
    s3 += __double2float_rn(__hiloint2double(hi0, lo0 + 5 * i));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s0 + s1 + s2 + s3;
}

}  // namespace

int main() {
  int dev = 0, nsm = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 512, blocks = nsm * 4;
  const size_t n = (size_t)threads * blocks;
  void* buf = nullptr;
  if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time = [&](auto launch) {
    float ms = 0.f;
    launch();  // warm
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms * 1e-3;
  };
  const double tdf = time([&] { p_dfma<<<blocks, threads>>>(static_cast<double*>(buf), 1.0000001, 1e-9); });
  const double tff = time([&] { p_ffma<<<blocks, threads>>>(static_cast<float*>(buf), 1.0000001f, 1e-9f); });
  const double tf2 = time([&] { p_ffma2<<<blocks, threads>>>(static_cast<float*>(buf), 1.0000001f, 1e-9f); });
  const double tcv = time([&] { p_d2f<<<blocks, threads>>>(static_cast<float*>(buf), 7); });
  const cudaError_t err = cudaGetLastError();
  cudaFree(buf);
  if (err != cudaSuccess) {
    std::printf("{\"error\": \"%s\"}\n", cudaGetErrorString(err));
    return 1;
  }
  std::printf("{\"fp64_fma_per_s\": %.6e, \"fp32_fma_per_s\": %.6e, \"fp32x2_lane_fma_per_s\": %.6e, "
              "\"f64_to_f32_per_s\": %.6e, \"sms\": %d, \"clock_mhz\": %.1f}\n",
              (double)n * IT * 8 / tdf, (double)n * IT * 64 / tff, (double)n * IT * 64 / tf2,
              (double)n * IT * 4 / tcv, nsm, clk_khz / 1000.0);
  return 0;
}
